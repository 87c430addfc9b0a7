/*
 * slabhash.h - C ABI of libslabhash.so, a GB300 (sm_103a) implementation of the
 * slab hash: a dynamic GPU hash table with chaining whose lists are slab lists
 * served by warp-cooperative work sharing (WCWS), with SlabAlloc extending the
 * lists (Ashkiani, Farach-Colton, Owens, "A Dynamic Hash Table for the GPU",
 * arXiv 1710.11246).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Pointers named d_* are CUDA device pointers on the device that was current
 *   when the table was created. Pointers named h_* are host pointers. The caller
 *   owns every batch array and keeps it alive until the work queued on `stream`
 *   has completed. The table owns its slabs, pool, bitmaps and counters.
 * - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *   stream. Batch calls are asynchronous: they queue kernels and return.
 * - Return value: SLAB_OK, or an error code for bad arguments (nothing queued)
 *   and for CUDA launch or copy failures. Errors that happen on the device
 *   while a batch runs (a sentinel key, an exhausted pool, an iteration cap
 *   reached) do not stop the batch; they set bits in the table's device status
 *   word, read and cleared by slab_status().
 * - Keys are uint32 in [0, 2^32 - 3]. 0xFFFFFFFF marks an empty slot and
 *   0xFFFFFFFE a deleted one (Sec. 3.2, footnote on the two reserved key
 *   values); an op on either is skipped and reported as SLAB_FLAG_RESERVED_KEY.
 * - Batch results are defined when each key appears in at most one op of a
 *   batch. Ops of one batch are concurrent (Sec. 6.3): with repeated keys every
 *   outcome is one of the serial orders of those ops.
 * - A table handle is not thread-safe: issue its calls from one host thread.
 */
#ifndef SLABHASH_H
#define SLABHASH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct slab_table slab_table; /* opaque, library-owned */

/* Element types (Sec. 4.2 "Choice of parameters"): 64-bit key-value pairs, 15 per
 * 128-byte slab (even lanes keys, odd lanes values), or 32-bit keys, 30 per slab. */
enum slab_mode { SLAB_MODE_KEY_VALUE = 0, SLAB_MODE_KEY_ONLY = 1 };

/* uint8 op codes of a mixed batch (Sec. 6.3 concurrent benchmark). */
enum slab_op { SLAB_OP_INSERT = 0, SLAB_OP_DELETE = 1, SLAB_OP_SEARCH = 2 };

enum slab_rc {
    SLAB_OK = 0,
    SLAB_ERR_INVALID_ARG = 1,
    SLAB_ERR_RESERVED_KEY = 2, /* a batch held a sentinel key */
    SLAB_ERR_OUT_OF_SLABS = 3, /* SlabAlloc found no free slab */
    SLAB_ERR_ITER_LIMIT = 4,   /* an op hit the per-op iteration cap */
    SLAB_ERR_CUDA = 5,
    SLAB_ERR_CORRUPT = 6,      /* a list held a next pointer outside the pool */
    SLAB_ERR_BUSY = 7          /* serving: no free slot, or the request has not finished */
};

/* Bits of the device status word (see slab_status). */
#define SLAB_FLAG_RESERVED_KEY 0x1u
#define SLAB_FLAG_OUT_OF_SLABS 0x2u
#define SLAB_FLAG_ITER_LIMIT 0x4u
#define SLAB_FLAG_BAD_POINTER 0x8u /* an op met a next pointer outside the pool and stopped */

#define SLAB_EMPTY_KEY 0xFFFFFFFFu     /* empty slot; also the empty next pointer */
#define SLAB_TOMBSTONE_KEY 0xFFFFFFFEu /* deleted slot */
#define SLAB_NOT_FOUND 0xFFFFFFFFu     /* search result for a missing key */
#define SLAB_HASH_PRIME 4294967291u    /* p = 2^32 - 5 in h(k) = ((a k + b) mod p) mod B */

/* Kernel families (see slab_config). */
enum slab_variant {
    SLAB_VARIANT_STAGED = 0, /* default: per-warp op window, slabs staged in shared memory */
    SLAB_VARIANT_DIRECT = 1  /* the Fig. "alg:search" loop: one op per lane, global reads */
};

/* Launch and safety parameters of one table. */
typedef struct slab_config {
    int32_t variant;           /* enum slab_variant */
    int32_t threads_per_block; /* multiple of 32, 32..1024 */
    int32_t blocks_per_sm;     /* resident blocks per SM used to size the persistent grid; 0 = occupancy maximum */
    uint32_t iter_limit;       /* cap on slab reads and retries of one op; reaching it ends the op with SLAB_FLAG_ITER_LIMIT */
    uint32_t random_probes;    /* per allocation: SlabAlloc block changes drawn by hash before a sweep of all blocks */
} slab_config;

/* Geometry of one table (read-only). */
typedef struct slab_info {
    uint32_t num_buckets;        /* B: base slabs */
    int32_t mode;                /* enum slab_mode */
    uint32_t elements_per_slab;  /* M: 15 or 30 (128-byte slabs), 7 or 14 (64-byte slabs) */
    uint32_t hash_a, hash_b;     /* universal hash parameters */
    uint64_t pool_slabs;         /* SlabAlloc memory units (multiple of 1024) */
    uint32_t num_memory_blocks;  /* pool_slabs / 1024 */
    uint32_t blocks_per_super;   /* memory blocks per super block in the 32-bit address (2^14) */
    uint32_t num_super_blocks;   /* ceil(num_memory_blocks / blocks_per_super) */
    uint32_t sm_count;
    uint64_t device_bytes;       /* bytes the table holds on the device */
    int32_t multiset;            /* 1: duplicates allowed (slab_set_multiset) */
    int32_t slab_bytes;          /* 128 or 64 (slab_create_width) */
} slab_info;

/*
 * Create an empty slab hash with B = num_buckets base slabs (Sec. 3.3, a
 * direct-address table of B slab lists) and a SlabAlloc pool of `pool_slabs`
 * 128-byte memory units (Sec. 5), rounded up to whole memory blocks of 1024
 * units. hash_a in [1, p-1] and hash_b in [0, p-1] are the random parameters
 * of h(k; a, b) = ((a k + b) mod p) mod B, p = 2^32 - 5 (Sec. 3.3); the caller
 * draws them. All super blocks sit in one contiguous allocation (the
 * "SlabAlloc-light" layout of Sec. 5, used in the paper's experiments, Sec. 6),
 * so a 32-bit slab address decodes with one multiply-add.
 * Errors: SLAB_ERR_INVALID_ARG for num_buckets = 0, a bad mode, a or b out of
 * range, pool_slabs = 0, or more than 2^32 - 2 slabs in total; SLAB_ERR_CUDA
 * if device memory cannot be allocated. On success *out owns device memory
 * until slab_destroy. The table starts empty (as after slab_reset).
 */
int slab_create(uint32_t num_buckets, int mode, uint32_t hash_a, uint32_t hash_b,
                uint64_t pool_slabs, slab_table **out);

/*
 * slab_create with the slab width as a parameter: slab_bytes = 128 (the paper's
 * slab, as slab_create) or 64. Sec. 4.2 sizes the slab to the warp's access
 * width (32 lanes x 4 bytes) and keeps its last two words for the auxiliary word
 * and the next pointer; a 64-byte slab is that layout at 16 words: 7 pairs at
 * even words 0..12 with their values after them (key-value mode) or 14 keys at
 * words 0..13 (key-only mode), the auxiliary word at 14 and the next pointer at
 * 15. The SlabAlloc pool then holds 64-byte memory units (still 1024 per memory
 * block, same bitmaps and addresses). Every batch call, slab_reset, slab_stats,
 * slab_export, slab_bucket_of, the SlabAlloc calls, slab_grow_pool,
 * slab_chain_histogram_noalloc, the learned bucket function, the serving loop
 * and groups take 64-byte tables; the paper-structured variant
 * (SLAB_VARIANT_DIRECT), multiset tables, SEARCHALL / DELETEALL and FLUSH
 * return SLAB_ERR_INVALID_ARG for them. Other errors as slab_create; a slab_bytes other
 * than 64 or 128 is SLAB_ERR_INVALID_ARG.
 */
int slab_create_width(uint32_t num_buckets, int mode, uint32_t slab_bytes, uint32_t hash_a, uint32_t hash_b,
                      uint64_t pool_slabs, slab_table **out);

/* The universal hash parameters drawn from a seed (Sec. 3.3 "a, b random"):
 * with x1, x2 the first two outputs of SplitMix64 seeded with `seed`,
 * a = 1 + x1 mod (p - 1) and b = x2 mod p. Host only; SLAB_ERR_INVALID_ARG for
 * NULL outputs. slab_create_seeded = slab_hash_params + slab_create; the drawn
 * parameters are reported by slab_get_info. */
int slab_hash_params(uint64_t seed, uint32_t *hash_a, uint32_t *hash_b);
int slab_create_seeded(uint32_t num_buckets, int mode, uint64_t seed, uint64_t pool_slabs, slab_table **out);

/* Free the table's device memory. Waits for the device first. NULL is a no-op. */
void slab_destroy(slab_table *t);

/* Empty the table: every slot and next pointer EMPTY, every SlabAlloc bitmap
 * bit clear, status word zero. One kernel on `stream` that refills the base
 * slabs and only the pool slabs the bitmaps mark as allocated: free pool slabs
 * always hold only EMPTY words (so slab_free_batch requires empty slabs). */
int slab_reset(slab_table *t, void *stream);

/* Geometry of the table. */
int slab_get_info(const slab_table *t, slab_info *out);

/* Current launch parameters; and replacing them (validated; SLAB_ERR_INVALID_ARG
 * leaves the old ones). */
int slab_get_config(const slab_table *t, slab_config *out);
int slab_set_config(slab_table *t, const slab_config *cfg);

/*
 * Bulk build / incremental insertion: REPLACE(k, v) for each of the n pairs
 * (Sec. 3.2 "Insertion", Sec. 4.3.2): if k is present its value is replaced,
 * otherwise the pair takes the first empty slot of its list, and a full list
 * grows by one SlabAlloc slab linked by a 32-bit CAS on the tail's next
 * pointer. Deleted slots are not reused, so keys stay unique (Sec. 3.2). An
 * insert that finds no free slab while other ops of the batch hold new slabs
 * not yet linked tries again in a later round; only when a search of every
 * memory block finds none does it end with SLAB_FLAG_OUT_OF_SLABS (the op's
 * found byte is then 0 and the pair is not stored; slab_status reports it).
 * d_keys, d_values: n uint32 each (d_values ignored in key-only mode, may be
 * NULL there). d_found (nullable): n bytes, 1 if the key was already present
 * (its value replaced), else 0.
 */
int slab_insert_batch(slab_table *t, const uint32_t *d_keys, const uint32_t *d_values,
                      uint8_t *d_found, uint32_t n, void *stream);

/*
 * DELETE(k) for each of the n keys (Sec. 3.2 "Deletion", Sec. 4.3.3): the slot
 * holding k gets the tombstone key; a missing key is not an error.
 * d_found (nullable): n bytes, 1 if k was present and deleted, else 0.
 */
int slab_delete_batch(slab_table *t, const uint32_t *d_keys, uint8_t *d_found, uint32_t n,
                      void *stream);

/*
 * SEARCH(k) for each of the n keys (Sec. 3.2 "Search", Sec. 4.3.1): the value
 * stored with k, or SLAB_NOT_FOUND. In key-only mode the value is 0 on a hit.
 * d_values_out: n uint32. d_found (nullable): n bytes, 1 on a hit; it tells a
 * stored value 0xFFFFFFFF apart from a miss. The table is read-only during the
 * batch, so slab reads may use the non-coherent cache path.
 */
int slab_search_batch(slab_table *t, const uint32_t *d_keys, uint32_t *d_values_out,
                      uint8_t *d_found, uint32_t n, void *stream);

/*
 * Concurrent batch (Sec. 6.3): op i is d_ops[i] (enum slab_op) on d_keys[i]
 * with d_values[i] (inserts only; may be NULL in key-only mode). One kernel
 * serves all three kinds; any mix can share a warp. d_results[i]:
 *   search -> the value or SLAB_NOT_FOUND (0 on a key-only hit);
 *   insert -> 1 if the key was new, 0 if an existing value was replaced;
 *   delete -> 1 if the key was deleted, 0 if it was absent.
 * d_found (nullable): 1 iff the key was present when op i took effect.
 * An op code > 2 is skipped (result 0).
 */
int slab_mixed_batch(slab_table *t, const uint8_t *d_ops, const uint32_t *d_keys,
                     const uint32_t *d_values, uint32_t *d_results, uint8_t *d_found,
                     uint32_t n, void *stream);

/*
 * Synchronize `stream`, then read and clear the device status word.
 * *h_flags (nullable) receives the SLAB_FLAG_* bits that were set. Returns
 * SLAB_OK if none were set, else the most serious of SLAB_ERR_CORRUPT,
 * SLAB_ERR_OUT_OF_SLABS, SLAB_ERR_ITER_LIMIT, SLAB_ERR_RESERVED_KEY, in that
 * order.
 */
int slab_status(slab_table *t, void *stream, uint32_t *h_flags);

/*
 * Chain statistics, one warp per bucket. d_slots (nullable): B uint32, used
 * slots of each list (live plus tombstones). d_slabs (nullable): B uint32,
 * slabs of each list (base slab included). h_totals (nullable): 6 uint64 =
 * {live elements, used slots, slabs, pool slabs marked allocated in the
 * bitmaps, lists whose used slots are not a prefix in (slab, lane) order
 * (always 0 for a set table; a multiset table's deletes leave holes), slabs
 * linked from a list}. Memory utilization (Sec. 3.3) is
 * (x / 128) * live / slabs with x = 8 (pairs) or 4 (keys). Synchronizes
 * `stream` when h_totals is given.
 */
int slab_stats(slab_table *t, uint32_t *d_slots, uint32_t *d_slabs, uint64_t *h_totals,
               void *stream);

/*
 * Every live element as (bucket, key, value), compacted in no particular
 * order. At most `capacity` are written; *h_count receives the number of live
 * elements (which may exceed capacity). d_buckets and d_values are nullable.
 * Synchronizes `stream`.
 */
int slab_export(slab_table *t, uint32_t *d_buckets, uint32_t *d_keys, uint32_t *d_values,
                uint64_t capacity, uint64_t *h_count, void *stream);

/*
 * Learned bucket function (a library extension; the paper hashes with the
 * universal hash of Sec. 3.3). A two-level piecewise-linear model of the key
 * set's CDF in FP32: a root line maps a key to one of 1024 leaves, the leaf's line
 * maps it to a bucket; each line is evaluated as fl(fl(a * x) + b) with x the key
 * rounded to float, floored and clamped. Model: 2 + 2 * 1024 floats (root a, b,
 * then a, b per leaf).
 *
 * slab_learn_buckets fits the model on the sample keys[0], keys[s], keys[2s], ...
 * (s = sample_stride; at most 2^20 sample keys): the sample is sorted; the root
 * fits leaf position i * 1024 / m against the i-th smallest of the m sample keys
 * by least squares, and each leaf fits bucket position i * B / m over the sample
 * keys the root sends to it (a leaf with none is flat where they would start).
 * Least-squares moments are exact integer sums over the targets scaled by m;
 * each line is a = (n Sxy - Sx Sy) / (n Sxx - Sx^2) / m,
 * b = ((Sy - a m Sx) / n) / m in correctly rounded double, then rounded to float
 * (flat at the mean when all x are equal). It
 * then counts, for all n keys, the slabs per bucket each function would give
 * (max(1, ceil(load / M))) and reports mean and maximum for both. Policy:
 * SLAB_LEARN_AUTO uses the model only if neither its mean nor its maximum is
 * worse than the universal hash's; SLAB_LEARN_ALWAYS uses it; SLAB_LEARN_MEASURE
 * keeps the universal hash. The table must hold no keys (call it after create or
 * slab_reset, before inserting): SLAB_ERR_INVALID_ARG otherwise. Uses
 * stream-ordered device scratch (sample + one counter per bucket) and
 * synchronizes `stream`.
 */
enum slab_learn_policy { SLAB_LEARN_AUTO = 0, SLAB_LEARN_ALWAYS = 1, SLAB_LEARN_MEASURE = 2 };
typedef struct slab_learn_report {
    uint32_t sample_size;          /* m */
    uint32_t use_learned;          /* bucket function now in use: 1 the model, 0 the universal hash */
    uint32_t max_slabs_learned, max_slabs_universal;
    double mean_slabs_learned, mean_slabs_universal;
} slab_learn_report;
int slab_learn_buckets(slab_table *t, const uint32_t *d_keys, uint32_t n, uint32_t sample_stride, int policy,
                       slab_learn_report *out, void *stream);

/* Copy the fitted model (2 + 2 * 1024 floats) to h_model; *h_in_use (nullable)
 * receives 1 if the table's buckets come from it. */
int slab_get_model(const slab_table *t, float *h_model, uint32_t *h_in_use);

/* The bucket of each of n keys as the batch kernels compute it: h(k) (Sec. 3.3),
 * or the learned model when the table uses it. d_buckets_out: n uint32. */
int slab_bucket_of(slab_table *t, const uint32_t *d_keys, uint32_t *d_buckets_out, uint32_t n,
                   void *stream);

/*
 * SlabAlloc allocation microbenchmark (Sec. 5: one 128-byte slab allocation
 * per thread). n requests, one per lane. With SLAB_VARIANT_DIRECT each warp
 * serves its lanes' requests one at a time as in the paper (ballot over the
 * resident block's register bitmaps, one atomic on the owning bitmap word,
 * resident change by hash when full); with SLAB_VARIANT_STAGED (the default)
 * the k-th lane holding a free bit claims it for the k-th requesting lane, so a
 * warp's 32 requests take one atomic round trip instead of 32. d_addrs_out: n uint32 slab addresses (unit bits [0,10), memory block
 * [10,24), super block [24,32)), or SLAB_EMPTY_KEY where the pool was
 * exhausted (and SLAB_FLAG_OUT_OF_SLABS set). The slabs are not linked into
 * any list; free them with slab_free_batch or slab_reset.
 */
int slab_alloc_batch(slab_table *t, uint32_t *d_addrs_out, uint32_t n, void *stream);

/* SlabAlloc deallocation (Sec. 5): clear the bitmap bit of each of n slab
 * addresses (SLAB_EMPTY_KEY entries are skipped). The slabs must hold only
 * empty slots, as slabs from slab_alloc_batch do. */
int slab_free_batch(slab_table *t, const uint32_t *d_addrs, uint32_t n, void *stream);

/* Copy the SlabAlloc bitmaps (32 uint32 words per memory block, bit u%32 of
 * word u/32 set iff unit u of that block is allocated) to d_dst. n_words must
 * equal 32 * num_memory_blocks. */
int slab_copy_bitmaps(const slab_table *t, uint32_t *d_dst, uint64_t n_words, void *stream);

/*
 * Slab-list length histogram and chain totals, with no device allocation at all.
 * The paper has no counterpart: this is a library service for callers that
 * cannot call cudaMalloc at the moment they need table statistics - a serving
 * loop whose device memory is fully reserved by another allocator (a fresh
 * cudaMalloc would fail or fragment that pool), or a latency-critical path that
 * cannot afford the device synchronization an allocation may cause. It walks
 * every list like slab_stats and counts buckets by slab count: h_hist[i]
 * (n_bins uint64, host) = buckets whose list has i + 1 slabs, the last bin
 * taking every longer list. h_totals (nullable, 6 uint64, host) = the
 * slab_stats totals. 1 <= n_bins <= 1024; a larger n_bins, or a current device
 * other than the table's, returns SLAB_ERR_INVALID_ARG.
 * It must be called outside CUDA stream capture: it ends by copying into host
 * memory and synchronizing `stream`, which a capturing stream does not allow,
 * so on a capturing stream (or on the legacy stream while another stream
 * captures) it returns SLAB_ERR_INVALID_ARG before enqueueing anything and the
 * capture stays valid.
 * Scratch: a fixed device array of 1032 uint64 (about 8 KiB) compiled into the
 * library; every GPU that loads the library holds it until the process exits.
 * slab_create resolves the array's device address on the table's device and
 * loads this call's kernels, so the call itself loads nothing on a device where
 * a table was created since the last device reset (a table of a group, on a
 * device where slab_create never ran, resolves the address on its first call).
 * The array is shared by all calls and keeps the last call's counts: each call
 * clears it on `stream` first, and calls that overlap on the GPU (other streams,
 * other host threads) race on it. Synchronizes `stream`. Calls no cudaMalloc,
 * cudaFree or other allocating routine.
 */
int slab_chain_histogram_noalloc(slab_table *t, uint32_t n_bins, uint64_t *h_hist, uint64_t *h_totals,
                                 void *stream);

/*
 * Multiset tables and the remaining operations of Sec. 3.2 / 4.3.4.
 *
 * slab_set_multiset: make a table that holds no keys (new, or after
 * slab_reset) a multiset (on = 1) or a set again (on = 0). In a multiset
 * table every insert (slab_insert_batch and the insert op of
 * slab_mixed_batch) is Sec. 3.2 INSERT: the pair goes into the first empty
 * slot of its list with no uniqueness check (found = 0, mixed result 1); a
 * delete removes the first instance met walking the list and empties its
 * slot, the whole pair at once, so later inserts reuse it (Sec. 3.2
 * "Deletion"). Search returns the first instance met. Within one batch each
 * key may appear in at most one op; a batch that both inserts and deletes in
 * the same bucket may leave an emptied slot behind a newly linked slab.
 * Not available for tables of a group. SLAB_ERR_INVALID_ARG if the table may
 * hold keys.
 *
 * slab_search_all_batch: SEARCHALL (Sec. 3.2) of n keys. d_counts[i]
 * receives how many live instances key i has; their values (0 in key-only
 * mode) go to d_values_out[i * max_per_key + j] for j < min(count,
 * max_per_key), in list order; the rest of the row is left as it was.
 * d_values_out holds n * max_per_key uint32 (may be NULL when max_per_key is
 * 0). Read-only: it may not share a batch window with writes to the table.
 *
 * slab_delete_all_batch: DELETEALL (Sec. 3.2): every live instance of each
 * key is removed (tombstone in a set table, emptied slot in a multiset
 * table); d_counts[i] (nullable) receives how many.
 *
 * slab_flush: FLUSH (Sec. 4.3.4) of every bucket, one warp per bucket: the
 * live elements keep their list order and move to the front of the list,
 * tombstones and emptied slots disappear, each list keeps max(1, ceil(live /
 * M)) slabs and the rest are emptied and returned to SlabAlloc. Must not run
 * concurrently with any other call on the table. *h_released (nullable; when
 * given, the call synchronizes `stream`) receives the number of slabs freed.
 *
 * slab_grow_pool: add ceil(extra_slabs / 1024) memory blocks to the SlabAlloc
 * pool (Sec. 5: more super blocks once the pool runs short). Existing slabs
 * keep their addresses; the table moves to a larger allocation. Synchronous:
 * waits for the device, and no other call may be in flight on the table.
 * SLAB_ERR_INVALID_ARG for a table of a group, extra_slabs = 0, or a pool
 * beyond the 32-bit address space; SLAB_ERR_CUDA if the allocation fails (the
 * table is left as it was).
 */
int slab_set_multiset(slab_table *t, int on);
int slab_search_all_batch(slab_table *t, const uint32_t *d_keys, uint32_t n, uint32_t max_per_key,
                          uint32_t *d_counts, uint32_t *d_values_out, void *stream);
int slab_delete_all_batch(slab_table *t, const uint32_t *d_keys, uint32_t *d_counts, uint32_t n, void *stream);
int slab_flush(slab_table *t, uint64_t *h_released, void *stream);
int slab_grow_pool(slab_table *t, uint64_t extra_slabs);

/*
 * Groups: many independent slab hashes served by one persistent launch (a library
 * extension; the paper runs one table). The tables' slabs, pools, bitmaps and
 * status words share one device arena owned by the group; each table keeps its
 * own B, hash parameters and pool and behaves exactly like a table from
 * slab_create. A batch for the group is one array of ops sorted by table:
 * d_op_start (device, ntables + 1 uint32, non-decreasing, d_op_start[0] = 0,
 * d_op_start[ntables] = total) gives table i the ops
 * [d_op_start[i], d_op_start[i + 1]); keys, values, results and found are as in
 * the single-table calls, indexed over the whole batch. One call queues a small
 * prefix-sum kernel and one persistent launch that serves tiles of 32 ops of one
 * table each, so the calls can be captured in a CUDA graph.
 */
typedef struct slab_group slab_group; /* opaque, library-owned */
int slab_group_create(uint32_t ntables, const uint32_t *h_num_buckets, const uint32_t *h_hash_a,
                      const uint32_t *h_hash_b, const uint64_t *h_pool_slabs, int mode, slab_group **out);
/* slab_group_create with every table of the group at slab width slab_bytes (128
 * or 64; see slab_create_width). */
int slab_group_create_width(uint32_t ntables, const uint32_t *h_num_buckets, const uint32_t *h_hash_a,
                            const uint32_t *h_hash_b, const uint64_t *h_pool_slabs, int mode, uint32_t slab_bytes,
                            slab_group **out);
/* Frees the arena and every table handle of the group. */
void slab_group_destroy(slab_group *g);
/* A handle to table i of the group, valid until the group is destroyed; every
 * single-table call accepts it (slab_destroy on it does nothing; the learned
 * bucket function is not available for tables of a group). */
int slab_group_table(slab_group *g, uint32_t i, slab_table **out);
int slab_group_get_config(const slab_group *g, slab_config *out);
/* threads_per_block, blocks_per_sm, iter_limit and random_probes apply to group launches. */
int slab_group_set_config(slab_group *g, const slab_config *cfg);
/* Empty every table of the group (one kernel). */
int slab_group_reset(slab_group *g, void *stream);
int slab_group_insert(slab_group *g, const uint32_t *d_op_start, const uint32_t *d_keys, const uint32_t *d_values,
                      uint8_t *d_found, uint32_t total, void *stream);
int slab_group_delete(slab_group *g, const uint32_t *d_op_start, const uint32_t *d_keys, uint8_t *d_found,
                      uint32_t total, void *stream);
int slab_group_search(slab_group *g, const uint32_t *d_op_start, const uint32_t *d_keys, uint32_t *d_values_out,
                      uint8_t *d_found, uint32_t total, void *stream);
int slab_group_mixed(slab_group *g, const uint32_t *d_op_start, const uint8_t *d_ops, const uint32_t *d_keys,
                     const uint32_t *d_values, uint32_t *d_results, uint8_t *d_found, uint32_t total, void *stream);
/* Synchronize `stream`, then read and clear every table's status word; *h_flags
 * (nullable) receives their OR; the return code ranks them as slab_status does. */
int slab_group_status(slab_group *g, void *stream, uint32_t *h_flags);

/*
 * Serving (a library extension; the paper benchmarks batches, not a request
 * loop). A server keeps one table resident and runs mixed-op requests on it:
 * it owns `slots` slots, each with its own CUDA stream, event, and pinned host
 * and device staging for max_request_ops ops. Work on a slot is one batch:
 * inputs to the device, one slab_mixed_batch, a one-block count of the
 * allocated pool slabs, outputs back. Batches on different slots overlap on
 * the device. slab_server_submit runs each request as its own batch;
 * slab_server_run serves a whole arrival trace with continuous batching (every
 * free slot takes all requests that have arrived, in order, as one batch).
 *
 * Admission by free SlabAlloc memory: a batch with k inserts (each links at
 * most one new slab) is admitted only if
 *     measured + reserved + k <= pool_high_water * pool_slabs,
 * where `measured` is the latest count of allocated pool slabs (each batch
 * counts the bitmaps after it ran, on its stream) and `reserved` sums the
 * inserts of batches whose count has not come back. Admitted batches run
 * concurrently (Sec. 6.3 concurrent semantics): a request's results equal its
 * results alone whenever no key of it is inserted or deleted by another
 * request in flight.
 *
 * The table must not be used by other calls while a server drives it, and a
 * server is not thread-safe.
 */
#define SLAB_SERVER_MAX_SLOTS 64u
#define SLAB_SERVER_MAX_REQUEST_OPS (1u << 24)
typedef struct slab_server slab_server; /* opaque, library-owned */
typedef struct slab_server_stats {
    uint64_t submitted;       /* requests admitted */
    uint64_t completed;       /* requests finished and handed back */
    uint64_t batches;         /* batches launched (one per submitted request, several requests per
                                 batch under slab_server_run) */
    uint64_t deferred_slot;   /* submit calls, or trace requests at the head of the queue, that
                                 found every slot busy */
    uint64_t deferred_memory; /* head-of-queue requests held back by the pool bound while others ran */
    uint64_t rejected_memory; /* requests refused: the pool bound failed with nothing in flight */
    uint64_t pool_grown;      /* pool growths (SLAB_SERVER_GROW_POOL) */
    uint64_t pool_slabs;      /* the table's pool size */
    uint64_t pool_measured;   /* latest allocated-slab count */
    uint64_t pool_reserved;   /* inserts of requests whose count is outstanding */
    uint32_t inflight;        /* slots holding a request */
    uint32_t pad;
} slab_server_stats;
/* t: a table on the current device (it may already hold keys); 1 <= slots <=
 * SLAB_SERVER_MAX_SLOTS; 1 <= max_request_ops <= SLAB_SERVER_MAX_REQUEST_OPS
 * (a slot's capacity: the largest request, and the largest batch
 * slab_server_run packs); 0 < pool_high_water <= 1; flags: any of
 * SLAB_SERVER_ZERO_COPY, SLAB_SERVER_GROW_POOL. Allocates the slots and measures the pool in use.
 * Errors: SLAB_ERR_INVALID_ARG for bad arguments or a table of another device;
 * SLAB_ERR_CUDA when an allocation fails (nothing is kept). */
#define SLAB_SERVER_ZERO_COPY 0x1u /* slab_server_run: kernels read and write page-locked, device-mapped
                                      caller arrays in place instead of copying them */
#define SLAB_SERVER_GROW_POOL 0x2u /* a request the pool bound refuses while nothing is in flight grows
                                      the pool (slab_grow_pool, by at least half) instead of failing;
                                      the table must own its memory (not a group's) */
int slab_server_create(slab_table *t, uint32_t slots, uint32_t max_request_ops, double pool_high_water,
                       uint32_t flags, slab_server **out);
/* Waits for every slot's stream, then frees the server (not the table). */
void slab_server_destroy(slab_server *sv);
/* Admit one request of n ops (host arrays, copied before the call returns;
 * op codes and semantics as slab_mixed_batch; h_values may be NULL in key-only
 * mode). On SLAB_OK *ticket names it. SLAB_ERR_BUSY: every slot holds a
 * request (collect one). SLAB_ERR_OUT_OF_SLABS: the pool bound refuses it now
 * (retry after collecting, or it will never fit if nothing is in flight).
 * Neither queues any work. SLAB_ERR_INVALID_ARG for n = 0 or n > max ops. */
int slab_server_submit(slab_server *sv, const uint8_t *h_ops, const uint32_t *h_keys, const uint32_t *h_values,
                       uint32_t n, uint64_t *ticket);
/* Hand back a request's results (n uint32 as slab_mixed_batch's d_results, n
 * found bytes; either pointer may be NULL) and free its slot. wait = 0 polls:
 * SLAB_ERR_BUSY while it runs. SLAB_ERR_INVALID_ARG for an unknown ticket. */
int slab_server_collect(slab_server *sv, uint64_t ticket, uint32_t *h_results, uint8_t *h_found, int wait);
int slab_server_get_stats(slab_server *sv, slab_server_stats *out);
/*
 * Serve a whole arrival trace on the calling thread: request r arrives
 * h_arrival_ns[r] nanoseconds after the call starts (non-decreasing) and owns
 * ops [h_op_start[r], h_op_start[r + 1]) of h_ops / h_keys / h_values
 * (h_op_start: n_requests + 1 entries, h_op_start[0] = 0; no request longer
 * than max_request_ops). Continuous batching: whenever a slot is free, the
 * requests that have arrived and are not yet running are packed in arrival
 * order, up to max_request_ops ops and the pool bound, into one batch on it;
 * a finished batch is retired as soon as its event fires. Data movement per
 * batch: with SLAB_SERVER_ZERO_COPY and page-locked, device-mapped caller
 * arrays (cudaHostAlloc / cudaHostRegister under unified addressing) the
 * kernels read the inputs and write the results in place; otherwise batches of
 * more than 8192 ops are copied by DMA straight between page-locked caller
 * arrays and device buffers, and the rest (and all pageable arrays) go through
 * the slot's pinned staging with one copy each way. Outputs (host, indexed like the
 * inputs; every pointer but h_status and h_arrival_ns/h_op_start nullable):
 * h_results / h_found per op; h_latency_ns[r] = retirement time - arrival;
 * h_wait_ns[r] = admission time - arrival; h_status[r] = SLAB_OK, or
 * SLAB_ERR_OUT_OF_SLABS for a request the pool could not take with nothing in
 * flight (not run; its outputs are untouched); *h_makespan_ns = time of the
 * last retirement. Requires no outstanding tickets (else SLAB_ERR_BUSY). On a
 * CUDA error every slot is drained and SLAB_ERR_CUDA is returned.
 */
int slab_server_run(slab_server *sv, uint64_t n_requests, const uint64_t *h_arrival_ns, const uint64_t *h_op_start,
                    const uint8_t *h_ops, const uint32_t *h_keys, const uint32_t *h_values, uint32_t *h_results,
                    uint8_t *h_found, uint64_t *h_latency_ns, uint64_t *h_wait_ns, uint8_t *h_status,
                    uint64_t *h_makespan_ns);

/*
 * A batch whose arrays live in host memory (a library service around the batch
 * calls above; the paper's batches start in device memory). kind is one of
 * enum slab_batch_kind; the arrays are those of the matching device call, in host
 * memory: h_keys (all kinds), h_values (insert and mixed; ignored in key-only
 * mode, required for inserts in key-value mode), h_ops (mixed), h_results
 * (search values, mixed results; not used by insert or delete), h_found
 * (nullable). Page-locked arrays (cudaHostAlloc, or pinned torch tensors) move at
 * the host link's full rate and leave the call asynchronous; pageable arrays
 * work, but their copies block the calling thread.
 * The call splits the batch into chunks of `chunk` ops (0: 2^22) and runs them in
 * order: each chunk's inputs are copied to device staging buffers owned by the
 * table (a ring of four sets of min(chunk, n) ops, 14 bytes per op each, made on
 * the first call and remade larger when a call needs more, which waits for the
 * device),
 * its batch runs on `stream`, and its results are copied back, the copies of one
 * chunk overlapping the kernels of its neighbours on internal copy streams. The
 * results equal those of the whole batch run at once: each key appears in at most
 * one op of a batch, and ops on distinct keys commute.
 * Completion: with done_event = NULL, `stream` completes only once every result
 * is in host memory (so a following batch on `stream` waits for these copies);
 * with a cudaEvent_t, the call records it after its last copy back and `stream`
 * does not wait for the copies, so the next batch can overlap them; the results
 * are in host memory once the event has completed. The host arrays must stay
 * valid until then. Not safe for concurrent calls on one table.
 * Errors: SLAB_ERR_INVALID_ARG for a bad kind or a missing required array;
 * SLAB_ERR_CUDA if staging cannot be allocated or a copy cannot be queued; the
 * device status word as for the device calls. n = 0 is a no-op.
 */
enum slab_batch_kind { SLAB_BATCH_INSERT = 0, SLAB_BATCH_DELETE = 1, SLAB_BATCH_SEARCH = 2, SLAB_BATCH_MIXED = 3 };
int slab_batch_host(slab_table *t, int kind, const uint8_t *h_ops, const uint32_t *h_keys, const uint32_t *h_values,
                    uint32_t *h_results, uint8_t *h_found, uint32_t n, uint32_t chunk, void *stream,
                    void *done_event);

/* Human-readable name of a return code. Never NULL. */
const char *slab_error_string(int rc);

/*
 * Roofline probes (measurement only; no table involved).
 *
 * slab_probe_random_lines: n_reads reads of whole 128-byte lines at uniformly
 * random line indices in [0, footprint_lines) of d_buf, one line per warp
 * access (32 lanes x 4 bytes), `lines_in_flight` independent lines per warp.
 * The xor of all words read lands in *d_sink (one uint32) so the reads cannot
 * be elided. d_buf must hold footprint_lines * 32 uint32.
 *
 * slab_probe_random_cas: n_ops 64-bit atomicCAS operations, each on one of
 * the 15 pair slots of a random line in [0, footprint_lines) of d_buf (which
 * holds footprint_lines * 16 uint64), expecting 0 and writing a nonzero value,
 * `ops_in_flight` independent CASes per thread. With d_buf zeroed and far more
 * slots than n_ops most CASes succeed, like an insert claiming an empty pair.
 */
int slab_probe_random_lines(const uint32_t *d_buf, uint64_t footprint_lines, uint64_t n_reads,
                            uint32_t seed, int lines_in_flight, int threads_per_block,
                            uint32_t *d_sink, void *stream);
/* slab_probe_random_lines_v4: n_reads random whole-line reads, each line read the
 * way the staged kernels move slabs, as 16-byte pieces, so one warp instruction
 * covers 128 / line_bytes * 4 lines (line_bytes = 128: four lines of 8 lanes;
 * 64: eight lines of 4 lanes). d_buf holds footprint_lines lines of line_bytes.
 * form 0: ld.global.cg.v4 into registers, lines_in_flight in {4, 8, 16, 32}
 * (at least one instruction's worth) lines issued per warp before any is
 * consumed. form 1: cp.async.cg 16-byte copies into a shared-memory stage of 32
 * lines per warp, lines_in_flight 32 (one stage, issued, waited for, consumed)
 * or 64 (two stages: the next 32 lines are issued before this round is
 * consumed). Same sink and error rules as above; an unsupported form, line size
 * or count returns SLAB_ERR_INVALID_ARG. */
int slab_probe_random_lines_v4(const uint32_t *d_buf, uint64_t footprint_lines, uint64_t n_reads,
                               uint32_t seed, int form, int line_bytes, int lines_in_flight, int threads_per_block,
                               uint32_t *d_sink, void *stream);
int slab_probe_random_cas(unsigned long long *d_buf, uint64_t footprint_lines, uint64_t n_ops,
                          uint32_t seed, int ops_in_flight, int threads_per_block, void *stream);
/* slab_probe_random_or: n_ops 32-bit atomicOr operations, each setting one random
 * bit of a random word in [0, footprint_words) of d_buf, `ops_in_flight` per
 * thread: the atomic a SlabAlloc claim issues on its bitmap word (Sec. 5). */
int slab_probe_random_or(uint32_t *d_buf, uint64_t footprint_words, uint64_t n_ops, uint32_t seed,
                         int ops_in_flight, int threads_per_block, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SLABHASH_H */
