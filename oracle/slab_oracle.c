/*
 * Plain CPU oracle for the slab hash (Ashkiani, Farach-Colton, Owens,
 * "A Dynamic Hash Table for the GPU", arXiv 1710.11246).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path calls, links or loads
 * this file; only the tests, the smoke check and the benchmark's CPU-baseline
 * leg do. It shares no code, header or constant table with the CUDA library.
 *
 * What it computes is the plain definition of the data structure, not the
 * GPU algorithm:
 *   - B buckets (Sec. 3.3). Each bucket is an insertion-ordered array of
 *     slots (key, value, live). A slot is "used" once written and stays used:
 *     deletion only clears `live` (a tombstone, Sec. 3.2 "Deletion"), and a
 *     tombstoned slot is never written again, so keys stay unique.
 *   - h(k) = ((a k + b) mod p) mod B with plain 64-bit `%` (Sec. 3.3).
 *   - replace / delete / search with the set semantics of Sec. 3.2
 *     (replace = insert with uniqueness; delete and search act on the only
 *     live instance of k, since keys are unique).
 *   - Slab bookkeeping that follows from the slab layout of Sec. 4.2: M data
 *     elements per slab (M = 15 pairs or 30 keys), so a bucket with `len` used
 *     slots occupies max(1, ceil(len / M)) slabs, and the slot at position s
 *     lies in slab floor(s / M).
 *   - "Lines touched" per operation: how many slabs a lookup must read in
 *     list order before it stops (Sec. 3.2 search / replace / delete walks).
 *
 * Pins for every function live in tests/test_oracle_pins.py.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_NOT_FOUND 0xFFFFFFFFu /* value reported for a search miss */
#define OR_KEY_LIMIT 0xFFFFFFFEu /* keys >= this are the two reserved sentinels (Sec. 3.2 footnote) */
#define OR_PRIME 4294967291ull   /* 2^32 - 5 */

enum { OR_OP_INSERT = 0, OR_OP_DELETE = 1, OR_OP_SEARCH = 2 };

typedef struct {
    uint32_t key;
    uint32_t value;
    uint8_t live;
} or_slot;

typedef struct {
    or_slot *s;
    uint32_t len;
    uint32_t cap;
} or_bucket;

typedef struct {
    uint32_t B;        /* number of buckets (base slabs) */
    uint32_t M;        /* data elements per slab: 15 (key-value) or 30 (key only) */
    int key_only;
    uint64_t a, b, p;  /* universal hash parameters */
    or_bucket *bk;
    uint64_t live;     /* number of live elements */
    uint64_t reserved; /* ops skipped because their key was a sentinel */
} or_table;

/* Sec. 3.3: M = 15 pairs per 128-byte slab in key-value mode, 30 keys in key-only
 * mode (Sec. 4.2: lanes 0-29 hold data; lane 30 auxiliary; lane 31 next pointer). */
or_table *oracle_create(uint32_t num_buckets, int key_only, uint32_t a, uint32_t b)
{
    if (num_buckets == 0) return NULL;
    or_table *t = (or_table *)calloc(1, sizeof(or_table));
    if (!t) return NULL;
    t->B = num_buckets;
    t->key_only = key_only ? 1 : 0;
    t->M = key_only ? 30u : 15u;
    t->a = a;
    t->b = b;
    t->p = OR_PRIME;
    t->bk = (or_bucket *)calloc(num_buckets, sizeof(or_bucket));
    if (!t->bk) { free(t); return NULL; }
    return t;
}

void oracle_destroy(or_table *t)
{
    if (!t) return;
    for (uint32_t i = 0; i < t->B; i++) free(t->bk[i].s);
    free(t->bk);
    free(t);
}

/* Sec. 3.3: h(k; a, b) = ((a k + b) mod p) mod B. a, b < p < 2^32, so a k + b < 2^64. */
uint32_t oracle_hash(uint32_t a, uint32_t b, uint32_t num_buckets, uint32_t key)
{
    uint64_t x = (uint64_t)a * (uint64_t)key + (uint64_t)b;
    return (uint32_t)((x % OR_PRIME) % num_buckets);
}

uint32_t oracle_bucket(const or_table *t, uint32_t key)
{
    return oracle_hash((uint32_t)t->a, (uint32_t)t->b, t->B, key);
}

/* Position of the live slot holding `key` in bucket `bk`, or -1. */
static int64_t find_live(const or_bucket *bk, uint32_t key)
{
    for (uint32_t s = 0; s < bk->len; s++)
        if (bk->s[s].live && bk->s[s].key == key) return (int64_t)s;
    return -1;
}

static uint64_t slabs_of(const or_table *t, uint32_t len)
{
    return len == 0 ? 1 : (len + t->M - 1) / t->M;
}

static void append(or_bucket *bk, uint32_t key, uint32_t value)
{
    if (bk->len == bk->cap) {
        uint32_t nc = bk->cap ? bk->cap * 2 : 4;
        or_slot *ns = (or_slot *)realloc(bk->s, (size_t)nc * sizeof(or_slot));
        if (!ns) abort();
        bk->s = ns;
        bk->cap = nc;
    }
    bk->s[bk->len].key = key;
    bk->s[bk->len].value = value;
    bk->s[bk->len].live = 1;
    bk->len++;
}

/* Sec. 3.2 REPLACE: S <- (S - {<k,*>}) U {<k,v>}. If k is live, overwrite its value
 * in place; otherwise write a new slot at the tail of the list (first empty slot;
 * tombstones are not reused). Returns 1 if k was already present.
 * Lines: a hit at slot s reads slabs 0..s/M; a new key lands in slot len and reads
 * slabs 0..len/M (the last one freshly allocated when len is a multiple of M). */
static int op_replace(or_table *t, uint32_t key, uint32_t value, uint64_t *lines)
{
    or_bucket *bk = &t->bk[oracle_bucket(t, key)];
    if (t->key_only) value = 0;
    int64_t s = find_live(bk, key);
    if (s >= 0) {
        bk->s[s].value = value;
        if (lines) *lines += (uint64_t)s / t->M + 1;
        return 1;
    }
    if (lines) *lines += (uint64_t)bk->len / t->M + 1;
    append(bk, key, value);
    t->live++;
    return 0;
}

/* Sec. 3.2 DELETE: remove the (only) live <k,v>; the slot becomes a tombstone.
 * Returns 1 if k was present. A miss reads every slab of the list. */
static int op_delete(or_table *t, uint32_t key, uint64_t *lines)
{
    or_bucket *bk = &t->bk[oracle_bucket(t, key)];
    int64_t s = find_live(bk, key);
    if (s >= 0) {
        bk->s[s].live = 0;
        t->live--;
        if (lines) *lines += (uint64_t)s / t->M + 1;
        return 1;
    }
    if (lines) *lines += slabs_of(t, bk->len);
    return 0;
}

/* Sec. 3.2 SEARCH: return the live <k,v> or "not found". */
static int op_search(const or_table *t, uint32_t key, uint32_t *value, uint64_t *lines)
{
    const or_bucket *bk = &t->bk[oracle_bucket(t, key)];
    int64_t s = find_live(bk, key);
    if (s >= 0) {
        *value = t->key_only ? 0 : bk->s[s].value;
        if (lines) *lines += (uint64_t)s / t->M + 1;
        return 1;
    }
    *value = OR_NOT_FOUND;
    if (lines) *lines += slabs_of(t, bk->len);
    return 0;
}

/* Batches apply their ops one after another in index order. Under the batch
 * contract (each key in at most one op per batch) every order gives the same
 * results. found[i] = 1 iff the key was live just before op i. */
void oracle_insert(or_table *t, const uint32_t *keys, const uint32_t *values, uint64_t n,
                   uint8_t *found, uint64_t *lines)
{
    for (uint64_t i = 0; i < n; i++) {
        int f = 0;
        if (keys[i] >= OR_KEY_LIMIT) t->reserved++;
        else f = op_replace(t, keys[i], values ? values[i] : 0u, lines);
        if (found) found[i] = (uint8_t)f;
    }
}

void oracle_delete(or_table *t, const uint32_t *keys, uint64_t n, uint8_t *found, uint64_t *lines)
{
    for (uint64_t i = 0; i < n; i++) {
        int f = 0;
        if (keys[i] >= OR_KEY_LIMIT) t->reserved++;
        else f = op_delete(t, keys[i], lines);
        if (found) found[i] = (uint8_t)f;
    }
}

void oracle_search(or_table *t, const uint32_t *keys, uint64_t n, uint32_t *values,
                   uint8_t *found, uint64_t *lines)
{
    for (uint64_t i = 0; i < n; i++) {
        uint32_t v = OR_NOT_FOUND;
        int f = 0;
        if (keys[i] >= OR_KEY_LIMIT) t->reserved++;
        else f = op_search(t, keys[i], &v, lines);
        if (values) values[i] = v;
        if (found) found[i] = (uint8_t)f;
    }
}

/* Sec. 6.3 concurrent batch: one op per element. results[i]:
 *   search -> stored value, or OR_NOT_FOUND on a miss;
 *   insert -> 1 if the key was new, 0 if an existing value was replaced;
 *   delete -> 1 if the key was deleted, 0 if it was absent.
 * Unknown op codes are skipped (result 0, found 0). */
void oracle_mixed(or_table *t, const uint8_t *ops, const uint32_t *keys, const uint32_t *values,
                  uint64_t n, uint32_t *results, uint8_t *found, uint64_t *lines)
{
    for (uint64_t i = 0; i < n; i++) {
        uint32_t r = 0;
        int f = 0;
        if (ops[i] == OR_OP_SEARCH) r = OR_NOT_FOUND;
        if (ops[i] > OR_OP_SEARCH) {
            /* not an op */
        } else if (keys[i] >= OR_KEY_LIMIT) {
            t->reserved++;
        } else if (ops[i] == OR_OP_INSERT) {
            f = op_replace(t, keys[i], values ? values[i] : 0u, lines);
            r = f ? 0u : 1u;
        } else if (ops[i] == OR_OP_DELETE) {
            f = op_delete(t, keys[i], lines);
            r = (uint32_t)f;
        } else {
            f = op_search(t, keys[i], &r, lines);
        }
        if (results) results[i] = r;
        if (found) found[i] = (uint8_t)f;
    }
}

/* Per-bucket used slots (live + tombstoned) and slab counts, plus totals
 * {live, used slots, slabs, reserved-key ops}. */
void oracle_stats(const or_table *t, uint32_t *slots, uint32_t *slabs, uint64_t *totals)
{
    uint64_t used = 0, nslabs = 0;
    for (uint32_t i = 0; i < t->B; i++) {
        uint32_t len = t->bk[i].len;
        uint64_t k = slabs_of(t, len);
        if (slots) slots[i] = len;
        if (slabs) slabs[i] = (uint32_t)k;
        used += len;
        nslabs += k;
    }
    if (totals) {
        totals[0] = t->live;
        totals[1] = used;
        totals[2] = nslabs;
        totals[3] = t->reserved;
    }
}

/* Sec. 3.3 memory utilization: (x / (M x + y)) * n / sum_i k_i, with x the bytes
 * of one element (8 for a pair, 4 for a key), y = 8 bytes of lanes 30-31, and
 * k_i the number of slabs of bucket i. */
double oracle_utilization(const or_table *t)
{
    uint64_t tot[4];
    oracle_stats(t, NULL, NULL, tot);
    double x = t->key_only ? 4.0 : 8.0;
    double y = 8.0;
    return (x / (t->M * x + y)) * (double)tot[0] / (double)tot[2];
}

/* All live elements as (bucket, key, value), buckets in order, slots in list order. */
uint64_t oracle_export(const or_table *t, uint32_t *buckets, uint32_t *keys, uint32_t *values,
                       uint64_t cap)
{
    uint64_t c = 0;
    for (uint32_t i = 0; i < t->B; i++) {
        const or_bucket *bk = &t->bk[i];
        for (uint32_t s = 0; s < bk->len; s++) {
            if (!bk->s[s].live) continue;
            if (c < cap) {
                if (buckets) buckets[c] = i;
                if (keys) keys[c] = bk->s[s].key;
                if (values) values[c] = t->key_only ? 0u : bk->s[s].value;
            }
            c++;
        }
    }
    return c;
}

/*
 * SlabAlloc state check (Sec. 5 "SlabAlloc" and "Memory structure").
 *
 * A 32-bit slab address has the unit index within its memory block in bits
 * [0,10), the memory block within its super block in bits [10,24) and the
 * super block in bits [24,32). A memory block holds 1024 units and one 32-bit
 * bitmap word per 32 units: word w of a block covers units 32w .. 32w+31, bit
 * (unit mod 32) of it set iff that unit is allocated. Blocks are numbered
 * super block by super block, `blocks_per_super` to a super block.
 *
 * Given the addresses a set of allocations returned and the bitmap words the
 * allocator holds afterwards, checks that every address decodes to an existing
 * unit, that no address appears twice, and that the bitmaps mark exactly those
 * units. Returns 0 if all hold; 1 bad address, 2 duplicate, 3 bitmap mismatch.
 * *where receives the offending address index (1, 2) or bitmap word (3).
 */
int oracle_check_alloc(const uint32_t *addrs, uint64_t n, const uint32_t *bitmaps,
                       uint64_t num_blocks, uint32_t blocks_per_super, uint64_t *where)
{
    uint64_t words = num_blocks * 32;
    uint32_t *expect = (uint32_t *)calloc(words ? words : 1, sizeof(uint32_t));
    if (!expect) abort();
    int rc = 0;
    for (uint64_t i = 0; i < n && rc == 0; i++) {
        uint32_t a = addrs[i];
        uint32_t unit = a & 1023u;
        uint32_t blk = (a >> 10) & 0x3FFFu;
        uint32_t sb = a >> 24;
        uint64_t block = (uint64_t)sb * blocks_per_super + blk;
        if (blk >= blocks_per_super || block >= num_blocks) { rc = 1; *where = i; break; }
        uint64_t w = block * 32 + unit / 32;
        uint32_t bit = 1u << (unit % 32);
        if (expect[w] & bit) { rc = 2; *where = i; break; }
        expect[w] |= bit;
    }
    for (uint64_t w = 0; w < words && rc == 0; w++)
        if (expect[w] != bitmaps[w]) { rc = 3; *where = w; }
    free(expect);
    return rc;
}
