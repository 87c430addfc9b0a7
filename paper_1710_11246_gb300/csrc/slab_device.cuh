// Device-side building blocks of the slab hash: slab layout, universal hash,
// coherent loads, and SlabAlloc (Sec. 5). Included by the kernel translation
// units only.
#pragma once
#include <cstdint>

namespace slab {

constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr uint32_t kEmptyKey = 0xFFFFFFFFu;   // empty slot and empty next pointer
constexpr uint32_t kTombstone = 0xFFFFFFFEu;  // deleted slot
constexpr uint32_t kNotFound = 0xFFFFFFFFu;
constexpr uint32_t kPrime = 4294967291u;      // 2^32 - 5
constexpr int kAddressLane = 31;              // lane holding the next pointer (Sec. 4.2)
constexpr uint32_t kWordsPerSlab = 32;        // 128-byte slab, one word per lane
constexpr uint32_t kUnitsPerBlock = 1024;     // memory units per memory block (Sec. 5)
constexpr uint32_t kBlocksPerSuper = 1u << 14;

// Key lanes of a slab: even lanes 0..28 for 15 pairs, lanes 0..29 for 30 keys.
constexpr uint32_t kKeyLanesKV = 0x15555555u;
constexpr uint32_t kKeyLanesKeyOnly = 0x3FFFFFFFu;

// Slab geometry for a slab of kW 4-byte words, kW = 32 (the paper's 128-byte
// slab) or 16 (a 64-byte slab). Sec. 4.2 keeps the last two words for the
// auxiliary word and the next pointer, so a key-value slab holds (kW - 2) / 2
// pairs (key at even words 0..kW-4, value after it) and a key-only slab kW - 2
// keys (words 0..kW-3).
template <uint32_t kW>
__host__ __device__ constexpr uint32_t next_word() { return kW - 1u; }
template <bool kKeyOnly, uint32_t kW>
__host__ __device__ constexpr uint32_t key_words() {
    return kKeyOnly ? ((1u << (kW - 2u)) - 1u) : (0x55555555u & ((1u << (kW - 3u)) - 1u));
}
template <bool kKeyOnly, uint32_t kW>
__host__ __device__ constexpr uint32_t elements_per_slab() { return kKeyOnly ? kW - 2u : (kW - 2u) / 2u; }
template <bool kKeyOnly, uint32_t kW>
__host__ __device__ constexpr uint32_t last_key_word() { return kKeyOnly ? kW - 3u : kW - 4u; }
static_assert(key_words<false, 32>() == kKeyLanesKV && key_words<true, 32>() == kKeyLanesKeyOnly,
              "the 128-byte layout");
static_assert(key_words<false, 16>() == 0x1555u && key_words<true, 16>() == 0x3FFFu, "the 64-byte layout");

enum : uint32_t { kFlagReserved = 1u, kFlagOutOfSlabs = 2u, kFlagIterLimit = 4u, kFlagBadPointer = 8u };
enum : uint8_t { kOpInsert = 0, kOpDelete = 1, kOpSearch = 2 };
// Kernel families by the ops they serve.
enum : int { kKindSearch = 0, kKindInsert = 1, kKindDelete = 2, kKindMixed = 3 };

struct TableView {
    uint32_t* slabs;      // B base slabs, then the SlabAlloc pool
    const float* model;   // learned bucket function (root a, b; 1024 leaves a, b)
    uint32_t* pool;       // slabs + B * slab_words: unit `a` of the pool at pool + a * slab_words
    uint32_t* bitmaps;    // 32 words per memory block
    uint32_t* status;     // device status word (kFlag*)
    uint64_t fastmod_m;   // ceil(2^64 / B) for the bucket reduction
    uint32_t num_buckets;
    uint32_t hash_a, hash_b;
    uint32_t num_blocks;  // memory blocks in the pool
    uint32_t pool_units;  // num_blocks * 1024: every valid pool address is below this
    uint32_t iter_limit;
    uint32_t random_probes;
    uint32_t epoch;       // distinct per launch; spreads resident blocks over launches
    uint32_t prefetch_l2; // staged kernels pull the next tile's base slabs into L2 (tables much larger than L2)
    uint32_t learned;     // 1: buckets come from the learned model, 0: from the universal hash
    uint32_t multiset;    // 1: duplicates allowed (INSERT, deletes empty their slot), 0: set (REPLACE, tombstones)
    uint32_t slab_words;  // words per slab: 32 (128-byte slabs) or 16 (64-byte slabs)
};

struct BatchArgs {
    const uint8_t* ops;
    const uint32_t* keys;
    const uint32_t* values;
    uint32_t* results;
    uint8_t* found;
    uint32_t n;
};

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

// h(k; a, b) = ((a k + b) mod p) mod B (Sec. 3.3). a k + b < 2^64 since a, b < p.
// mod p folds the high word with 2^32 = 5 (mod p) twice; mod B is Lemire, Kaser
// and Kurz's direct remainder ("Faster remainder by direct computation", 2019):
// with m = ceil(2^64 / B), n mod B = floor(((m n) mod 2^64) * B / 2^64) for
// every 32-bit n and B.
__device__ __forceinline__ uint32_t universal_bucket(const TableView& T, uint32_t k) {
    uint64_t x = (uint64_t)T.hash_a * k + T.hash_b;
    uint64_t t = (x >> 32) * 5ull + (x & 0xFFFFFFFFull);  // < 6 * 2^32
    t = (t >> 32) * 5ull + (t & 0xFFFFFFFFull);           // < 2^32 + 30
    uint32_t r = (uint32_t)(t >= kPrime ? t - kPrime : t);
    uint64_t low = T.fastmod_m * r;
    return (uint32_t)__umul64hi(low, (uint64_t)T.num_buckets);
}

// One linear piece of the learned bucket function, evaluated in FP32 with a
// separately rounded multiply and add (no fused multiply-add), then floored and
// clamped to [0, limit): p = a * x + b; NaN and negatives give 0.
__device__ __forceinline__ uint32_t linear_piece(float a, float b, float x, uint32_t limit) {
    const float p = __fadd_rn(__fmul_rn(a, x), b);
    if (!(p >= 0.0f)) return 0u;
    if (p >= __uint2float_rn(limit)) return limit - 1u;
    return (uint32_t)p;
}

// Learned bucket function: two-level piecewise-linear CDF of the key set. The root
// piece picks one of 1024 leaves, the leaf piece maps the key to a bucket.
__device__ __forceinline__ uint32_t learned_bucket(const float* model, uint32_t num_buckets, uint32_t k) {
    const float x = __uint2float_rn(k);
    const uint32_t leaf = linear_piece(__ldg(model), __ldg(model + 1), x, 1024u);
    return linear_piece(__ldg(model + 2 + 2 * leaf), __ldg(model + 3 + 2 * leaf), x, num_buckets);
}

__device__ __forceinline__ uint32_t bucket_of(const TableView& T, uint32_t k) {
    return T.learned ? learned_bucket(T.model, T.num_buckets, k) : universal_bucket(T, k);
}

// Slab word reads. Mutating kernels read through L2 with relaxed gpu-scope
// loads so that a re-read after a failed CAS sees other warps' writes; the
// search-only kernel may use the non-coherent path because nothing writes the
// table while it runs.
__device__ __forceinline__ uint32_t ld_coherent(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_readonly(const uint32_t* p) { return __ldg(p); }

template <bool kReadOnly>
__device__ __forceinline__ uint32_t ld_slab(const uint32_t* p) {
    if constexpr (kReadOnly) return ld_readonly(p);
    else return ld_coherent(p);
}

__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed64(uint32_t* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Remove the element whose key sits at word d of the slab at p (Sec. 3.2
// "Deletion"): a set table marks it deleted (the tombstone keeps later replaces
// from re-inserting a key further down the list); a multiset table empties it,
// the whole pair in one store, so a later insert can claim the slot.
template <bool kKeyOnly>
__device__ __forceinline__ void remove_at(const TableView& T, uint32_t* p, uint32_t d) {
    if (!T.multiset) st_relaxed(p + d, kTombstone);
    else if (kKeyOnly) st_relaxed(p + d, kEmptyKey);
    else st_relaxed64(p + d, ~0ull);
}

// The key an op's WCWS step matches: a multiset insert looks for an empty slot
// only (no uniqueness check, Sec. 3.2 INSERT); every other op for its own key.
__device__ __forceinline__ uint32_t match_key(const TableView& T, uint32_t key, uint32_t op) {
    return T.multiset && op == kOpInsert ? kEmptyKey : key;
}

// Streaming loads for the op arrays: each element is read once, so mark it
// evict-first (ld.global.cs) and keep it from displacing table lines in L2.
__device__ __forceinline__ uint32_t ld_stream(const uint32_t* p) { return __ldcs(p); }
__device__ __forceinline__ uint32_t ld_stream_u8(const uint8_t* p) { return __ldcs(p); }

__device__ __forceinline__ void set_flag(const TableView& T, uint32_t f) { atomicOr(T.status, f); }

// A next pointer read from a slab must name a pool unit; anything else means the
// table was overwritten from outside, and the op stops instead of reading out of
// bounds.
__device__ __forceinline__ bool valid_next(const TableView& T, uint32_t a) { return a < T.pool_units; }

__device__ __forceinline__ uint32_t* slab_ptr(const TableView& T, uint32_t bucket, uint32_t cur) {
    // cur == kEmptyKey means "the base slab of `bucket`", otherwise a pool address.
    // SlabAlloc-light decode (Sec. 5): the pool is contiguous and the 32-bit
    // address is the linear unit index (super block * 2^14 + block) * 1024 + unit.
    return cur == kEmptyKey ? T.slabs + (uint64_t)bucket * T.slab_words : T.pool + (uint64_t)cur * T.slab_words;
}

// --------------------------------------------------------------------------
// SlabAlloc (Sec. 5). Each warp owns a resident memory block; lane i keeps word i
// of its bitmap (units 32i..32i+31) in a register. An allocation ballots the
// lanes with a free bit, the lowest such lane claims its lowest free bit with one
// atomic on the global bitmap word and the address is broadcast by shuffle. When
// the block looks full the warp moves to another block chosen by hashing its
// global warp id with its count of resident changes; the new block's 32 bitmap
// words arrive in one coalesced 128-byte read.
// --------------------------------------------------------------------------
struct AllocCtx {
    uint32_t block;    // resident memory block, or kNoBlock (warp-uniform)
    uint32_t bitmap;   // this lane's word of the resident block's bitmap
    uint32_t changes;  // resident changes so far (warp-uniform)
};
constexpr uint32_t kNoBlock = 0xFFFFFFFFu;
constexpr uint32_t kAllocFailed = 0xFFFFFFFFu;
static_assert(kAllocFailed == kEmptyKey, "an unlinked next pointer reads as a failed allocation");
constexpr uint32_t kAllocRetry = 0xFFFFFFFEu;  // no slab this time; the pool may still have some

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    // murmur3 finalizer
    x ^= x >> 16;
    x *= 0x85EBCA6Bu;
    x ^= x >> 13;
    x *= 0xC2B2AE35u;
    x ^= x >> 16;
    return x;
}

__device__ __forceinline__ uint32_t resident_block(const TableView& T, uint32_t warp_gid,
                                                   uint32_t attempt) {
    // First `random_probes` changes: a hash of (warp id, attempt, launch epoch).
    // After that a sweep of every block from a hashed start, so that a pool with
    // any free unit left is always found before the allocation gives up.
    uint32_t seed = mix32(warp_gid * 0x9E3779B1u + T.epoch * 0x7F4A7C15u);
    if (attempt < T.random_probes) return mix32(seed ^ (attempt * 0x632BE5ABu)) % T.num_blocks;
    // start < num_blocks and the offset < num_blocks < 2^22: no wrap-around.
    return (seed % T.num_blocks + (attempt - T.random_probes)) % T.num_blocks;
}

// Returns a pool address, or kAllocFailed once every block has been probed.
// Each call may change the resident block random_probes + num_blocks times, so a
// call that gives up has swept every block, and a warp that met a momentarily
// full pool can allocate again later.
// Must be called by all 32 lanes with warp-uniform control flow.
__device__ __forceinline__ uint32_t warp_allocate(const TableView& T, AllocCtx& c, uint32_t warp_gid) {
    const uint32_t lane = lane_id();
    const uint32_t max_changes = T.random_probes + T.num_blocks;
    const uint32_t start = c.changes;
    for (;;) {
        if (c.block == kNoBlock) {
            if (c.changes - start >= max_changes) return kAllocFailed;
            c.block = resident_block(T, warp_gid, c.changes);
            c.changes++;
            c.bitmap = ld_coherent(T.bitmaps + (uint64_t)c.block * 32 + lane);
        }
        uint32_t free_lanes = __ballot_sync(kFull, c.bitmap != 0xFFFFFFFFu);
        if (free_lanes == 0) {
            c.block = kNoBlock;
            continue;
        }
        int src = __ffs(free_lanes) - 1;
        uint32_t addr = 0, ok = 0;
        if ((int)lane == src) {
            uint32_t bit = (uint32_t)(__ffs(~c.bitmap) - 1);
            uint32_t mask = 1u << bit;
            uint32_t old = atomicOr(T.bitmaps + (uint64_t)c.block * 32 + lane, mask);
            c.bitmap = old | mask;  // refresh from what the atomic saw
            ok = (old & mask) == 0;
            addr = (c.block << 10) | (lane << 5) | bit;
        }
        ok = __shfl_sync(kFull, ok, src);
        addr = __shfl_sync(kFull, addr, src);
        if (ok) return addr;
    }
}

// Batched allocation: every lane with `want` set receives its own pool address,
// or kAllocFailed once every block has been probed (the budget is per call, as
// above). Lane i owns word i of the resident block's bitmap, so in one round the
// k-th lane holding a free bit claims it for the k-th requesting lane (lane
// order), and up to 32 claims are in flight together instead of one per round
// trip. Losers of a bit race (the atomic found the bit already set) refresh
// their word and go round again.
// With `yield`, a call that has already handed out slabs does not move on when
// its block fills: the lanes still waiting get kAllocRetry. List growth uses
// this so that a warp never holds new slabs while it searches the pool for
// more; when many warps grow many lists at once, holding while searching can
// keep the pool full until every search gives up.
// Must be called by all 32 lanes with warp-uniform control flow.
__device__ __forceinline__ uint32_t warp_allocate_many(const TableView& T, AllocCtx& c, uint32_t warp_gid, bool want,
                                                       bool yield = false) {
    const uint32_t lane = lane_id();
    const uint32_t below = (1u << lane) - 1u;
    const uint32_t max_changes = T.random_probes + T.num_blocks;
    const uint32_t start = c.changes;
    uint32_t got = kAllocFailed;
    const uint32_t wanted = __ballot_sync(kFull, want);
    for (uint32_t pending = wanted; pending;) {
        if (c.block == kNoBlock) {
            if (yield && pending != wanted) {  // some lanes hold new slabs already
                if ((pending >> lane) & 1u) got = kAllocRetry;
                break;
            }
            if (c.changes - start >= max_changes) break;
            c.block = resident_block(T, warp_gid, c.changes);
            c.changes++;
            c.bitmap = ld_coherent(T.bitmaps + (uint64_t)c.block * 32 + lane);
        }
        const uint32_t free_lanes = __ballot_sync(kFull, c.bitmap != 0xFFFFFFFFu);
        if (free_lanes == 0) {
            c.block = kNoBlock;
            continue;
        }
        const uint32_t serve = min(__popc(free_lanes), __popc(pending));
        uint32_t addr = 0, ok = 0;
        if (((free_lanes >> lane) & 1u) && (uint32_t)__popc(free_lanes & below) < serve) {
            const uint32_t bit = (uint32_t)(__ffs(~c.bitmap) - 1);
            const uint32_t mask = 1u << bit;
            const uint32_t old = atomicOr(T.bitmaps + (uint64_t)c.block * 32 + lane, mask);
            c.bitmap = old | mask;  // refresh from what the atomic saw
            ok = (old & mask) == 0;
            addr = (c.block << 10) | (lane << 5) | bit;
        }
        // requester of rank r takes the result of the r-th free lane
        const uint32_t rank = __popc(pending & below);
        const bool mine = ((pending >> lane) & 1u) && rank < serve;
        const int src = mine ? (int)__fns(free_lanes, 0, (int)rank + 1) : (int)lane;
        const uint32_t a = __shfl_sync(kFull, addr, src);
        const uint32_t o = __shfl_sync(kFull, ok, src);
        if (mine && o) got = a;
        pending = __ballot_sync(kFull, want && got == kAllocFailed);
    }
    return got;
}

// Deallocation (Sec. 5): clear the unit's bit in its memory block's bitmap.
__device__ __forceinline__ void deallocate(const TableView& T, uint32_t addr) {
    uint32_t block = addr >> 10, word = (addr >> 5) & 31u, bit = addr & 31u;
    atomicAnd(T.bitmaps + (uint64_t)block * 32 + word, ~(1u << bit));
}

}  // namespace slab
