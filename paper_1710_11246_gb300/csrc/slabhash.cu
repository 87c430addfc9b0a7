// Host side of the slab-hash C ABI (include/slabhash.h) and the table's
// maintenance kernels: fill, chain statistics, export, hash, and the SlabAlloc
// allocation / deallocation batches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <atomic>
#include <mutex>
#include <new>
#include <type_traits>

#include "../../include/slabhash.h"
#include "slab_device.cuh"
#include "slab_staged.cuh"
#include "slab_table.cuh"
#include "slab_wcws.cuh"

using namespace slab;

namespace {

constexpr uint32_t kDefaultIterLimit = 1u << 22;
constexpr uint32_t kDefaultRandomProbes = 256;

using slab_host::counters;
using slab_host::launch_rc;
using slab_host::S;
using slab_host::util_grid;
using slab_host::view;

// Calls f(key_only, words_per_slab) with both as compile-time constants
// (std::integral_constant) for the table's mode and slab width.
template <class F>
int with_layout(int mode, uint32_t slab_words, F&& f) {
    using KO = std::true_type;
    using KV = std::false_type;
    using W16 = std::integral_constant<uint32_t, 16u>;
    using W32 = std::integral_constant<uint32_t, 32u>;
    const bool ko = mode == SLAB_MODE_KEY_ONLY;
    if (slab_words == 16u) return ko ? f(KO{}, W16{}) : f(KV{}, W16{});
    return ko ? f(KO{}, W32{}) : f(KV{}, W32{});
}

// Set-up of the no-allocation statistics call on device `dev` (defined with it at
// the end of this file): resolves its scratch array's device address and loads
// its kernels. Returns false on a CUDA error.
bool noalloc_setup(int dev);

bool valid_config(const slab_config& c) {
    return (c.variant == SLAB_VARIANT_STAGED || c.variant == SLAB_VARIANT_DIRECT) &&
           c.threads_per_block >= 32 && c.threads_per_block <= 1024 && c.threads_per_block % 32 == 0 &&
           c.blocks_per_sm >= 0 && c.blocks_per_sm <= 64 && c.iter_limit >= 1 && c.random_probes <= (1u << 20) &&
           // staged kernels hold one 4 KB stage per warp, plus up to 2.7 KB of keys, ballots and waiting ops
           (c.variant != SLAB_VARIANT_STAGED ||
            c.threads_per_block / 32 * kMixedWordsPerWarp<32u> * 4 <= 227 * 1024);
}

// The largest block every staged kernel of a mode and slab width can launch:
// their register caps put it below 1024 threads (65,536 registers per SM).
// Cached per layout.
int staged_block_limit(int mode, uint32_t slab_words) {
    static std::atomic<int> cached[2][2] = {{0, 0}, {0, 0}};
    const int m = mode == SLAB_MODE_KEY_ONLY ? 1 : 0, w = slab_words == 16u ? 1 : 0;
    int lim = cached[m][w].load(std::memory_order_relaxed);
    if (lim) return lim;
    lim = 1024;
    auto take = [&](const void* k) {
        cudaFuncAttributes a;
        if (cudaFuncGetAttributes(&a, k) == cudaSuccess) lim = std::min(lim, a.maxThreadsPerBlock);
        else cudaGetLastError();
    };
    with_layout(mode, slab_words, [&](auto ko, auto wd) {
        constexpr bool K = decltype(ko)::value;
        constexpr uint32_t W = decltype(wd)::value;
        take((const void*)staged_kernel<kKindSearch, K, W>);
        take((const void*)staged_kernel<kKindInsert, K, W>);
        take((const void*)staged_kernel<kKindDelete, K, W>);
        take((const void*)staged_kernel<kKindMixed, K, W>);
        return 0;
    });
    lim -= lim % 32;
    cached[m][w].store(lim, std::memory_order_relaxed);
    return lim;
}

// ------------------------------------------------------------------ kernels
__global__ void fill_kernel(uint4* slabs, uint64_t n16, uint4* bitmaps, uint64_t b16, uint32_t* misc) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint4 ones = make_uint4(kEmptyKey, kEmptyKey, kEmptyKey, kEmptyKey);
    const uint4 zero = make_uint4(0, 0, 0, 0);
    for (uint64_t i = tid; i < n16; i += stride) slabs[i] = ones;
    for (uint64_t i = tid; i < b16; i += stride) bitmaps[i] = zero;
    if (tid == 0) misc[0] = 0;
}

// Reset of a table in use: refill the base slabs with EMPTY and, through the
// bitmaps, exactly the pool slabs that are allocated, then clear the bitmaps.
// Pool slabs that are free always hold only EMPTY words: they are filled at
// create, written only after being allocated and linked, and a slab that lost its
// link race is freed unwritten.
__global__ void reset_kernel(uint4* base, uint64_t base16, uint4* pool, uint32_t* bitmaps, uint64_t words,
                             uint32_t pieces, uint32_t* misc) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint4 ones = make_uint4(kEmptyKey, kEmptyKey, kEmptyKey, kEmptyKey);
    for (uint64_t i = tid; i < base16; i += stride) base[i] = ones;
    // A warp per bitmap word: the word's 32 slabs are 32 * pieces 16-byte pieces
    // (pieces = 8 for 128-byte slabs, 4 for 64-byte ones), and store k of the warp
    // refills pieces 32k..32k+31, so one store instruction refills 32 / pieces slabs.
    const uint32_t lane = threadIdx.x & 31u;
    for (uint64_t w = tid >> 5; w < words; w += stride >> 5) {
        const uint32_t bits = bitmaps[w];  // the same word in every lane
        if (!bits) continue;                // warp-uniform
        __syncwarp();
        if (lane == 0) bitmaps[w] = 0;
        uint4* first = pool + ((w >> 5) * kUnitsPerBlock + (w & 31u) * 32u) * pieces;
        for (uint32_t k = lane; k < 32u * pieces; k += 32u) {
            const uint32_t slab = k / pieces;
            if ((bits >> slab) & 1u) first[k] = ones;
        }
    }
    if (tid == 0) misc[0] = 0;
}

// One warp per bucket: walk the list, count used and live key lanes and slabs,
// and check that used slots form a prefix in (slab, lane) order.
// Slabs of kW words: lane w reads word w (lanes kW and up see EMPTY).
template <bool kKeyOnly, uint32_t kW>
__global__ void stats_kernel(TableView T, uint32_t* slots, uint32_t* slabs, unsigned long long* acc) {
    constexpr uint32_t kMask = key_words<kKeyOnly, kW>();
    constexpr uint32_t kPerSlab = elements_per_slab<kKeyOnly, kW>();
    const uint32_t lane = lane_id();
    const uint32_t warp_gid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    unsigned long long live_sum = 0, used_sum = 0, slab_sum = 0, bad = 0, linked = 0;
    for (uint32_t b = warp_gid; b < T.num_buckets; b += nwarps) {
        uint32_t cur = kEmptyKey, used = 0, live = 0, n = 0;
        bool prefix_ok = true, prev_full = true;
        // a list can hold at most every pool slab plus its base slab
        for (uint64_t guard = 0; guard <= (uint64_t)T.num_blocks * kUnitsPerBlock; ++guard) {
            const uint32_t w = lane < kW ? ld_coherent(slab_ptr(T, b, cur) + lane) : kEmptyKey;
            const uint32_t u = __ballot_sync(kFull, w != kEmptyKey) & kMask;
            const uint32_t l = __ballot_sync(kFull, w != kEmptyKey && w != kTombstone) & kMask;
            const uint32_t cnt = __popc(u);
            // used lanes must be the lowest `cnt` key lanes, and only the last slab may be partial
            uint32_t want = 0, m = kMask;
            for (uint32_t i = 0; i < cnt; ++i) { want |= m & (0u - m); m &= m - 1u; }
            if (u != want || !prev_full) prefix_ok = false;
            prev_full = cnt == kPerSlab;
            used += cnt;
            live += __popc(l);
            ++n;
            const uint32_t nx = __shfl_sync(kFull, w, next_word<kW>());
            if (nx == kEmptyKey) break;
            if (!valid_next(T, nx)) {
                prefix_ok = false;
                break;
            }
            cur = nx;
        }
        if (lane == 0) {
            if (slots) slots[b] = used;
            if (slabs) slabs[b] = n;
        }
        live_sum += live; used_sum += used; slab_sum += n; linked += n - 1; bad += prefix_ok ? 0 : 1;
    }
    if (lane == 0) {
        atomicAdd(acc + 0, live_sum);
        atomicAdd(acc + 1, used_sum);
        atomicAdd(acc + 2, slab_sum);
        atomicAdd(acc + 4, bad);
        atomicAdd(acc + 5, linked);
    }
}

__global__ void popcount_kernel(const uint32_t* words, uint64_t n, unsigned long long* acc) {
    unsigned long long c = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        c += __popc(words[i]);
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(kFull, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(acc + 3, c);
}

template <bool kKeyOnly, uint32_t kW>
__global__ void export_kernel(TableView T, uint32_t* ob, uint32_t* ok, uint32_t* ov, uint64_t cap,
                              unsigned long long* count) {
    constexpr uint32_t kMask = key_words<kKeyOnly, kW>();
    const uint32_t lane = lane_id();
    const uint32_t warp_gid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t b = warp_gid; b < T.num_buckets; b += nwarps) {
        uint32_t cur = kEmptyKey;
        for (uint64_t guard = 0; guard <= (uint64_t)T.num_blocks * kUnitsPerBlock; ++guard) {
            const uint32_t w = lane < kW ? ld_coherent(slab_ptr(T, b, cur) + lane) : kEmptyKey;
            const uint32_t v = __shfl_down_sync(kFull, w, 1);
            const uint32_t l = __ballot_sync(kFull, w != kEmptyKey && w != kTombstone) & kMask;
            unsigned long long base = 0;
            if (lane == 0 && l) base = atomicAdd(count, (unsigned long long)__popc(l));
            base = __shfl_sync(kFull, base, 0);
            if ((l >> lane) & 1u) {
                const uint64_t at = base + __popc(l & ((1u << lane) - 1u));
                if (at < cap) {
                    ok[at] = w;
                    if (ob) ob[at] = b;
                    if (ov) ov[at] = kKeyOnly ? 0u : v;
                }
            }
            const uint32_t nx = __shfl_sync(kFull, w, next_word<kW>());
            if (nx == kEmptyKey || !valid_next(T, nx)) break;
            cur = nx;
        }
    }
}

__global__ void bucket_kernel(TableView T, const uint32_t* keys, uint32_t* out, uint32_t n) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = bucket_of(T, keys[i]);
}

// SlabAlloc microbenchmark: one request per lane. The paper's warp serves its
// requests one at a time (warp_allocate, one atomic round trip each); `batched`
// serves all 32 of a tile together (warp_allocate_many).
template <bool kBatched>
__global__ void alloc_kernel(TableView T, uint32_t* out, uint32_t n) {
    const uint32_t lane = lane_id();
    const uint32_t warp_gid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    AllocCtx ac{kNoBlock, 0u, 0u};
    bool failed = false;
    for (uint32_t tile = warp_gid; tile < (n + 31u) / 32u; tile += nwarps) {
        const uint32_t idx = tile * 32u + lane;
        uint32_t mine = kEmptyKey;
        if constexpr (kBatched) {
            mine = failed ? kAllocFailed : warp_allocate_many(T, ac, warp_gid, idx < n);
            failed = __any_sync(kFull, idx < n && mine == kAllocFailed);
        } else {
            uint32_t queue = __ballot_sync(kFull, idx < n);
            while (queue) {
                const int s = __ffs(queue) - 1;
                queue &= queue - 1u;
                const uint32_t a = failed ? kAllocFailed : warp_allocate(T, ac, warp_gid);
                if (a == kAllocFailed) failed = true;
                if ((int)lane == s) mine = a;
            }
        }
        if (idx < n) out[idx] = mine;
    }
    if (failed && lane == 0) set_flag(T, kFlagOutOfSlabs);
}

__global__ void free_kernel(TableView T, const uint32_t* addrs, uint32_t n) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t a = addrs[i];
        if (a != kEmptyKey && (a >> 10) < T.num_blocks) deallocate(T, a);
    }
}

// ------------------------------------------------------------ batch launch
#ifndef SLAB_PDL
#define SLAB_PDL 1
#endif
template <int kKind, bool kKeyOnly, uint32_t kW>
int launch_batch(slab_table* t, const BatchArgs& a, void* stream) {
    if (a.n == 0) return SLAB_OK;
    const TableView T = view(t);
    const int tpb = t->cfg.threads_per_block;
    const int wpb = tpb / 32;
    if (t->cfg.variant == SLAB_VARIANT_DIRECT) {
        if constexpr (kW != 32u) return SLAB_ERR_INVALID_ARG;  // refused by slab_set_config already
        auto k = direct_kernel<kKind, kKeyOnly>;
        int bps = t->cfg.blocks_per_sm;
        if (bps == 0) {  // the occupancy query costs microseconds: ask once per configuration
            int& occ = t->occupancy[SLAB_VARIANT_DIRECT][kKind];
            if (!occ && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, tpb, 0) != cudaSuccess)
                return SLAB_ERR_CUDA;
            bps = occ;
        }
        const uint64_t tiles = (a.n + 31u) / 32u;
        const uint64_t want = (tiles + wpb - 1) / wpb;
        const uint32_t grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)std::max(bps, 1) * t->sm_count));
        k<<<grid, tpb, 0, S(stream)>>>(T, a);
    } else {
        auto k = staged_kernel<kKind, kKeyOnly, kW>;
        const size_t smem = (size_t)wpb * kWordsPerWarp<kKind, kW> * 4;
        if ((int)smem > t->max_smem_optin) return SLAB_ERR_INVALID_ARG;
        if (smem > 48 * 1024 &&
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return SLAB_ERR_CUDA;
        int bps = t->cfg.blocks_per_sm;
        if (bps == 0) {
            int& occ = t->occupancy[SLAB_VARIANT_STAGED][kKind];
            if (!occ && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, tpb, smem) != cudaSuccess)
                return SLAB_ERR_CUDA;
            bps = occ;
        }
        const uint64_t tiles = (a.n + 31u) / 32u;
        const uint64_t want = (tiles + wpb - 1) / wpb;
        const uint64_t grid = std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)std::max(bps, 1) * t->sm_count));
        // Programmatic dependent launch: this grid may be scheduled while the
        // previous kernel on the stream drains; the kernel waits for that kernel
        // to complete (griddepcontrol.wait) before its first memory access.
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3((uint32_t)grid);
        lc.blockDim = dim3(tpb);
        lc.dynamicSmemBytes = smem;
        lc.stream = S(stream);
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = SLAB_PDL;
        lc.attrs = attr;
        lc.numAttrs = 1;
        if (cudaLaunchKernelEx(&lc, k, T, a) != cudaSuccess) return SLAB_ERR_CUDA;
    }
    return launch_rc();
}

template <int kKind>
int dispatch(slab_table* t, const BatchArgs& a, void* stream) {
    return with_layout(t->mode, t->slab_words, [&](auto ko, auto wd) {
        return launch_batch<kKind, decltype(ko)::value, decltype(wd)::value>(t, a, stream);
    });
}


// Every slab EMPTY, every bitmap word zero: the state of a new table.
int fill_table(slab_table* t, void* stream) {
    const uint64_t n16 = ((uint64_t)t->num_buckets + t->pool_slabs) * (t->slab_words / 4u);  // uint4 per 16 bytes
    const uint64_t b16 = (uint64_t)t->num_blocks * 8;
    fill_kernel<<<util_grid(t, n16, 256), 256, 0, S(stream)>>>(
        reinterpret_cast<uint4*>(t->d_slabs), n16, reinterpret_cast<uint4*>(t->d_bitmaps), b16, t->d_misc);
    return launch_rc();
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

const char* slab_error_string(int rc) {
    switch (rc) {
        case SLAB_OK: return "ok";
        case SLAB_ERR_INVALID_ARG: return "invalid argument";
        case SLAB_ERR_RESERVED_KEY: return "a batch held a reserved (sentinel) key";
        case SLAB_ERR_OUT_OF_SLABS: return "SlabAlloc pool exhausted";
        case SLAB_ERR_ITER_LIMIT: return "an op reached the iteration cap";
        case SLAB_ERR_CUDA: return "CUDA error";
        case SLAB_ERR_CORRUPT: return "a slab list held a next pointer outside the pool";
        case SLAB_ERR_BUSY: return "no free serving slot, or the request has not finished";
        default: return "unknown error";
    }
}

int slab_create_width(uint32_t num_buckets, int mode, uint32_t slab_bytes, uint32_t hash_a, uint32_t hash_b,
                      uint64_t pool_slabs, slab_table** out) {
    if (!out) return SLAB_ERR_INVALID_ARG;
    *out = nullptr;
    if (num_buckets == 0 || (mode != SLAB_MODE_KEY_VALUE && mode != SLAB_MODE_KEY_ONLY) ||
        (slab_bytes != 64u && slab_bytes != 128u) || hash_a == 0 || hash_a >= kPrime || hash_b >= kPrime ||
        pool_slabs == 0)
        return SLAB_ERR_INVALID_ARG;
    const uint64_t blocks = (pool_slabs + kUnitsPerBlock - 1) / kUnitsPerBlock;
    const uint64_t pool = blocks * kUnitsPerBlock;
    // every pool address must differ from the empty pointer, and the base slabs
    // plus the pool must be indexable by 32 bits
    if (blocks >= (1ull << 22) || (uint64_t)num_buckets + pool > 0xFFFFFFFEull) return SLAB_ERR_INVALID_ARG;

    slab_table* t = new (std::nothrow) slab_table();
    if (!t) return SLAB_ERR_CUDA;
    if (cudaGetDevice(&t->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&t->sm_count, cudaDevAttrMultiProcessorCount, t->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&t->max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, t->device) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&t->l2_bytes, cudaDevAttrL2CacheSize, t->device) != cudaSuccess) {
        delete t;
        return SLAB_ERR_CUDA;
    }
    t->num_buckets = num_buckets;
    t->mode = mode;
    t->slab_words = slab_bytes / 4u;
    t->hash_a = hash_a;
    t->hash_b = hash_b;
    t->fastmod_m = UINT64_MAX / num_buckets + 1;  // wraps to 0 for B = 1, which yields 0 as needed
    t->pool_slabs = pool;
    t->num_blocks = (uint32_t)blocks;
    const uint64_t all_slab_bytes = ((uint64_t)num_buckets + pool) * slab_bytes;
    const uint64_t bitmap_bytes = blocks * 128ull;
    if (cudaMalloc(&t->d_slabs, all_slab_bytes) != cudaSuccess) { delete t; cudaGetLastError(); return SLAB_ERR_CUDA; }
    const uint64_t model_bytes = (2 + 2 * 1024) * sizeof(float);
    if (cudaMalloc(&t->d_bitmaps, bitmap_bytes) != cudaSuccess ||
        cudaMalloc(&t->d_misc, 128) != cudaSuccess || cudaMalloc(&t->d_model, model_bytes) != cudaSuccess) {
        cudaFree(t->d_slabs);
        cudaFree(t->d_bitmaps);
        cudaFree(t->d_misc);
        delete t;
        cudaGetLastError();
        return SLAB_ERR_CUDA;
    }
    t->device_bytes = all_slab_bytes + bitmap_bytes + 128 + model_bytes;
    t->cfg.variant = SLAB_VARIANT_STAGED;
    t->cfg.threads_per_block = 128;
    t->cfg.blocks_per_sm = 0;
    t->cfg.iter_limit = kDefaultIterLimit;
    t->cfg.random_probes = kDefaultRandomProbes;
    if (cudaMemset(t->d_misc, 0, 128) != cudaSuccess || cudaMemset(t->d_model, 0, model_bytes) != cudaSuccess ||
        fill_table(t, nullptr) != SLAB_OK ||
        cudaDeviceSynchronize() != cudaSuccess || !noalloc_setup(t->device)) {
        slab_destroy(t);
        return SLAB_ERR_CUDA;
    }
    *out = t;
    return SLAB_OK;
}

int slab_create(uint32_t num_buckets, int mode, uint32_t hash_a, uint32_t hash_b, uint64_t pool_slabs,
                slab_table** out) {
    return slab_create_width(num_buckets, mode, 128u, hash_a, hash_b, pool_slabs, out);
}

// SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014): add the golden-ratio increment to the state, then
// two xor-shift-multiply rounds and a final xor-shift.
static uint64_t splitmix64(uint64_t& state) {
    uint64_t z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

int slab_hash_params(uint64_t seed, uint32_t* hash_a, uint32_t* hash_b) {
    if (!hash_a || !hash_b) return SLAB_ERR_INVALID_ARG;
    uint64_t st = seed;
    *hash_a = (uint32_t)(1 + splitmix64(st) % (kPrime - 1ull));
    *hash_b = (uint32_t)(splitmix64(st) % kPrime);
    return SLAB_OK;
}

int slab_create_seeded(uint32_t num_buckets, int mode, uint64_t seed, uint64_t pool_slabs, slab_table** out) {
    uint32_t a = 0, b = 0;
    slab_hash_params(seed, &a, &b);
    return slab_create(num_buckets, mode, a, b, pool_slabs, out);
}

void slab_destroy(slab_table* t) {
    if (!t || !t->owns_memory) return;  // tables of a group are freed with the group
    cudaDeviceSynchronize();
    slab_host::free_host_io(t);
    cudaFree(t->d_slabs);
    cudaFree(t->d_bitmaps);
    cudaFree(t->d_misc);
    cudaFree(t->d_model);
    delete t;
}

int slab_reset(slab_table* t, void* stream) {
    if (!t) return SLAB_ERR_INVALID_ARG;
    t->dirty = false;
    const uint32_t pieces = t->slab_words / 4u;  // 16-byte pieces per slab
    const uint64_t base16 = (uint64_t)t->num_buckets * pieces;
    const uint64_t words = (uint64_t)t->num_blocks * 32;
    reset_kernel<<<util_grid(t, std::max(base16, words), 256), 256, 0, S(stream)>>>(
        reinterpret_cast<uint4*>(t->d_slabs), base16,
        reinterpret_cast<uint4*>(t->d_slabs + (uint64_t)t->num_buckets * t->slab_words), t->d_bitmaps, words, pieces,
        t->d_misc);
    return launch_rc();
}

int slab_get_info(const slab_table* t, slab_info* out) {
    if (!t || !out) return SLAB_ERR_INVALID_ARG;
    out->num_buckets = t->num_buckets;
    out->mode = t->mode;
    out->elements_per_slab = t->mode == SLAB_MODE_KEY_ONLY ? t->slab_words - 2u : (t->slab_words - 2u) / 2u;
    out->hash_a = t->hash_a;
    out->hash_b = t->hash_b;
    out->pool_slabs = t->pool_slabs;
    out->num_memory_blocks = t->num_blocks;
    out->blocks_per_super = kBlocksPerSuper;
    out->num_super_blocks = (t->num_blocks + kBlocksPerSuper - 1) / kBlocksPerSuper;
    out->sm_count = (uint32_t)t->sm_count;
    out->device_bytes = t->device_bytes;
    out->multiset = t->multiset ? 1 : 0;
    out->slab_bytes = (int32_t)(t->slab_words * 4u);
    return SLAB_OK;
}

int slab_get_config(const slab_table* t, slab_config* out) {
    if (!t || !out) return SLAB_ERR_INVALID_ARG;
    *out = t->cfg;
    return SLAB_OK;
}

int slab_set_config(slab_table* t, const slab_config* cfg) {
    if (!t || !cfg || !valid_config(*cfg)) return SLAB_ERR_INVALID_ARG;
    if (cfg->variant == SLAB_VARIANT_STAGED && cfg->threads_per_block > staged_block_limit(t->mode, t->slab_words))
        return SLAB_ERR_INVALID_ARG;
    // the paper-structured kernels read one word per lane of 128-byte slabs only
    if (cfg->variant == SLAB_VARIANT_DIRECT && t->slab_words != 32u) return SLAB_ERR_INVALID_ARG;
    if (cfg->threads_per_block != t->cfg.threads_per_block)
        for (auto& v : t->occupancy)
            for (int& o : v) o = 0;
    t->cfg = *cfg;
    return SLAB_OK;
}

int slab_insert_batch(slab_table* t, const uint32_t* d_keys, const uint32_t* d_values, uint8_t* d_found,
                      uint32_t n, void* stream) {
    if (!t || (n && !d_keys) || (n && !d_values && t->mode == SLAB_MODE_KEY_VALUE)) return SLAB_ERR_INVALID_ARG;
    BatchArgs a{nullptr, d_keys, d_values, nullptr, d_found, n};
    if (n) t->dirty = true;
    return dispatch<kKindInsert>(t, a, stream);
}

int slab_delete_batch(slab_table* t, const uint32_t* d_keys, uint8_t* d_found, uint32_t n, void* stream) {
    if (!t || (n && !d_keys)) return SLAB_ERR_INVALID_ARG;
    BatchArgs a{nullptr, d_keys, nullptr, nullptr, d_found, n};
    return dispatch<kKindDelete>(t, a, stream);
}

int slab_search_batch(slab_table* t, const uint32_t* d_keys, uint32_t* d_values_out, uint8_t* d_found,
                      uint32_t n, void* stream) {
    if (!t || (n && (!d_keys || !d_values_out))) return SLAB_ERR_INVALID_ARG;
    BatchArgs a{nullptr, d_keys, nullptr, d_values_out, d_found, n};
    return dispatch<kKindSearch>(t, a, stream);
}

int slab_mixed_batch(slab_table* t, const uint8_t* d_ops, const uint32_t* d_keys, const uint32_t* d_values,
                     uint32_t* d_results, uint8_t* d_found, uint32_t n, void* stream) {
    if (!t || (n && (!d_ops || !d_keys || !d_results)) ||
        (n && !d_values && t->mode == SLAB_MODE_KEY_VALUE))
        return SLAB_ERR_INVALID_ARG;
    BatchArgs a{d_ops, d_keys, d_values, d_results, d_found, n};
    if (n) t->dirty = true;
    return dispatch<kKindMixed>(t, a, stream);
}

int slab_status(slab_table* t, void* stream, uint32_t* h_flags) {
    if (!t) return SLAB_ERR_INVALID_ARG;
    uint32_t f = 0;
    if (cudaMemcpyAsync(&f, t->d_misc, 4, cudaMemcpyDeviceToHost, S(stream)) != cudaSuccess ||
        cudaMemsetAsync(t->d_misc, 0, 4, S(stream)) != cudaSuccess ||
        cudaStreamSynchronize(S(stream)) != cudaSuccess)
        return SLAB_ERR_CUDA;
    if (h_flags) *h_flags = f;
    if (f & kFlagBadPointer) return SLAB_ERR_CORRUPT;
    if (f & kFlagOutOfSlabs) return SLAB_ERR_OUT_OF_SLABS;
    if (f & kFlagIterLimit) return SLAB_ERR_ITER_LIMIT;
    if (f & kFlagReserved) return SLAB_ERR_RESERVED_KEY;
    return SLAB_OK;
}

int slab_stats(slab_table* t, uint32_t* d_slots, uint32_t* d_slabs, uint64_t* h_totals, void* stream) {
    if (!t) return SLAB_ERR_INVALID_ARG;
    unsigned long long* acc = counters(t);
    if (cudaMemsetAsync(acc, 0, 8 * sizeof(unsigned long long), S(stream)) != cudaSuccess) return SLAB_ERR_CUDA;
    const TableView T = view(t);
    const uint32_t grid = util_grid(t, (uint64_t)t->num_buckets * 32, 256);
    const int krc = with_layout(t->mode, t->slab_words, [&](auto ko, auto wd) {
        stats_kernel<decltype(ko)::value, decltype(wd)::value><<<grid, 256, 0, S(stream)>>>(T, d_slots, d_slabs, acc);
        return launch_rc();
    });
    if (krc != SLAB_OK) return SLAB_ERR_CUDA;
    const uint64_t words = (uint64_t)t->num_blocks * 32;
    popcount_kernel<<<util_grid(t, words, 256), 256, 0, S(stream)>>>(t->d_bitmaps, words, acc);
    if (launch_rc() != SLAB_OK) return SLAB_ERR_CUDA;
    if (h_totals) {
        unsigned long long h[8];
        if (cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, S(stream)) != cudaSuccess ||
            cudaStreamSynchronize(S(stream)) != cudaSuccess)
            return SLAB_ERR_CUDA;
        for (int i = 0; i < 6; ++i) h_totals[i] = h[i];
    }
    return SLAB_OK;
}

int slab_export(slab_table* t, uint32_t* d_buckets, uint32_t* d_keys, uint32_t* d_values, uint64_t capacity,
                uint64_t* h_count, void* stream) {
    if (!t || !h_count || (capacity && !d_keys)) return SLAB_ERR_INVALID_ARG;
    unsigned long long* acc = counters(t);
    if (cudaMemsetAsync(acc + 6, 0, sizeof(unsigned long long), S(stream)) != cudaSuccess) return SLAB_ERR_CUDA;
    const TableView T = view(t);
    const uint32_t grid = util_grid(t, (uint64_t)t->num_buckets * 32, 256);
    const int krc = with_layout(t->mode, t->slab_words, [&](auto ko, auto wd) {
        export_kernel<decltype(ko)::value, decltype(wd)::value><<<grid, 256, 0, S(stream)>>>(T, d_buckets, d_keys,
                                                                                           d_values, capacity, acc + 6);
        return launch_rc();
    });
    if (krc != SLAB_OK) return SLAB_ERR_CUDA;
    unsigned long long c = 0;
    if (cudaMemcpyAsync(&c, acc + 6, sizeof(c), cudaMemcpyDeviceToHost, S(stream)) != cudaSuccess ||
        cudaStreamSynchronize(S(stream)) != cudaSuccess)
        return SLAB_ERR_CUDA;
    *h_count = c;
    return SLAB_OK;
}

int slab_bucket_of(slab_table* t, const uint32_t* d_keys, uint32_t* d_buckets_out, uint32_t n, void* stream) {
    if (!t || (n && (!d_keys || !d_buckets_out))) return SLAB_ERR_INVALID_ARG;
    if (n == 0) return SLAB_OK;
    const TableView T = view(t);
    bucket_kernel<<<util_grid(t, n, 256), 256, 0, S(stream)>>>(T, d_keys, d_buckets_out, n);
    return launch_rc();
}

int slab_alloc_batch(slab_table* t, uint32_t* d_addrs_out, uint32_t n, void* stream) {
    if (!t || (n && !d_addrs_out)) return SLAB_ERR_INVALID_ARG;
    if (n == 0) return SLAB_OK;
    const TableView T = view(t);
    const int tpb = t->cfg.threads_per_block;
    const bool batched = t->cfg.variant == SLAB_VARIANT_STAGED;
    const void* k = batched ? (const void*)alloc_kernel<true> : (const void*)alloc_kernel<false>;
    int bps = t->cfg.blocks_per_sm;
    if (bps == 0 && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k, tpb, 0) != cudaSuccess)
        return SLAB_ERR_CUDA;
    const uint64_t warps = (n + 31u) / 32u;
    const uint64_t want = (warps * 32 + tpb - 1) / tpb;
    const uint32_t grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)std::max(bps, 1) * t->sm_count));
    if (batched) alloc_kernel<true><<<grid, tpb, 0, S(stream)>>>(T, d_addrs_out, n);
    else alloc_kernel<false><<<grid, tpb, 0, S(stream)>>>(T, d_addrs_out, n);
    return launch_rc();
}

int slab_free_batch(slab_table* t, const uint32_t* d_addrs, uint32_t n, void* stream) {
    if (!t || (n && !d_addrs)) return SLAB_ERR_INVALID_ARG;
    if (n == 0) return SLAB_OK;
    const TableView T = view(t);
    free_kernel<<<util_grid(t, n, 256), 256, 0, S(stream)>>>(T, d_addrs, n);
    return launch_rc();
}

int slab_copy_bitmaps(const slab_table* t, uint32_t* d_dst, uint64_t n_words, void* stream) {
    if (!t || !d_dst || n_words != (uint64_t)t->num_blocks * 32) return SLAB_ERR_INVALID_ARG;
    return cudaMemcpyAsync(d_dst, t->d_bitmaps, n_words * 4, cudaMemcpyDeviceToDevice, S(stream)) == cudaSuccess
               ? SLAB_OK
               : SLAB_ERR_CUDA;
}

}  // extern "C"

// ======================================================= no-allocation variant
// A variant of the chain-statistics kernel for callers that must not allocate
// device memory: its counters live in a file-scope device array instead of the
// table's own counter block. See slab_chain_histogram_noalloc in slabhash.h.
namespace {

constexpr uint32_t kNoAllocTotals = 8;      // the six slab_stats totals, padded
constexpr uint32_t kNoAllocMaxBins = 1024;  // largest histogram the array can hold
constexpr int kNoAllocMaxDevices = 64;

// 8 KiB + 64 B on every device that loads the library, held until exit.
static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNoAllocTotals + kNoAllocMaxBins];

std::mutex g_noalloc_mutex;
unsigned long long* g_noalloc_ptr[kNoAllocMaxDevices] = {};

template <bool kKeyOnly, uint32_t kW>
__global__ void chain_histogram_kernel(TableView T, uint32_t n_bins, unsigned long long* acc);

// Device address of g_noalloc_scratch on `dev`, resolved with that device
// current. The host-side name of the array is only a stand-in and must never be
// passed to a kernel. `refresh` resolves it again even if it is cached: every
// slab_create does so (allocation is allowed there, and loading the module may
// allocate), which also replaces an address left over from before a device
// reset, since every table in use was created after the last reset.
unsigned long long* noalloc_scratch(int dev, bool refresh) {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (refresh || !g_noalloc_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
            g_noalloc_ptr[dev] = nullptr;
            return nullptr;
        }
        g_noalloc_ptr[dev] = static_cast<unsigned long long*>(p);
    }
    return g_noalloc_ptr[dev];
}

// stats_kernel's walk, binning each list's slab count (last bin: that many or
// more) in a block-shared histogram that is added to the scratch at the end.
template <bool kKeyOnly, uint32_t kW>
__global__ void chain_histogram_kernel(TableView T, uint32_t n_bins, unsigned long long* acc) {
    extern __shared__ unsigned int hist[];
    constexpr uint32_t kMask = key_words<kKeyOnly, kW>();
    constexpr uint32_t kPerSlab = elements_per_slab<kKeyOnly, kW>();
    for (uint32_t i = threadIdx.x; i < n_bins; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    const uint32_t lane = lane_id();
    const uint32_t warp_gid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    unsigned long long live_sum = 0, used_sum = 0, slab_sum = 0, bad = 0, linked = 0;
    for (uint32_t b = warp_gid; b < T.num_buckets; b += nwarps) {
        uint32_t cur = kEmptyKey, used = 0, live = 0, n = 0;
        bool prefix_ok = true, prev_full = true;
        for (uint64_t guard = 0; guard <= (uint64_t)T.num_blocks * kUnitsPerBlock; ++guard) {
            const uint32_t w = lane < kW ? ld_coherent(slab_ptr(T, b, cur) + lane) : kEmptyKey;
            const uint32_t u = __ballot_sync(kFull, w != kEmptyKey) & kMask;
            const uint32_t l = __ballot_sync(kFull, w != kEmptyKey && w != kTombstone) & kMask;
            const uint32_t cnt = __popc(u);
            uint32_t want = 0, m = kMask;
            for (uint32_t i = 0; i < cnt; ++i) { want |= m & (0u - m); m &= m - 1u; }
            if (u != want || !prev_full) prefix_ok = false;
            prev_full = cnt == kPerSlab;
            used += cnt;
            live += __popc(l);
            ++n;
            const uint32_t nx = __shfl_sync(kFull, w, next_word<kW>());
            if (nx == kEmptyKey) break;
            if (!valid_next(T, nx)) {
                prefix_ok = false;
                break;
            }
            cur = nx;
        }
        if (lane == 0) atomicAdd(&hist[min(n, n_bins) - 1u], 1u);
        live_sum += live; used_sum += used; slab_sum += n; linked += n - 1; bad += prefix_ok ? 0 : 1;
    }
    if (lane == 0) {
        atomicAdd(acc + 0, live_sum);
        atomicAdd(acc + 1, used_sum);
        atomicAdd(acc + 2, slab_sum);
        atomicAdd(acc + 4, bad);
        atomicAdd(acc + 5, linked);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < n_bins; i += blockDim.x)
        if (hist[i]) atomicAdd(acc + kNoAllocTotals + i, (unsigned long long)hist[i]);
}

bool noalloc_setup(int dev) {
    if (dev < 0 || dev >= kNoAllocMaxDevices) return true;  // such devices are refused by the call itself
    // load the call's kernels now, so that its first launch does not
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, chain_histogram_kernel<false, 32u>) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, chain_histogram_kernel<true, 32u>) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, chain_histogram_kernel<false, 16u>) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, chain_histogram_kernel<true, 16u>) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, popcount_kernel) != cudaSuccess)
        return false;
    return noalloc_scratch(dev, true) != nullptr;
}

}  // namespace

extern "C" int slab_chain_histogram_noalloc(slab_table* t, uint32_t n_bins, uint64_t* h_hist, uint64_t* h_totals,
                                            void* stream) {
    if (!t || !h_hist || n_bins == 0 || n_bins > kNoAllocMaxBins) return SLAB_ERR_INVALID_ARG;
    // the call ends with copies into host memory and a stream synchronization,
    // neither of which a capturing stream allows: refuse before enqueueing anything
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    const cudaError_t qe = cudaStreamIsCapturing(S(stream), &cap);
    if (qe == cudaErrorStreamCaptureImplicit) {  // the legacy stream while another stream captures
        cudaGetLastError();
        return SLAB_ERR_INVALID_ARG;
    }
    if (qe != cudaSuccess) return SLAB_ERR_CUDA;
    if (cap != cudaStreamCaptureStatusNone) return SLAB_ERR_INVALID_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return SLAB_ERR_CUDA;
    if (dev != t->device || dev < 0 || dev >= kNoAllocMaxDevices) return SLAB_ERR_INVALID_ARG;
    unsigned long long* acc = noalloc_scratch(dev, false);
    if (!acc) return SLAB_ERR_CUDA;
    // every call starts from zeroed counters; the array keeps the previous call's values
    if (cudaMemsetAsync(acc, 0, (kNoAllocTotals + n_bins) * sizeof(unsigned long long), S(stream)) != cudaSuccess)
        return SLAB_ERR_CUDA;
    const TableView T = view(t);
    const uint32_t grid = util_grid(t, (uint64_t)t->num_buckets * 32, 256);
    const size_t smem = n_bins * sizeof(unsigned int);
    const int krc = with_layout(t->mode, t->slab_words, [&](auto ko, auto wd) {
        chain_histogram_kernel<decltype(ko)::value, decltype(wd)::value><<<grid, 256, smem, S(stream)>>>(T, n_bins,
                                                                                                       acc);
        return launch_rc();
    });
    if (krc != SLAB_OK) return SLAB_ERR_CUDA;
    const uint64_t words = (uint64_t)t->num_blocks * 32;
    popcount_kernel<<<util_grid(t, words, 256), 256, 0, S(stream)>>>(t->d_bitmaps, words, acc);
    if (launch_rc() != SLAB_OK) return SLAB_ERR_CUDA;
    unsigned long long tot[kNoAllocTotals];
    if (cudaMemcpyAsync(h_hist, acc + kNoAllocTotals, n_bins * sizeof(uint64_t), cudaMemcpyDeviceToHost,
                        S(stream)) != cudaSuccess ||
        cudaMemcpyAsync(tot, acc, sizeof(tot), cudaMemcpyDeviceToHost, S(stream)) != cudaSuccess ||
        cudaStreamSynchronize(S(stream)) != cudaSuccess)
        return SLAB_ERR_CUDA;
    if (h_totals)
        for (int i = 0; i < 6; ++i) h_totals[i] = tot[i];
    return SLAB_OK;
}
