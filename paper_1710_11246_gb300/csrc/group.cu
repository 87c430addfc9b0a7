// Groups of independent slab hashes served by one persistent launch.
//
// A group keeps every table's base slabs, pool, bitmaps and status word in one
// device arena and a device array of the tables' views. A batch for the group is
// one array of ops sorted by table, with op_start[i] the first op of table i. The
// group kernel walks tiles of 32 ops of one table each (a prefix sum of per-table
// tile counts maps a tile to its table) and serves every tile with the same WCWS
// tile service as the single-table kernels, staging each tile's base slabs just
// before serving it. One launch replaces one launch per table, so a group of
// hundreds of small tables costs one launch latency and keeps every SM busy.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <new>
#include <type_traits>
#include <vector>

#include "../../include/slabhash.h"
#include "slab_device.cuh"
#include "slab_staged.cuh"
#include "slab_table.cuh"

using namespace slab;
using slab_host::launch_rc;
using slab_host::S;
using slab_host::view;

struct slab_group {
    int device = 0;
    int sm_count = 0;
    int max_smem_optin = 0;
    uint32_t ntables = 0;
    int mode = 0;
    uint32_t slab_words = 32;         // words per slab of every table: 32 (128 bytes) or 16 (64 bytes)
    char* d_arena = nullptr;
    uint64_t arena_bytes = 0;
    TableView* d_views = nullptr;     // ntables views (epoch set per launch)
    uint32_t* d_tile_start = nullptr; // ntables + 1 prefix of tile counts, rebuilt per batch
    uint32_t* d_status = nullptr;     // OR of the tables' status words (slab_group_status)
    std::vector<slab_table*> tables;  // non-owning handles into the arena
    slab_config cfg{};
    uint32_t epoch = 0;
    int occupancy[4] = {};            // resident blocks per SM by kernel kind for cfg; 0 = not yet asked
};

namespace {

template <uint32_t kW>
constexpr uint32_t kGroupWordsPerWarp = kServeWordsPerWarp<kW>;  // stage, ballots, keys, alternate keys

// Tiles of table i: ceil(ops / 32); a decreasing pair of starts counts as no ops.
__device__ __forceinline__ uint32_t tiles_of(const uint32_t* op_start, uint32_t i) {
    const uint32_t a = op_start[i], b = op_start[i + 1];
    return b > a ? (b - a + 31u) / 32u : 0u;
}

// tile_start[i] = sum of the tiles of tables j < i, one block.
__global__ void tile_prefix_kernel(const uint32_t* op_start, uint32_t ntables, uint32_t* tile_start) {
    __shared__ uint32_t part[1024];
    const uint32_t per = (ntables + blockDim.x - 1) / blockDim.x;
    const uint32_t lo = min(ntables, threadIdx.x * per), hi = min(ntables, lo + per);
    uint32_t s = 0;
    for (uint32_t i = lo; i < hi; ++i) s += tiles_of(op_start, i);
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (uint32_t k = 0; k < blockDim.x; ++k) {
            const uint32_t v = part[k];
            part[k] = run;
            run += v;
        }
        tile_start[ntables] = run;
    }
    __syncthreads();
    uint32_t run = part[threadIdx.x];
    for (uint32_t i = lo; i < hi; ++i) {
        tile_start[i] = run;
        run += tiles_of(op_start, i);
    }
}

#ifndef SLAB_GROUP_MAXNREG
#define SLAB_GROUP_MAXNREG 72
#endif

// The group's tiles in order: tile g belongs to the last table whose first tile
// is <= g (a binary search of the tile prefix), lane op idx of that table's ops.
// Tables of a group use the universal hash (no learned model), so a tile's
// buckets need only its table's hash parameters.
template <int kKind, bool kKeyOnly, uint32_t kW>
__global__ void __maxnreg__(SLAB_GROUP_MAXNREG)
    group_kernel(const TableView* __restrict__ views, const uint32_t* __restrict__ op_start,
                 const uint32_t* __restrict__ tile_start, uint32_t ntables, uint32_t epoch, BatchArgs A) {
    extern __shared__ __align__(16) uint32_t smem[];
    constexpr bool kNeedsValue = (kKind == kKindInsert || kKind == kKindMixed) && !kKeyOnly;
    const uint32_t lane = lane_id();
    uint32_t* buf = smem + (threadIdx.x >> 5) * kGroupWordsPerWarp<kW>;
    uint32_t* ballots = buf + kTileWords<kW>;
    uint32_t* skeys = ballots + 32;
    uint32_t* salts = skeys + 32;
    const uint32_t buf_s = (uint32_t)__cvta_generic_to_shared(buf);
    const uint32_t warp_gid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t total = tile_start[ntables];
    uint32_t g = warp_gid;
    if (g >= total) return;  // warp-uniform
    uint32_t off[8];
    stage_offsets<kW>(lane, off);
    AllocCtx ac{kNoBlock, 0u, 0u};
    uint32_t cur_table = 0xFFFFFFFFu;

    // one tile's table, op index and operands (nothing past the group's tiles)
    struct Tile {
        uint32_t lo, idx, k, v, o;
        bool has;
    };
    auto fetch = [&](uint32_t gg) {
        Tile f{0u, 0u, 0u, 0u, kNoOpCode, false};
        if (gg >= total) return f;
        uint32_t lo = 0, hi = ntables;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (tile_start[mid] <= gg) lo = mid;
            else hi = mid;
        }
        f.lo = lo;
        f.idx = op_start[lo] + (gg - tile_start[lo]) * 32u + lane;
        f.has = f.idx < op_start[lo + 1] && f.idx < A.n;  // never past the batch arrays
        if (f.has) {
            f.o = kKind == kKindMixed ? ld_stream_u8(A.ops + f.idx) : fixed_op<kKind>();
            f.k = ld_stream(A.keys + f.idx);
            if (kNeedsValue && A.values) f.v = ld_stream(A.values + f.idx);
        }
        return f;
    };
    auto walks = [](const Tile& f) { return f.o <= kOpSearch && f.k < kTombstone; };
    auto bucket = [&](const Tile& f) {
        if (!walks(f)) return 0u;
        TableView H{};  // the hash parameters of the tile's table
        H.hash_a = views[f.lo].hash_a;
        H.hash_b = views[f.lo].hash_b;
        H.fastmod_m = views[f.lo].fastmod_m;
        H.num_buckets = views[f.lo].num_buckets;
        return universal_bucket(H, f.k);
    };

    // prologue: this tile hashed, the next one loading
    Tile c = fetch(g);
    uint32_t cb = bucket(c);
    Tile n = fetch(g + nwarps);
    for (; g < total; g += nwarps) {
        TableView T = views[c.lo];
        T.epoch = epoch;
        if (c.lo != cur_table) {  // resident blocks belong to one table's pool
            ac = AllocCtx{kNoBlock, 0u, 0u};
            cur_table = c.lo;
        }
        // (1) this tile's base slabs start moving into the stage
        stage_slabs<kW>(T, buf_s, cb, __ballot_sync(kFull, walks(c)), lane);
        cp_async_commit();
        // (2) meanwhile: hash the next tile, start loading the one after it,
        //     publish this tile's keys
        const uint32_t nb = bucket(n);
        const Tile m = fetch(g + 2u * nwarps);
        if constexpr (!SLAB_LANE_MATCH) {  // the WCWS steps read the tile's keys from here
            skeys[lane] = match_key(T, c.k, c.o);
            if constexpr (kKind == kKindMixed) salts[lane] = alt_key(c.k, c.o);
        }
        // (3) serve this tile once its slabs have landed
        cp_async_wait<0>();
        __syncwarp();
        serve_tile<kKind, kKeyOnly, kW>(T, A, ac, warp_gid, buf, buf_s, ballots, skeys, salts, off, c.k, c.v, c.o,
                                        cb, c.idx, c.has);
        // (4) rotate the pipeline
        c = n;
        cb = nb;
        n = m;
        __syncwarp();
    }
}

// Empty every table of the group: base slabs refilled, allocated pool slabs
// refilled through the bitmaps, bitmaps and status words cleared. Block b takes
// tables b, b + gridDim.x, ...
__global__ void group_reset_kernel(const TableView* views, uint32_t ntables) {
    const uint4 ones = make_uint4(kEmptyKey, kEmptyKey, kEmptyKey, kEmptyKey);
    for (uint32_t i = blockIdx.x; i < ntables; i += gridDim.x) {
        const TableView T = views[i];
        uint4* base = reinterpret_cast<uint4*>(T.slabs);
        uint4* pool = reinterpret_cast<uint4*>(T.pool);
        const uint32_t pieces = T.slab_words / 4u;  // 16-byte pieces per slab
        const uint64_t base16 = (uint64_t)T.num_buckets * pieces;
        for (uint64_t k = threadIdx.x; k < base16; k += blockDim.x) base[k] = ones;
        const uint64_t words = (uint64_t)T.num_blocks * 32;
        for (uint64_t w = threadIdx.x; w < words; w += blockDim.x) {
            uint32_t bits = T.bitmaps[w];
            if (!bits) continue;
            T.bitmaps[w] = 0;
            const uint64_t first = (w >> 5) * kUnitsPerBlock + (w & 31u) * 32u;
            for (; bits; bits &= bits - 1u) {
                uint4* slab = pool + (first + (uint64_t)(__ffs(bits) - 1)) * pieces;
                for (uint32_t c = 0; c < pieces; ++c) slab[c] = ones;
            }
        }
        if (threadIdx.x == 0) T.status[0] = 0;
    }
}

__global__ void group_status_kernel(const TableView* views, uint32_t ntables, uint32_t* out) {
    uint32_t f = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < ntables; i += gridDim.x * blockDim.x) {
        f |= views[i].status[0];
        views[i].status[0] = 0;
    }
    for (int o = 16; o > 0; o >>= 1) f |= __shfl_down_sync(kFull, f, o);
    if ((threadIdx.x & 31) == 0 && f) atomicOr(out, f);
}

uint64_t align256(uint64_t x) { return (x + 255) & ~255ull; }

template <int kKind, bool kKeyOnly, uint32_t kW>
int launch_group(slab_group* g, const uint32_t* d_op_start, const BatchArgs& a, void* stream) {
    const int tpb = g->cfg.threads_per_block;
    const size_t smem = (size_t)(tpb / 32) * kGroupWordsPerWarp<kW> * 4;
    if ((int)smem > g->max_smem_optin) return SLAB_ERR_INVALID_ARG;
    auto k = group_kernel<kKind, kKeyOnly, kW>;
    if (smem > 48 * 1024 && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return SLAB_ERR_CUDA;
    int bps = g->cfg.blocks_per_sm;
    if (bps == 0) {  // asked once per configuration: the query costs microseconds
        int& occ = g->occupancy[kKind];
        if (!occ && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, tpb, smem) != cudaSuccess)
            return SLAB_ERR_CUDA;
        bps = occ;
    }
    tile_prefix_kernel<<<1, 1024, 0, S(stream)>>>(d_op_start, g->ntables, g->d_tile_start);
    const uint32_t grid = (uint32_t)std::max(1, std::max(bps, 1) * g->sm_count);
    k<<<grid, tpb, smem, S(stream)>>>(g->d_views, d_op_start, g->d_tile_start, g->ntables, ++g->epoch, a);
    return launch_rc();
}

template <int kKind>
int group_dispatch(slab_group* g, const uint32_t* d_op_start, const BatchArgs& a, void* stream) {
    if (a.n == 0) return SLAB_OK;
    const bool ko = g->mode == SLAB_MODE_KEY_ONLY;
    if (g->slab_words == 16u)
        return ko ? launch_group<kKind, true, 16u>(g, d_op_start, a, stream)
                  : launch_group<kKind, false, 16u>(g, d_op_start, a, stream);
    return ko ? launch_group<kKind, true, 32u>(g, d_op_start, a, stream)
              : launch_group<kKind, false, 32u>(g, d_op_start, a, stream);
}

}  // namespace

extern "C" {

int slab_group_create_width(uint32_t ntables, const uint32_t* h_num_buckets, const uint32_t* h_hash_a,
                            const uint32_t* h_hash_b, const uint64_t* h_pool_slabs, int mode, uint32_t slab_bytes,
                            slab_group** out) {
    if (!out) return SLAB_ERR_INVALID_ARG;
    *out = nullptr;
    if (ntables == 0 || ntables > (1u << 20) || !h_num_buckets || !h_hash_a || !h_hash_b || !h_pool_slabs ||
        (mode != SLAB_MODE_KEY_VALUE && mode != SLAB_MODE_KEY_ONLY) || (slab_bytes != 64u && slab_bytes != 128u))
        return SLAB_ERR_INVALID_ARG;
    // arena layout: [slabs of every table][bitmaps of every table][128-byte status block per table]
    std::vector<uint64_t> slab_off(ntables), bm_off(ntables), misc_off(ntables), pools(ntables);
    const uint64_t slab_bytes_each = slab_bytes;
    uint64_t all_slab_bytes = 0, bm_bytes = 0;
    for (uint32_t i = 0; i < ntables; ++i) {
        const uint32_t B = h_num_buckets[i];
        if (B == 0 || h_hash_a[i] == 0 || h_hash_a[i] >= kPrime || h_hash_b[i] >= kPrime || h_pool_slabs[i] == 0)
            return SLAB_ERR_INVALID_ARG;
        const uint64_t blocks = (h_pool_slabs[i] + kUnitsPerBlock - 1) / kUnitsPerBlock;
        if (blocks >= (1ull << 22) || (uint64_t)B + blocks * kUnitsPerBlock > 0xFFFFFFFEull) return SLAB_ERR_INVALID_ARG;
        pools[i] = blocks * kUnitsPerBlock;
        slab_off[i] = all_slab_bytes;
        all_slab_bytes += align256(((uint64_t)B + pools[i]) * slab_bytes_each);
        bm_off[i] = bm_bytes;
        bm_bytes += align256(blocks * 128ull);
    }
    const uint64_t misc_bytes = (uint64_t)ntables * 128;
    slab_group* g = new (std::nothrow) slab_group();
    if (!g) return SLAB_ERR_CUDA;
    g->ntables = ntables;
    g->mode = mode;
    g->slab_words = slab_bytes_each / 4u;
    g->cfg.variant = SLAB_VARIANT_STAGED;
    g->cfg.threads_per_block = 128;
    g->cfg.blocks_per_sm = 0;
    g->cfg.iter_limit = 1u << 22;
    g->cfg.random_probes = 256;
    int rc = SLAB_OK;
    do {
        if (cudaGetDevice(&g->device) != cudaSuccess ||
            cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, g->device) != cudaSuccess ||
            cudaDeviceGetAttribute(&g->max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, g->device) !=
                cudaSuccess) {
            rc = SLAB_ERR_CUDA;
            break;
        }
        int l2 = 0;
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, g->device);
        g->arena_bytes = all_slab_bytes + bm_bytes + misc_bytes;
        if (cudaMalloc(&g->d_arena, g->arena_bytes) != cudaSuccess ||
            cudaMalloc(&g->d_views, sizeof(TableView) * ntables) != cudaSuccess ||
            cudaMalloc(&g->d_tile_start, 4ull * (ntables + 1)) != cudaSuccess ||
            cudaMalloc(&g->d_status, 4) != cudaSuccess) {
            rc = SLAB_ERR_CUDA;
            break;
        }
        if (cudaMemset(g->d_arena, 0xFF, all_slab_bytes) != cudaSuccess ||
            cudaMemset(g->d_arena + all_slab_bytes, 0, bm_bytes + misc_bytes) != cudaSuccess) {
            rc = SLAB_ERR_CUDA;
            break;
        }
        std::vector<TableView> views(ntables);
        g->tables.reserve(ntables);
        for (uint32_t i = 0; i < ntables; ++i) {
            slab_table* t = new (std::nothrow) slab_table();
            if (!t) {
                rc = SLAB_ERR_CUDA;
                break;
            }
            g->tables.push_back(t);
            t->owns_memory = false;
            t->device = g->device;
            t->sm_count = g->sm_count;
            t->max_smem_optin = g->max_smem_optin;
            t->l2_bytes = l2;
            t->num_buckets = h_num_buckets[i];
            t->mode = mode;
            t->slab_words = g->slab_words;
            t->hash_a = h_hash_a[i];
            t->hash_b = h_hash_b[i];
            t->fastmod_m = UINT64_MAX / h_num_buckets[i] + 1;
            t->pool_slabs = pools[i];
            t->num_blocks = (uint32_t)(pools[i] / kUnitsPerBlock);
            t->d_slabs = reinterpret_cast<uint32_t*>(g->d_arena + slab_off[i]);
            t->d_bitmaps = reinterpret_cast<uint32_t*>(g->d_arena + all_slab_bytes + bm_off[i]);
            t->d_misc = reinterpret_cast<uint32_t*>(g->d_arena + all_slab_bytes + bm_bytes + 128ull * i);
            t->d_model = nullptr;
            t->device_bytes = ((uint64_t)t->num_buckets + pools[i]) * slab_bytes_each + (uint64_t)t->num_blocks * 128 + 128;
            t->cfg = g->cfg;
            views[i] = view(t);
        }
        if (rc != SLAB_OK) break;
        if (cudaMemcpy(g->d_views, views.data(), sizeof(TableView) * ntables, cudaMemcpyHostToDevice) != cudaSuccess)
            rc = SLAB_ERR_CUDA;
    } while (false);
    if (rc != SLAB_OK) {
        slab_group_destroy(g);
        cudaGetLastError();
        return rc;
    }
    *out = g;
    return SLAB_OK;
}

int slab_group_create(uint32_t ntables, const uint32_t* h_num_buckets, const uint32_t* h_hash_a,
                      const uint32_t* h_hash_b, const uint64_t* h_pool_slabs, int mode, slab_group** out) {
    return slab_group_create_width(ntables, h_num_buckets, h_hash_a, h_hash_b, h_pool_slabs, mode, 128u, out);
}

void slab_group_destroy(slab_group* g) {
    if (!g) return;
    cudaDeviceSynchronize();
    for (slab_table* t : g->tables) {
        slab_host::free_host_io(t);
        delete t;
    }
    cudaFree(g->d_arena);
    cudaFree(g->d_views);
    cudaFree(g->d_tile_start);
    cudaFree(g->d_status);
    delete g;
}

int slab_group_table(slab_group* g, uint32_t i, slab_table** out) {
    if (!g || !out || i >= g->ntables) return SLAB_ERR_INVALID_ARG;
    *out = g->tables[i];
    return SLAB_OK;
}

int slab_group_get_config(const slab_group* g, slab_config* out) {
    if (!g || !out) return SLAB_ERR_INVALID_ARG;
    *out = g->cfg;
    return SLAB_OK;
}

// The largest block every group kernel of a mode can launch (register caps).
static int group_block_limit(int mode, uint32_t slab_words) {
    int lim = 1024;
    auto take = [&](const void* k) {
        cudaFuncAttributes a;
        if (cudaFuncGetAttributes(&a, k) == cudaSuccess) lim = std::min(lim, a.maxThreadsPerBlock);
        else cudaGetLastError();
    };
    auto all = [&](auto ko, auto wd) {
        constexpr bool K = decltype(ko)::value;
        constexpr uint32_t W = decltype(wd)::value;
        take((const void*)group_kernel<kKindSearch, K, W>);
        take((const void*)group_kernel<kKindInsert, K, W>);
        take((const void*)group_kernel<kKindDelete, K, W>);
        take((const void*)group_kernel<kKindMixed, K, W>);
    };
    using W16 = std::integral_constant<uint32_t, 16u>;
    using W32 = std::integral_constant<uint32_t, 32u>;
    if (mode == SLAB_MODE_KEY_ONLY) {
        if (slab_words == 16u) all(std::true_type{}, W16{});
        else all(std::true_type{}, W32{});
    } else {
        if (slab_words == 16u) all(std::false_type{}, W16{});
        else all(std::false_type{}, W32{});
    }
    return lim - lim % 32;
}

int slab_group_set_config(slab_group* g, const slab_config* c) {
    if (!g || !c || c->threads_per_block < 32 || c->threads_per_block > 1024 || c->threads_per_block % 32 ||
        c->blocks_per_sm < 0 || c->blocks_per_sm > 64 || c->iter_limit < 1 || c->random_probes > (1u << 20) ||
        (uint64_t)(c->threads_per_block / 32) * kGroupWordsPerWarp<32u> * 4 > 227 * 1024 ||
        c->threads_per_block > group_block_limit(g->mode, g->slab_words))
        return SLAB_ERR_INVALID_ARG;
    if (c->threads_per_block != g->cfg.threads_per_block)
        for (int& o : g->occupancy) o = 0;
    g->cfg = *c;
    g->cfg.variant = SLAB_VARIANT_STAGED;
    std::vector<TableView> views(g->ntables);
    for (uint32_t i = 0; i < g->ntables; ++i) {
        g->tables[i]->cfg.iter_limit = c->iter_limit;
        g->tables[i]->cfg.random_probes = c->random_probes;
        views[i] = view(g->tables[i]);
    }
    return cudaMemcpy(g->d_views, views.data(), sizeof(TableView) * g->ntables, cudaMemcpyHostToDevice) ==
                   cudaSuccess
               ? SLAB_OK
               : SLAB_ERR_CUDA;
}

int slab_group_reset(slab_group* g, void* stream) {
    if (!g) return SLAB_ERR_INVALID_ARG;
    const uint32_t grid = std::min<uint32_t>(g->ntables, (uint32_t)g->sm_count * 8);
    group_reset_kernel<<<grid, 256, 0, S(stream)>>>(g->d_views, g->ntables);
    return launch_rc();
}

int slab_group_insert(slab_group* g, const uint32_t* d_op_start, const uint32_t* d_keys, const uint32_t* d_values,
                      uint8_t* d_found, uint32_t total, void* stream) {
    if (!g || !d_op_start || (total && (!d_keys || (!d_values && g->mode == SLAB_MODE_KEY_VALUE))))
        return SLAB_ERR_INVALID_ARG;
    BatchArgs a{nullptr, d_keys, d_values, nullptr, d_found, total};
    return group_dispatch<kKindInsert>(g, d_op_start, a, stream);
}

int slab_group_delete(slab_group* g, const uint32_t* d_op_start, const uint32_t* d_keys, uint8_t* d_found,
                      uint32_t total, void* stream) {
    if (!g || !d_op_start || (total && !d_keys)) return SLAB_ERR_INVALID_ARG;
    BatchArgs a{nullptr, d_keys, nullptr, nullptr, d_found, total};
    return group_dispatch<kKindDelete>(g, d_op_start, a, stream);
}

int slab_group_search(slab_group* g, const uint32_t* d_op_start, const uint32_t* d_keys, uint32_t* d_values_out,
                      uint8_t* d_found, uint32_t total, void* stream) {
    if (!g || !d_op_start || (total && (!d_keys || !d_values_out))) return SLAB_ERR_INVALID_ARG;
    BatchArgs a{nullptr, d_keys, nullptr, d_values_out, d_found, total};
    return group_dispatch<kKindSearch>(g, d_op_start, a, stream);
}

int slab_group_mixed(slab_group* g, const uint32_t* d_op_start, const uint8_t* d_ops, const uint32_t* d_keys,
                     const uint32_t* d_values, uint32_t* d_results, uint8_t* d_found, uint32_t total, void* stream) {
    if (!g || !d_op_start ||
        (total && (!d_ops || !d_keys || !d_results || (!d_values && g->mode == SLAB_MODE_KEY_VALUE))))
        return SLAB_ERR_INVALID_ARG;
    BatchArgs a{d_ops, d_keys, d_values, d_results, d_found, total};
    return group_dispatch<kKindMixed>(g, d_op_start, a, stream);
}

int slab_group_status(slab_group* g, void* stream, uint32_t* h_flags) {
    if (!g) return SLAB_ERR_INVALID_ARG;
    uint32_t f = 0;
    if (cudaMemsetAsync(g->d_status, 0, 4, S(stream)) != cudaSuccess) return SLAB_ERR_CUDA;
    group_status_kernel<<<std::max<uint32_t>(1, std::min<uint32_t>((g->ntables + 255) / 256, 1024)), 256, 0,
                          S(stream)>>>(g->d_views, g->ntables, g->d_status);
    if (launch_rc() != SLAB_OK || cudaMemcpyAsync(&f, g->d_status, 4, cudaMemcpyDeviceToHost, S(stream)) != cudaSuccess ||
        cudaStreamSynchronize(S(stream)) != cudaSuccess)
        return SLAB_ERR_CUDA;
    if (h_flags) *h_flags = f;
    if (f & kFlagBadPointer) return SLAB_ERR_CORRUPT;
    if (f & kFlagOutOfSlabs) return SLAB_ERR_OUT_OF_SLABS;
    if (f & kFlagIterLimit) return SLAB_ERR_ITER_LIMIT;
    if (f & kFlagReserved) return SLAB_ERR_RESERVED_KEY;
    return SLAB_OK;
}

}  // extern "C"
