// The paper's operations beyond the bulk hot path: multiset tables (Sec. 3.2
// INSERT with duplicates allowed, deletes that empty their slot), SEARCHALL and
// DELETEALL (Sec. 3.2), FLUSH (Sec. 4.3.4) and growing the SlabAlloc pool by
// whole memory blocks (Sec. 5, "add super blocks").
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "../../include/slabhash.h"
#include "slab_device.cuh"
#include "slab_table.cuh"
#include "slab_wcws.cuh"

using namespace slab;
using slab_host::counters;
using slab_host::launch_rc;
using slab_host::S;
using slab_host::util_grid;
using slab_host::view;

namespace {

// SEARCHALL / DELETEALL: the WCWS loop of Fig. "alg:search" with the walk going
// on past a match to the end of the list. One op per lane; the warp serves its
// queue one op at a time and reads each slab of the op's list coalesced (word
// `lane` per lane). Matching key lanes act in parallel: they copy out their
// values in list order (search) or remove their elements (delete).
template <bool kKeyOnly, bool kDelete>
__global__ void all_kernel(TableView T, const uint32_t* keys, uint32_t n, uint32_t cap, uint32_t* counts,
                           uint32_t* values) {
    constexpr uint32_t kMask = kKeyOnly ? kKeyLanesKeyOnly : kKeyLanesKV;
    const uint32_t lane = lane_id();
    const uint32_t warp_gid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t tile = warp_gid; tile < (n + 31u) / 32u; tile += nwarps) {
        const uint32_t idx = tile * 32u + lane;
        const bool has = idx < n;
        const uint32_t key = has ? ld_stream(keys + idx) : 0u;
        bool active = has;
        if (active && key >= kTombstone) {
            set_flag(T, kFlagReserved);
            active = false;
        }
        const uint32_t bucket = active ? bucket_of(T, key) : 0u;
        uint32_t mine = 0;
        for (uint32_t queue = __ballot_sync(kFull, active); queue; queue &= queue - 1u) {
            const int s = __ffs(queue) - 1;
            const uint32_t skey = __shfl_sync(kFull, key, s);
            const uint32_t sb = __shfl_sync(kFull, bucket, s);
            const uint64_t row = (uint64_t)(tile * 32u + (uint32_t)s) * cap;
            uint32_t cur = kEmptyKey, found = 0;
            for (uint64_t steps = 0;; ++steps) {
                uint32_t* p = slab_ptr(T, sb, cur);
                const uint32_t w = kDelete ? ld_coherent(p + lane) : ld_readonly(p + lane);
                const uint32_t v = __shfl_down_sync(kFull, w, 1);
                const uint32_t m = __ballot_sync(kFull, w == skey) & kMask;
                if ((m >> lane) & 1u) {
                    if constexpr (kDelete) {
                        remove_at<kKeyOnly>(T, p, lane);
                    } else {
                        const uint32_t rank = found + __popc(m & ((1u << lane) - 1u));
                        if (rank < cap) values[row + rank] = kKeyOnly ? 0u : v;
                    }
                }
                found += __popc(m);
                const uint32_t nx = __shfl_sync(kFull, w, kAddressLane);
                if (nx == kEmptyKey) break;
                // a list holds at most every pool slab once
                if (!valid_next(T, nx) || steps >= T.pool_units) {
                    if (lane == 0) set_flag(T, kFlagBadPointer);
                    break;
                }
                cur = nx;
            }
            if ((int)lane == s) mine = found;
        }
        if (has && counts) counts[idx] = mine;
    }
}

// FLUSH (Sec. 4.3.4): one warp per bucket compacts its list in place. Walking the
// list in order, the live elements of each slab are written, in list order,
// behind the ones kept so far; the write position never passes the read
// position, so every slab is read before anything is written into it. The last
// kept slab is padded with empty elements and terminated; the slabs after it are
// emptied and returned to SlabAlloc. Runs alone on the table (a separate launch,
// as in the paper), so plain loads and stores suffice.
template <bool kKeyOnly>
__global__ void flush_kernel(TableView T, unsigned long long* released) {
    constexpr uint32_t kMask = kKeyOnly ? kKeyLanesKeyOnly : kKeyLanesKV;
    constexpr uint32_t kPer = kKeyOnly ? 30u : 15u;      // elements per slab
    constexpr uint32_t kWordsPer = kKeyOnly ? 1u : 2u;  // words per element
    const uint32_t lane = lane_id();
    const uint32_t warp_gid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    unsigned long long freed = 0;
    for (uint32_t b = warp_gid; b < T.num_buckets; b += nwarps) {
        uint32_t* const base = T.slabs + (uint64_t)b * kWordsPerSlab;
        uint32_t* wp = base;        // write slab: index ws = cursor / kPer of the list
        uint32_t* prev = nullptr;   // the write slab before it
        uint32_t ws = 0;
        uint64_t cursor = 0;        // elements kept so far
        uint32_t* rp = base;        // read slab
        bool ok = true;
        for (uint64_t steps = 0;; ++steps) {
            const uint32_t w = rp[lane];
            const uint32_t v = kKeyOnly ? 0u : __shfl_down_sync(kFull, w, 1);
            const uint32_t nx = __shfl_sync(kFull, w, kAddressLane);
            const uint32_t live = __ballot_sync(kFull, w != kEmptyKey && w != kTombstone) & kMask;
            // the slab after the write slab, for elements that spill into it
            const uint32_t wnx = wp ? wp[kAddressLane] : kEmptyKey;
            uint32_t* const spill = (wnx != kEmptyKey && valid_next(T, wnx)) ? T.pool + (uint64_t)wnx * kWordsPerSlab
                                                                           : nullptr;
            if ((live >> lane) & 1u) {
                const uint64_t e = cursor + __popc(live & ((1u << lane) - 1u));
                uint32_t* dst = (e / kPer == ws) ? wp : spill;
                if (dst) {
                    const uint32_t at = (uint32_t)(e % kPer) * kWordsPer;
                    dst[at] = w;
                    if (!kKeyOnly) dst[at + 1] = v;
                }
            }
            cursor += __popc(live);
            if (cursor / kPer > ws) {  // the write slab is full: move to the next one
                prev = wp;
                wp = spill;
                ++ws;
            }
            if (nx == kEmptyKey) break;
            if (!valid_next(T, nx) || steps >= T.pool_units) {
                ok = false;
                break;
            }
            rp = T.pool + (uint64_t)nx * kWordsPerSlab;
        }
        __syncwarp();
        if (!ok) {
            if (lane == 0) set_flag(T, kFlagBadPointer);
            continue;
        }
        // the last kept slab: max(1, ceil(cursor / kPer)) slabs stay in the list
        uint32_t* last = (cursor > 0 && cursor % kPer == 0) ? prev : wp;
        if (!last) {  // cannot happen for a well-formed list
            if (lane == 0) set_flag(T, kFlagBadPointer);
            continue;
        }
        const uint32_t kept = (uint32_t)(cursor - (cursor == 0 ? 0 : ((cursor - 1) / kPer) * kPer));
        if (lane < kPer * kWordsPer && lane >= kept * kWordsPer) last[lane] = kEmptyKey;
        uint32_t q = last[kAddressLane];
        __syncwarp();
        if (lane == kAddressLane) last[kAddressLane] = kEmptyKey;
        for (uint64_t steps = 0; q != kEmptyKey && valid_next(T, q) && steps <= T.pool_units; ++steps) {
            uint32_t* slab = T.pool + (uint64_t)q * kWordsPerSlab;
            const uint32_t next = slab[kAddressLane];
            __syncwarp();
            slab[lane] = kEmptyKey;
            __syncwarp();
            if (lane == 0) deallocate(T, q);
            ++freed;
            q = next;
        }
    }
    if (lane == 0 && freed) atomicAdd(released, freed);
}

int check_table(const slab_table* t) {
    int dev = -1;
    if (!t) return SLAB_ERR_INVALID_ARG;
    if (cudaGetDevice(&dev) != cudaSuccess) return SLAB_ERR_CUDA;
    return dev == t->device ? SLAB_OK : SLAB_ERR_INVALID_ARG;
}

template <bool kDelete>
int launch_all(slab_table* t, const uint32_t* d_keys, uint32_t n, uint32_t cap, uint32_t* d_counts,
               uint32_t* d_values, void* stream) {
    if (n == 0) return SLAB_OK;
    const TableView T = view(t);
    const uint32_t grid = util_grid(t, ((uint64_t)n + 31) / 32 * 32, 256);
    if (t->mode == SLAB_MODE_KEY_ONLY)
        all_kernel<true, kDelete><<<grid, 256, 0, S(stream)>>>(T, d_keys, n, cap, d_counts, d_values);
    else
        all_kernel<false, kDelete><<<grid, 256, 0, S(stream)>>>(T, d_keys, n, cap, d_counts, d_values);
    return launch_rc();
}

}  // namespace

extern "C" {

int slab_set_multiset(slab_table* t, int on) {
    if (!t || !t->owns_memory || t->dirty || (on && t->slab_words != 32u)) return SLAB_ERR_INVALID_ARG;
    t->multiset = on != 0;
    return SLAB_OK;
}

int slab_search_all_batch(slab_table* t, const uint32_t* d_keys, uint32_t n, uint32_t max_per_key,
                          uint32_t* d_counts, uint32_t* d_values_out, void* stream) {
    if (!t || t->slab_words != 32u || (n && (!d_keys || !d_counts || (max_per_key && !d_values_out))))
        return SLAB_ERR_INVALID_ARG;
    return launch_all<false>(t, d_keys, n, max_per_key, d_counts, d_values_out, stream);
}

int slab_delete_all_batch(slab_table* t, const uint32_t* d_keys, uint32_t* d_counts, uint32_t n, void* stream) {
    if (!t || t->slab_words != 32u || (n && !d_keys)) return SLAB_ERR_INVALID_ARG;
    return launch_all<true>(t, d_keys, n, 0, d_counts, nullptr, stream);
}

int slab_flush(slab_table* t, uint64_t* h_released, void* stream) {
    if (!t || t->slab_words != 32u) return SLAB_ERR_INVALID_ARG;
    unsigned long long* acc = counters(t) + 7;
    if (cudaMemsetAsync(acc, 0, sizeof(unsigned long long), S(stream)) != cudaSuccess) return SLAB_ERR_CUDA;
    const TableView T = view(t);
    const uint32_t grid = util_grid(t, (uint64_t)t->num_buckets * 32, 256);
    if (t->mode == SLAB_MODE_KEY_ONLY)
        flush_kernel<true><<<grid, 256, 0, S(stream)>>>(T, acc);
    else
        flush_kernel<false><<<grid, 256, 0, S(stream)>>>(T, acc);
    if (launch_rc() != SLAB_OK) return SLAB_ERR_CUDA;
    if (h_released) {
        unsigned long long r = 0;
        if (cudaMemcpyAsync(&r, acc, sizeof(r), cudaMemcpyDeviceToHost, S(stream)) != cudaSuccess ||
            cudaStreamSynchronize(S(stream)) != cudaSuccess)
            return SLAB_ERR_CUDA;
        *h_released = r;
    }
    return SLAB_OK;
}

int slab_grow_pool(slab_table* t, uint64_t extra_slabs) {
    int rc = check_table(t);
    if (rc != SLAB_OK) return rc;
    if (!t->owns_memory || extra_slabs == 0) return SLAB_ERR_INVALID_ARG;
    const uint64_t add = (extra_slabs + kUnitsPerBlock - 1) / kUnitsPerBlock;
    const uint64_t blocks = (uint64_t)t->num_blocks + add;
    const uint64_t pool = blocks * kUnitsPerBlock;
    if (blocks >= (1ull << 22) || (uint64_t)t->num_buckets + pool > 0xFFFFFFFEull) return SLAB_ERR_INVALID_ARG;
    const uint64_t old_slab_bytes = ((uint64_t)t->num_buckets + t->pool_slabs) * t->slab_words * 4ull;
    const uint64_t slab_bytes = ((uint64_t)t->num_buckets + pool) * t->slab_words * 4ull;
    const uint64_t old_bitmap_bytes = (uint64_t)t->num_blocks * 128ull, bitmap_bytes = blocks * 128ull;
    uint32_t *slabs = nullptr, *bitmaps = nullptr;
    if (cudaDeviceSynchronize() != cudaSuccess) return SLAB_ERR_CUDA;
    if (cudaMalloc(&slabs, slab_bytes) != cudaSuccess || cudaMalloc(&bitmaps, bitmap_bytes) != cudaSuccess) {
        cudaFree(slabs);
        cudaGetLastError();
        return SLAB_ERR_CUDA;
    }
    // existing slabs and bitmap words keep their addresses; the new blocks start
    // empty (every word EMPTY, every bitmap bit clear)
    if (cudaMemcpy(slabs, t->d_slabs, old_slab_bytes, cudaMemcpyDeviceToDevice) != cudaSuccess ||
        cudaMemset(reinterpret_cast<uint8_t*>(slabs) + old_slab_bytes, 0xFF, slab_bytes - old_slab_bytes) !=
            cudaSuccess ||
        cudaMemcpy(bitmaps, t->d_bitmaps, old_bitmap_bytes, cudaMemcpyDeviceToDevice) != cudaSuccess ||
        cudaMemset(reinterpret_cast<uint8_t*>(bitmaps) + old_bitmap_bytes, 0, bitmap_bytes - old_bitmap_bytes) !=
            cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {
        cudaFree(slabs);
        cudaFree(bitmaps);
        return SLAB_ERR_CUDA;
    }
    cudaFree(t->d_slabs);
    cudaFree(t->d_bitmaps);
    t->d_slabs = slabs;
    t->d_bitmaps = bitmaps;
    t->device_bytes += (slab_bytes - old_slab_bytes) + (bitmap_bytes - old_bitmap_bytes);
    t->pool_slabs = pool;
    t->num_blocks = (uint32_t)blocks;
    return SLAB_OK;
}

}  // extern "C"
