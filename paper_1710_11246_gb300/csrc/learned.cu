// Learned bucket function: fitting the two-level piecewise-linear CDF model on a
// sample of the keys the table is about to hold, measuring the slab lists each
// bucket function would give those keys, and choosing between the model and the
// universal hash (Sec. 3.3) on that measurement.
//
// Every step is exactly reproducible: the least-squares moments are exact
// 128-bit integer sums (their order does not matter), and the line through them
// is computed with a fixed sequence of correctly rounded double operations and
// one rounding to float, so any implementation that follows the same steps gets
// the same model bit for bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "../../include/slabhash.h"
#include "slab_device.cuh"
#include "slab_table.cuh"

using namespace slab;
using slab_host::launch_rc;
using slab_host::S;
using slab_host::util_grid;
using slab_host::view;

namespace {

constexpr uint32_t kLeaves = 1024;
constexpr uint32_t kMaxSample = 1u << 20;
constexpr int kFitThreads = 256;

typedef unsigned __int128 u128;
typedef __int128 s128;

// Exact moments of points (x, y): count, sum x, sum y, sum x^2, sum x*y.
struct Moments {
    unsigned long long n;
    u128 sx, sy, sxx, sxy;
};

__device__ __forceinline__ void add_point(Moments& m, uint32_t x, unsigned long long y) {
    m.n += 1;
    m.sx += x;
    m.sy += y;
    m.sxx += (u128)((unsigned long long)x * x);
    m.sxy += (u128)x * (u128)y;
}

// u128 -> double as hi * 2^64 + lo, each step correctly rounded.
__device__ __forceinline__ double u128_to_double(u128 v) {
    return __dadd_rn(__dmul_rn(__ull2double_rn((unsigned long long)(v >> 64)), 18446744073709551616.0),
                     __ull2double_rn((unsigned long long)v));
}
__device__ __forceinline__ double s128_to_double(s128 v) {
    return v < 0 ? -u128_to_double((u128)(-v)) : u128_to_double((u128)v);
}

// Least-squares line y = (a' x + b') / q through points (x, q y) with moments m
// (m.n >= 1) of x and of the integer targets q y:
//   den = n Sxx - Sx^2, num = n Sxy - Sx Sy (exact), a' = num / den,
//   b' = (Sy - a' Sx) / n, a = a' / q, b = b' / q
// in correctly rounded double, then rounded to float; points with one distinct x
// give a flat line at their mean.
__device__ void fit_line(const Moments& m, unsigned long long q, float* a, float* b) {
    const s128 n = (s128)m.n;
    const s128 den = n * (s128)m.sxx - (s128)m.sx * (s128)m.sx;
    const s128 num = n * (s128)m.sxy - (s128)m.sx * (s128)m.sy;
    const double dn = __ull2double_rn(m.n), dq = __ull2double_rn(q);
    double a1 = 0.0, b1;
    if (den > 0) {
        a1 = __ddiv_rn(s128_to_double(num), s128_to_double(den));
        b1 = __ddiv_rn(__dadd_rn(u128_to_double(m.sy), -__dmul_rn(a1, u128_to_double(m.sx))), dn);
    } else {
        b1 = __ddiv_rn(u128_to_double(m.sy), dn);
    }
    *a = __double2float_rn(__ddiv_rn(a1, dq));
    *b = __double2float_rn(__ddiv_rn(b1, dq));
}

// sample[i] = keys[i * stride] for i < m, padded with 0xFFFFFFFF up to p entries.
__global__ void sample_kernel(const uint32_t* keys, uint32_t stride, uint32_t m, uint32_t p, uint32_t* sample) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < p; i += gridDim.x * blockDim.x)
        sample[i] = i < m ? keys[(uint64_t)i * stride] : 0xFFFFFFFFu;
}

// Ascending bitonic sort of p (a power of two) words over many blocks. The
// network's compare-exchange stages with partner distance j >= kSortTile / 2 run
// one launch each over global memory (bitonic_global_kernel); every run of stages
// with smaller distances works inside aligned tiles of kSortTile words, so it runs
// as one launch that sorts each tile's part in shared memory (bitonic_tile_kernel).
constexpr uint32_t kSortTile = 2048;  // words per shared-memory tile (two per thread)

__device__ __forceinline__ void compare_exchange(uint32_t& x, uint32_t& y, bool ascending) {
    if ((x > y) == ascending) {
        const uint32_t t = x;
        x = y;
        y = t;
    }
}

// Stage (k, j) of the network for all pairs (i, i ^ j), j >= kSortTile / 2.
__global__ void bitonic_global_kernel(uint32_t* v, uint32_t p, uint32_t k, uint32_t j) {
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < p / 2; t += gridDim.x * blockDim.x) {
        const uint32_t i = (t / j) * 2u * j + (t % j);  // the lower index of pair t
        uint32_t x = v[i], y = v[i + j];
        compare_exchange(x, y, (i & k) == 0);
        v[i] = x;
        v[i + j] = y;
    }
}

// Stages (k, j) for j = j0, j0 / 2, ..., 1 of one merge size k (or, with
// k0 = 0, every stage of every k <= kSortTile) inside each tile of kSortTile words.
__global__ void __launch_bounds__(kSortTile / 2) bitonic_tile_kernel(uint32_t* v, uint32_t k_fixed, uint32_t j0) {
    __shared__ uint32_t sm[kSortTile];
    const uint32_t base = blockIdx.x * kSortTile;
    for (uint32_t i = threadIdx.x; i < kSortTile; i += blockDim.x) sm[i] = v[base + i];
    __syncthreads();
    auto run = [&](uint32_t k, uint32_t jstart) {
        for (uint32_t j = jstart; j > 0; j >>= 1) {
            const uint32_t t = threadIdx.x;  // pair t of the tile's kSortTile / 2
            const uint32_t i = (t / j) * 2u * j + (t % j);
            uint32_t x = sm[i], y = sm[i + j];
            compare_exchange(x, y, ((base + i) & k) == 0);
            sm[i] = x;
            sm[i + j] = y;
            __syncthreads();
        }
    };
    if (k_fixed == 0) {
        for (uint32_t k = 2; k <= kSortTile; k <<= 1) run(k, k >> 1);
    } else {
        run(k_fixed, j0);
    }
    for (uint32_t i = threadIdx.x; i < kSortTile; i += blockDim.x) v[base + i] = sm[i];
}

// Sort p words (a power of two) ascending: a sequence of launches on `s`.
void bitonic_sort(uint32_t* v, uint32_t p, cudaStream_t s, const slab_table* t) {
    if (p <= kSortTile) {  // one tile: one block of the tile kernel on a padded copy is not needed
        // p < kSortTile only for tiny samples; run the global stages, which cover any p
        for (uint32_t k = 2; k <= p; k <<= 1)
            for (uint32_t j = k >> 1; j > 0; j >>= 1)
                bitonic_global_kernel<<<util_grid(t, p / 2, 256), 256, 0, s>>>(v, p, k, j);
        return;
    }
    const uint32_t tiles = p / kSortTile;
    bitonic_tile_kernel<<<tiles, kSortTile / 2, 0, s>>>(v, 0u, 0u);
    for (uint32_t k = 2 * kSortTile; k <= p; k <<= 1) {
        for (uint32_t j = k >> 1; j >= kSortTile / 2 * 2; j >>= 1)
            bitonic_global_kernel<<<util_grid(t, p / 2, 256), 256, 0, s>>>(v, p, k, j);
        bitonic_tile_kernel<<<tiles, kSortTile / 2, 0, s>>>(v, k, kSortTile / 2);
    }
}

__device__ void add_moments(Moments& a, const Moments& b) {
    a.n += b.n;
    a.sx += b.sx;
    a.sy += b.sy;
    a.sxx += b.sxx;
    a.sxy += b.sxy;
}

// The block's exact moments summed into part[0] (integer sums: the order of the
// additions does not change the result).
__device__ void block_moments(Moments mine, Moments* part) {
    part[threadIdx.x] = mine;
    __syncthreads();
    for (uint32_t o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) add_moments(part[threadIdx.x], part[threadIdx.x + o]);
        __syncthreads();
    }
}

// Root, part 1: block b's moments of the points (sorted[i], i * 1024), i < m.
__global__ void __launch_bounds__(kFitThreads) root_moments_kernel(const uint32_t* sorted, uint32_t m,
                                                                   Moments* partial) {
    __shared__ Moments part[kFitThreads];
    Moments mo{};
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
        add_point(mo, sorted[i], (unsigned long long)i * kLeaves);
    block_moments(mo, part);
    if (threadIdx.x == 0) partial[blockIdx.x] = part[0];
}

// Root, part 2 (one block): the root line from the blocks' moments: leaf position
// i * 1024 / m fitted against the i-th smallest sample key.
__global__ void __launch_bounds__(kFitThreads) root_fit_kernel(const Moments* partial, uint32_t nparts, uint32_t m,
                                                               float* model) {
    __shared__ Moments part[kFitThreads];
    Moments mo{};
    for (uint32_t b = threadIdx.x; b < nparts; b += blockDim.x) add_moments(mo, partial[b]);
    block_moments(mo, part);
    if (threadIdx.x == 0) fit_line(part[0], m, &model[0], &model[1]);
}

// Leaves, one block per leaf j: the sample points the root sends to j (a
// contiguous run, since the root's slope is >= 0) fit bucket position i * B / m;
// a leaf with no point is flat at the position where its run would start.
__global__ void __launch_bounds__(kFitThreads) leaf_fit_kernel(const uint32_t* sorted, uint32_t m,
                                                               uint32_t num_buckets, float* model) {
    __shared__ Moments part[kFitThreads];
    const uint32_t j = blockIdx.x;
    const float ra = model[0], rb = model[1];
    auto leaf_of = [&](uint32_t i) { return linear_piece(ra, rb, __uint2float_rn(sorted[i]), kLeaves); };
    auto first_at_least = [&](uint32_t jj) {  // smallest i with leaf_of(i) >= jj, or m
        uint32_t lo = 0, hi = m;
        while (lo < hi) {
            const uint32_t mid = lo + (hi - lo) / 2;
            if (leaf_of(mid) >= jj) hi = mid;
            else lo = mid + 1;
        }
        return lo;
    };
    const uint32_t lo = first_at_least(j), hi = first_at_least(j + 1);
    Moments lm{};
    for (uint32_t i = lo + threadIdx.x; i < hi; i += blockDim.x)
        add_point(lm, sorted[i], (unsigned long long)i * num_buckets);
    block_moments(lm, part);
    if (threadIdx.x == 0) {
        float a = 0.0f, b;
        if (hi > lo) {
            fit_line(part[0], m, &a, &b);
        } else {
            b = __double2float_rn(__ddiv_rn(__ull2double_rn((unsigned long long)lo * num_buckets),
                                            __ull2double_rn(m)));
        }
        model[2 + 2 * j] = a;
        model[3 + 2 * j] = b;
    }
}

// counts[bucket(k)] += 1 under the learned model or the universal hash.
__global__ void count_kernel(TableView T, const uint32_t* keys, uint32_t n, uint32_t learned, uint32_t* counts) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t k = keys[i];
        if (k >= kTombstone) continue;
        atomicAdd(&counts[learned ? learned_bucket(T.model, T.num_buckets, k) : universal_bucket(T, k)], 1u);
    }
}

// Slab lists the counted keys would form: sum and maximum of max(1, ceil(c / M)).
__global__ void chain_kernel(const uint32_t* counts, uint32_t num_buckets, uint32_t per_slab,
                             unsigned long long* sum, uint32_t* max_slabs) {
    unsigned long long s = 0;
    uint32_t mx = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < num_buckets; i += gridDim.x * blockDim.x) {
        const uint32_t c = counts[i];
        const uint32_t slabs = c == 0 ? 1u : (c + per_slab - 1) / per_slab;
        s += slabs;
        mx = max(mx, slabs);
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_down_sync(kFull, s, o);
        mx = max(mx, __shfl_down_sync(kFull, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(sum, s);
        atomicMax(max_slabs, mx);
    }
}

}  // namespace

extern "C" {

int slab_learn_buckets(slab_table* t, const uint32_t* d_keys, uint32_t n, uint32_t sample_stride, int policy,
                       slab_learn_report* out, void* stream) {
    if (!t || !d_keys || n == 0 || sample_stride == 0 || policy < SLAB_LEARN_AUTO || policy > SLAB_LEARN_MEASURE)
        return SLAB_ERR_INVALID_ARG;
    if (t->dirty) return SLAB_ERR_INVALID_ARG;  // keys already stored under the current bucket function
    if (!t->d_model) return SLAB_ERR_INVALID_ARG;  // tables inside a group have no model storage
    const uint32_t m = (uint32_t)(((uint64_t)n + sample_stride - 1) / sample_stride);
    if (m > kMaxSample) return SLAB_ERR_INVALID_ARG;
    uint32_t p = 2;
    while (p < m) p <<= 1;
    const cudaStream_t s = S(stream);
    const uint64_t B = t->num_buckets;
    // scratch: padded sample, per-bucket counts, two sums and two maxima, the root's
    // per-block moments
    constexpr uint32_t kRootParts = 512;
    char* scratch = nullptr;
    const size_t moments_at = (((size_t)p + B) * 4 + 32 + 15) / 16 * 16;
    const size_t bytes = moments_at + kRootParts * sizeof(Moments);
    if (cudaMallocAsync(reinterpret_cast<void**>(&scratch), bytes, s) != cudaSuccess) return SLAB_ERR_CUDA;
    uint32_t* sample = reinterpret_cast<uint32_t*>(scratch);
    uint32_t* counts = sample + p;
    unsigned long long* sums = reinterpret_cast<unsigned long long*>(scratch + (((size_t)p + B) * 4 + 7) / 8 * 8);
    uint32_t* maxima = reinterpret_cast<uint32_t*>(sums + 2);
    Moments* root_parts = reinterpret_cast<Moments*>(scratch + moments_at);
    int rc = SLAB_OK;
    unsigned long long h_sums[2] = {0, 0};
    uint32_t h_max[2] = {0, 0};
    const uint32_t per_slab = t->mode == SLAB_MODE_KEY_ONLY ? t->slab_words - 2u : (t->slab_words - 2u) / 2u;
    do {
        sample_kernel<<<util_grid(t, p, 256), 256, 0, s>>>(d_keys, sample_stride, m, p, sample);
        bitonic_sort(sample, p, s, t);
        const uint32_t parts = std::min<uint32_t>(kRootParts, (m + kFitThreads - 1) / kFitThreads);
        root_moments_kernel<<<parts, kFitThreads, 0, s>>>(sample, m, root_parts);
        root_fit_kernel<<<1, kFitThreads, 0, s>>>(root_parts, parts, m, t->d_model);
        leaf_fit_kernel<<<kLeaves, kFitThreads, 0, s>>>(sample, m, t->num_buckets, t->d_model);
        if ((rc = launch_rc()) != SLAB_OK) break;
        if (cudaMemsetAsync(sums, 0, 24, s) != cudaSuccess) { rc = SLAB_ERR_CUDA; break; }
        TableView T = view(t);
        for (uint32_t which = 0; which < 2; ++which) {  // 0: learned, 1: universal
            if (cudaMemsetAsync(counts, 0, B * 4, s) != cudaSuccess) { rc = SLAB_ERR_CUDA; break; }
            count_kernel<<<util_grid(t, n, 256), 256, 0, s>>>(T, d_keys, n, which == 0, counts);
            chain_kernel<<<util_grid(t, B, 256), 256, 0, s>>>(counts, (uint32_t)B, per_slab, sums + which,
                                                               maxima + which);
        }
        if (rc != SLAB_OK || (rc = launch_rc()) != SLAB_OK) break;
        if (cudaMemcpyAsync(h_sums, sums, 16, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(h_max, maxima, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess)
            rc = SLAB_ERR_CUDA;
    } while (false);
    cudaFreeAsync(scratch, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) rc = SLAB_ERR_CUDA;
    if (rc != SLAB_OK) return rc;
    const double mean_l = (double)h_sums[0] / (double)B, mean_u = (double)h_sums[1] / (double)B;
    bool use = policy == SLAB_LEARN_ALWAYS;
    if (policy == SLAB_LEARN_AUTO) use = mean_l <= mean_u && h_max[0] <= h_max[1];
    t->learned = use;
    t->model_fitted = true;
    if (out) {
        out->sample_size = m;
        out->use_learned = use ? 1u : 0u;
        out->max_slabs_learned = h_max[0];
        out->max_slabs_universal = h_max[1];
        out->mean_slabs_learned = mean_l;
        out->mean_slabs_universal = mean_u;
    }
    return SLAB_OK;
}

int slab_get_model(const slab_table* t, float* h_model, uint32_t* h_in_use) {
    if (!t || !h_model || !t->d_model) return SLAB_ERR_INVALID_ARG;
    if (cudaMemcpy(h_model, t->d_model, (2 + 2 * kLeaves) * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
        return SLAB_ERR_CUDA;
    if (h_in_use) *h_in_use = t->learned ? 1u : 0u;
    return SLAB_OK;
}

}  // extern "C"
