// Roofline probes for the slab hash: the rate at which the GPU can read whole
// 128-byte lines at random positions of a buffer of a given size, and the rate
// of random 64-bit atomicCAS operations. A search or insert reads one such line
// per slab it visits, so these rates bound the table's throughput at the same
// footprint.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "../../include/slabhash.h"

namespace {

__device__ __forceinline__ uint32_t mix(uint64_t x) {
    // splitmix64 finalizer, folded to 32 bits
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    x ^= x >> 31;
    return (uint32_t)(x >> 32);
}

// Lemire's multiply-shift range reduction: uniform in [0, n) for n < 2^32.
__device__ __forceinline__ uint64_t pick(uint64_t r, uint64_t seed, uint64_t n) {
    return ((uint64_t)mix(r ^ (seed << 40)) * n) >> 32;
}

// Each warp takes 32 reads at a time: lane j draws the line of read j, then the
// warp reads the 32 lines one after another (32 lanes x 4 bytes each), L lines
// issued before any is consumed.
template <int L>
__global__ void probe_lines_kernel(const uint32_t* __restrict__ buf, uint64_t footprint, uint64_t n_reads,
                                   uint32_t seed, uint32_t* sink) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t groups = (n_reads + 31) / 32;
    uint32_t acc = 0;
    for (uint64_t g = warp; g < groups; g += nwarps) {
        const uint64_t r = g * 32 + lane;
        const uint32_t my_line = (uint32_t)pick(r, seed, footprint);
        const uint32_t valid = __ballot_sync(0xFFFFFFFFu, r < n_reads);
#pragma unroll
        for (int j0 = 0; j0 < 32; j0 += L) {
            uint32_t v[L];
#pragma unroll
            for (int j = 0; j < L; ++j) {
                const uint32_t line = __shfl_sync(0xFFFFFFFFu, my_line, j0 + j);
                v[j] = ((valid >> (j0 + j)) & 1u) ? __ldcg(buf + (uint64_t)line * 32 + lane) : 0u;
            }
#pragma unroll
            for (int j = 0; j < L; ++j) acc ^= v[j];
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc ^= __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if (lane == 0) atomicXor(sink, acc);
}

template <int L>
__global__ void probe_cas_kernel(unsigned long long* buf, uint64_t footprint, uint64_t n_ops, uint32_t seed) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t per = (n_ops + nthreads - 1) / nthreads;
    const uint64_t begin = tid * per;
    const uint64_t end = min(begin + per, n_ops);
    for (uint64_t i = begin; i < end; i += L) {
        unsigned long long got[L];
#pragma unroll
        for (int j = 0; j < L; ++j) {
            const uint64_t r = i + j;
            if (r < end) {
                // one of the 15 pair slots of a random line, like an insert's claim
                const uint64_t line = pick(r, seed, footprint);
                const uint64_t slot = line * 16 + (mix(r + 0x51ED) % 15u);
                got[j] = atomicCAS(buf + slot, 0ull, (unsigned long long)(r | 1u));
            } else {
                got[j] = 0;
            }
        }
        unsigned long long x = 0;
#pragma unroll
        for (int j = 0; j < L; ++j) x |= got[j];
        if (x == 1ull) buf[0] = x;  // keeps the results live; practically never taken
    }
}

template <int L>
__global__ void probe_or_kernel(uint32_t* buf, uint64_t footprint, uint64_t n_ops, uint32_t seed) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t per = (n_ops + nthreads - 1) / nthreads;
    const uint64_t begin = tid * per;
    const uint64_t end = min(begin + per, n_ops);
    for (uint64_t i = begin; i < end; i += L) {
        uint32_t got[L];
#pragma unroll
        for (int j = 0; j < L; ++j) {
            const uint64_t r = i + j;
            got[j] = r < end ? atomicOr(buf + pick(r, seed, footprint), 1u << (mix(r + 0xB17) & 31u)) : 0u;
        }
        uint32_t x = 0;
#pragma unroll
        for (int j = 0; j < L; ++j) x ^= got[j];
        if (x == 0x5A5A5A5Au) buf[0] |= 1u;  // keeps the results live; practically never taken
    }
}

int occupancy_grid(const void* fn, int tpb) {
    int dev = 0, sms = 0, bps = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, tpb, 0);
    return std::max(1, bps) * sms;
}

}  // namespace

extern "C" {

int slab_probe_random_lines(const uint32_t* d_buf, uint64_t footprint_lines, uint64_t n_reads, uint32_t seed,
                            int lines_in_flight, int threads_per_block, uint32_t* d_sink, void* stream) {
    if (!d_buf || !d_sink || footprint_lines == 0 || footprint_lines >= (1ull << 32) || threads_per_block < 32 ||
        threads_per_block > 1024 || threads_per_block % 32)
        return SLAB_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int tpb = threads_per_block;
#define LAUNCH(L)                                                                                         \
    case L: {                                                                                             \
        const int g = occupancy_grid((const void*)probe_lines_kernel<L>, tpb);                            \
        probe_lines_kernel<L><<<g, tpb, 0, s>>>(d_buf, footprint_lines, n_reads, seed, d_sink);           \
        break;                                                                                            \
    }
    switch (lines_in_flight) {
        LAUNCH(1) LAUNCH(2) LAUNCH(4) LAUNCH(8) LAUNCH(16) LAUNCH(32)
        default: return SLAB_ERR_INVALID_ARG;
    }
#undef LAUNCH
    return cudaGetLastError() == cudaSuccess ? SLAB_OK : SLAB_ERR_CUDA;
}

int slab_probe_random_cas(unsigned long long* d_buf, uint64_t footprint_lines, uint64_t n_ops, uint32_t seed,
                          int ops_in_flight, int threads_per_block, void* stream) {
    if (!d_buf || footprint_lines == 0 || footprint_lines >= (1ull << 32) || threads_per_block < 32 ||
        threads_per_block > 1024 || threads_per_block % 32)
        return SLAB_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int tpb = threads_per_block;
#define LAUNCH(L)                                                                                         \
    case L: {                                                                                             \
        const int g = occupancy_grid((const void*)probe_cas_kernel<L>, tpb);                              \
        probe_cas_kernel<L><<<g, tpb, 0, s>>>(d_buf, footprint_lines, n_ops, seed);                       \
        break;                                                                                            \
    }
    switch (ops_in_flight) {
        LAUNCH(1) LAUNCH(2) LAUNCH(4) LAUNCH(8)
        default: return SLAB_ERR_INVALID_ARG;
    }
#undef LAUNCH
    return cudaGetLastError() == cudaSuccess ? SLAB_OK : SLAB_ERR_CUDA;
}

int slab_probe_random_or(uint32_t* d_buf, uint64_t footprint_words, uint64_t n_ops, uint32_t seed,
                         int ops_in_flight, int threads_per_block, void* stream) {
    if (!d_buf || footprint_words == 0 || footprint_words >= (1ull << 32) || threads_per_block < 32 ||
        threads_per_block > 1024 || threads_per_block % 32)
        return SLAB_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int tpb = threads_per_block;
#define LAUNCH(L)                                                                                         \
    case L: {                                                                                             \
        const int g = occupancy_grid((const void*)probe_or_kernel<L>, tpb);                               \
        probe_or_kernel<L><<<g, tpb, 0, s>>>(d_buf, footprint_words, n_ops, seed);                        \
        break;                                                                                            \
    }
    switch (ops_in_flight) {
        LAUNCH(1) LAUNCH(2) LAUNCH(4) LAUNCH(8)
        default: return SLAB_ERR_INVALID_ARG;
    }
#undef LAUNCH
    return cudaGetLastError() == cudaSuccess ? SLAB_OK : SLAB_ERR_CUDA;
}

}  // extern "C"
