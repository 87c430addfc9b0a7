// Roofline probes for the slab hash: the rate at which the GPU can read whole
// 128-byte lines at random positions of a buffer of a given size, and the rate
// of random 64-bit atomicCAS operations. A search or insert reads one such line
// per slab it visits, so these rates bound the table's throughput at the same
// footprint.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

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

// The same random lines read the way the staged kernels move slabs: 16 bytes
// per lane, so a line of kLW words takes kLW / 4 lanes and one warp instruction
// covers 128 / kLW lines (four 128-byte lines or eight 64-byte ones). kCpAsync =
// false: ld.global.cg.v4 into registers, L lines issued before any is consumed.
// kCpAsync = true: cp.async.cg 16-byte copies into the warp's shared-memory stage
// of 32 lines, all 32 lines of a round in flight, then waited for and consumed
// from the stage; L = 64 double-buffers (two stages, the next round issued
// before this one is consumed).
template <bool kCpAsync, int L, uint32_t kLW>
__global__ void probe_lines_v4_kernel(const uint32_t* __restrict__ buf, uint64_t footprint, uint64_t n_reads,
                                      uint32_t seed, uint32_t* sink) {
    extern __shared__ __align__(16) uint32_t stage_all[];
    constexpr uint32_t kLanesPerLine = kLW / 4u, kLinesPerInst = 32u / kLanesPerLine;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t g = lane / kLanesPerLine, c = lane % kLanesPerLine;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t groups = (n_reads + 31) / 32;
    uint32_t acc = 0;
    if constexpr (!kCpAsync) {
        constexpr int kInst = L / (int)kLinesPerInst;  // load instructions in flight
        static_assert(kInst >= 1 && 32 % L == 0, "lines in flight");
        for (uint64_t gr = warp; gr < groups; gr += nwarps) {
            const uint64_t r = gr * 32 + lane;
            const uint32_t my_line = (uint32_t)pick(r, seed, footprint);
            const uint32_t valid = __ballot_sync(0xFFFFFFFFu, r < n_reads);
#pragma unroll
            for (int j0 = 0; j0 < (int)kLanesPerLine; j0 += kInst) {
                uint4 v[kInst];
#pragma unroll
                for (int j = 0; j < kInst; ++j) {
                    const uint32_t s = kLinesPerInst * (j0 + j) + g;  // the line of group g in instruction j0 + j
                    const uint32_t line = __shfl_sync(0xFFFFFFFFu, my_line, s);
                    if ((valid >> s) & 1u) {
                        const uint32_t* p = buf + (uint64_t)line * kLW + c * 4u;
                        asm volatile("ld.global.cg.v4.u32 {%0, %1, %2, %3}, [%4];"
                                     : "=r"(v[j].x), "=r"(v[j].y), "=r"(v[j].z), "=r"(v[j].w)
                                     : "l"(p));
                    } else {
                        v[j] = make_uint4(0u, 0u, 0u, 0u);
                    }
                }
#pragma unroll
                for (int j = 0; j < kInst; ++j) acc ^= v[j].x ^ v[j].y ^ v[j].z ^ v[j].w;
            }
        }
    } else {
        constexpr int kStages = L / 32;
        constexpr uint32_t kStageWords = 32u * kLW;
        uint32_t* stage = stage_all + (threadIdx.x >> 5) * (kStageWords * kStages);
        const uint32_t stage_s = (uint32_t)__cvta_generic_to_shared(stage);
        auto issue = [&](uint64_t gr, int st) {
            const uint64_t r = gr * 32 + lane;
            const uint32_t my_line = (uint32_t)pick(r, seed, footprint);
            const uint32_t valid = __ballot_sync(0xFFFFFFFFu, gr < groups && r < n_reads);
#pragma unroll
            for (uint32_t j = 0; j < kLanesPerLine; ++j) {
                const uint32_t s = kLinesPerInst * j + g;
                const uint32_t line = __shfl_sync(0xFFFFFFFFu, my_line, s);
                if ((valid >> s) & 1u) {
                    const uint32_t dst = stage_s + ((uint32_t)st * kStageWords + s * kLW + c * 4u) * 4u;
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst),
                                 "l"(buf + (uint64_t)line * kLW + c * 4u)
                                 : "memory");
                }
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        auto consume = [&](int st) {
            // each lane xors one word of every line of the round
#pragma unroll 8
            for (uint32_t k = lane; k < kStageWords; k += 32u) acc ^= stage[st * kStageWords + k];
        };
        int st = 0;
        if (warp < groups) issue(warp, 0);
        for (uint64_t gr = warp; gr < groups; gr += nwarps) {
            if constexpr (kStages == 2) {
                issue(gr + nwarps, st ^ 1);
                asm volatile("cp.async.wait_group 1;" ::: "memory");
            } else {
                asm volatile("cp.async.wait_group 0;" ::: "memory");
            }
            __syncwarp();
            consume(st);
            __syncwarp();
            if constexpr (kStages == 2) {
                st ^= 1;
            } else if (gr + nwarps < groups) {
                issue(gr + nwarps, 0);
            }
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");
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

int occupancy_grid(const void* fn, int tpb, size_t smem = 0) {
    int dev = 0, sms = 0, bps = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, tpb, smem);
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

int slab_probe_random_lines_v4(const uint32_t* d_buf, uint64_t footprint_lines, uint64_t n_reads, uint32_t seed,
                               int form, int line_bytes, int lines_in_flight, int threads_per_block, uint32_t* d_sink,
                               void* stream) {
    if (!d_buf || !d_sink || footprint_lines == 0 || footprint_lines >= (1ull << 32) || threads_per_block < 32 ||
        threads_per_block > 1024 || threads_per_block % 32 || (form != 0 && form != 1) ||
        (line_bytes != 64 && line_bytes != 128))
        return SLAB_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int tpb = threads_per_block;
    auto run = [&](auto lw) -> int {
        constexpr uint32_t LW = decltype(lw)::value;
        if (form == 0) {
#define LAUNCH(L)                                                                                          \
    case L: {                                                                                              \
        if constexpr (L >= (int)(128u / LW)) {                                                             \
            const int g = occupancy_grid((const void*)probe_lines_v4_kernel<false, L, LW>, tpb);           \
            probe_lines_v4_kernel<false, L, LW><<<g, tpb, 0, s>>>(d_buf, footprint_lines, n_reads, seed, d_sink); \
            break;                                                                                         \
        } else {                                                                                           \
            return SLAB_ERR_INVALID_ARG;                                                                   \
        }                                                                                                  \
    }
            switch (lines_in_flight) {
                LAUNCH(4) LAUNCH(8) LAUNCH(16) LAUNCH(32)
                default: return SLAB_ERR_INVALID_ARG;
            }
#undef LAUNCH
        } else {
            const size_t smem = (size_t)(tpb / 32) * (32u * LW * 4u) * (size_t)(lines_in_flight / 32);
            int dev = 0, optin = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
            if (smem > (size_t)optin) return SLAB_ERR_INVALID_ARG;
#define LAUNCH(L)                                                                                          \
    case L: {                                                                                              \
        const void* fn = (const void*)probe_lines_v4_kernel<true, L, LW>;                                  \
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) \
            return SLAB_ERR_CUDA;                                                                          \
        const int g = occupancy_grid(fn, tpb, smem);                                                       \
        probe_lines_v4_kernel<true, L, LW><<<g, tpb, smem, s>>>(d_buf, footprint_lines, n_reads, seed, d_sink); \
        break;                                                                                             \
    }
            switch (lines_in_flight) {
                LAUNCH(32) LAUNCH(64)
                default: return SLAB_ERR_INVALID_ARG;
            }
#undef LAUNCH
        }
        return cudaGetLastError() == cudaSuccess ? SLAB_OK : SLAB_ERR_CUDA;
    };
    return line_bytes == 64 ? run(std::integral_constant<uint32_t, 16u>{}) : run(std::integral_constant<uint32_t, 32u>{});
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
