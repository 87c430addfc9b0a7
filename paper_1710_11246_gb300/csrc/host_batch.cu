// Batches whose arrays live in host memory (slab_batch_host in slabhash.h).
//
// The table owns kSets sets of device staging buffers of `chunk` ops each and two
// copy streams. A batch of n ops runs as ceil(n / chunk) chunks in order: chunk c
// goes to the next set of the ring, its inputs are copied in on the input stream, its kernel
// runs on the caller's stream, and its results are copied out on the output
// stream; events order each set's three steps and keep a set from being refilled
// before its previous results have left. So the copies of one chunk overlap the
// kernels of its neighbours, and the calls of successive batches overlap in the
// same way. Splitting a batch into chunks run in order gives the results of the
// whole batch: every op of a batch acts on its own key.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <new>

#include "../../include/slabhash.h"
#include "slab_table.cuh"

using slab_host::S;

// Staging sets: the input copies can run this many chunks ahead of the kernels
// (a set is refilled only after its previous results have left).
#ifndef SLAB_HOST_SETS
#define SLAB_HOST_SETS 4
#endif
constexpr int kSets = SLAB_HOST_SETS;

struct slab_host_io {
    uint32_t chunk = 0;  // ops per staging set
    uint8_t* d_ops[kSets] = {};
    uint32_t* d_keys[kSets] = {};
    uint32_t* d_values[kSets] = {};
    uint32_t* d_results[kSets] = {};
    uint8_t* d_found[kSets] = {};
    cudaStream_t s_in = nullptr, s_out = nullptr;
    cudaEvent_t in_ready[kSets] = {}, done[kSets] = {}, freed[kSets] = {};
    uint32_t next_set = 0;
};

namespace {

constexpr uint32_t kDefaultChunk = 1u << 22;  // each chunk is a kernel launch with a fixed cost of ~10 us

void release(slab_host_io* h) {
    if (!h) return;
    for (int i = 0; i < kSets; ++i) {
        cudaFree(h->d_ops[i]);
        cudaFree(h->d_keys[i]);
        cudaFree(h->d_values[i]);
        cudaFree(h->d_results[i]);
        cudaFree(h->d_found[i]);
        if (h->in_ready[i]) cudaEventDestroy(h->in_ready[i]);
        if (h->done[i]) cudaEventDestroy(h->done[i]);
        if (h->freed[i]) cudaEventDestroy(h->freed[i]);
    }
    if (h->s_in) cudaStreamDestroy(h->s_in);
    if (h->s_out) cudaStreamDestroy(h->s_out);
    delete h;
}

// The table's staging for chunks of at least `chunk` ops (made on first use,
// remade larger when a call asks for more).
slab_host_io* staging(slab_table* t, uint32_t chunk) {
    if (t->host_io && t->host_io->chunk >= chunk) return t->host_io;
    if (t->host_io) {
        if (cudaDeviceSynchronize() != cudaSuccess) return nullptr;
        release(t->host_io);
        t->host_io = nullptr;
    }
    slab_host_io* h = new (std::nothrow) slab_host_io();
    if (!h) return nullptr;
    h->chunk = chunk;
    bool ok = cudaStreamCreateWithFlags(&h->s_in, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&h->s_out, cudaStreamNonBlocking) == cudaSuccess;
    for (int i = 0; ok && i < kSets; ++i) {
        ok = cudaMalloc(&h->d_ops[i], chunk) == cudaSuccess &&
             cudaMalloc(&h->d_keys[i], 4ull * chunk) == cudaSuccess &&
             cudaMalloc(&h->d_values[i], 4ull * chunk) == cudaSuccess &&
             cudaMalloc(&h->d_results[i], 4ull * chunk) == cudaSuccess &&
             cudaMalloc(&h->d_found[i], chunk) == cudaSuccess &&
             cudaEventCreateWithFlags(&h->in_ready[i], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&h->done[i], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&h->freed[i], cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        release(h);
        return nullptr;
    }
    t->host_io = h;
    return h;
}

}  // namespace

namespace slab_host {
void free_host_io(slab_table* t) {
    release(t->host_io);
    t->host_io = nullptr;
}
}  // namespace slab_host

extern "C" int slab_batch_host(slab_table* t, int kind, const uint8_t* h_ops, const uint32_t* h_keys,
                               const uint32_t* h_values, uint32_t* h_results, uint8_t* h_found, uint32_t n,
                               uint32_t chunk, void* stream, void* done_event) {
    if (!t || kind < SLAB_BATCH_INSERT || kind > SLAB_BATCH_MIXED) return SLAB_ERR_INVALID_ARG;
    if (n == 0) return SLAB_OK;
    const bool kv = t->mode == SLAB_MODE_KEY_VALUE;
    if (!h_keys || (kind == SLAB_BATCH_MIXED && (!h_ops || !h_results)) ||
        (kind == SLAB_BATCH_INSERT && kv && !h_values) || (kind == SLAB_BATCH_SEARCH && !h_results))
        return SLAB_ERR_INVALID_ARG;
    if (chunk == 0) chunk = kDefaultChunk;
    slab_host_io* h = staging(t, std::min(chunk, n));
    if (!h) return SLAB_ERR_CUDA;
    chunk = std::min(chunk, h->chunk);
    const cudaStream_t ks = S(stream);
    const bool values_in = (kind == SLAB_BATCH_INSERT || kind == SLAB_BATCH_MIXED) && h_values;
    int rc = SLAB_OK;
    for (uint32_t off = 0; off < n && rc == SLAB_OK; off += chunk) {
        const uint32_t m = std::min(chunk, n - off);
        const uint32_t i = h->next_set;
        h->next_set = (h->next_set + 1u) % kSets;
        // inputs: once this set's previous results have left
        if (cudaStreamWaitEvent(h->s_in, h->freed[i], 0) != cudaSuccess ||
            cudaMemcpyAsync(h->d_keys[i], h_keys + off, 4ull * m, cudaMemcpyHostToDevice, h->s_in) != cudaSuccess ||
            (kind == SLAB_BATCH_MIXED &&
             cudaMemcpyAsync(h->d_ops[i], h_ops + off, m, cudaMemcpyHostToDevice, h->s_in) != cudaSuccess) ||
            (values_in &&
             cudaMemcpyAsync(h->d_values[i], h_values + off, 4ull * m, cudaMemcpyHostToDevice, h->s_in) != cudaSuccess) ||
            cudaEventRecord(h->in_ready[i], h->s_in) != cudaSuccess || cudaStreamWaitEvent(ks, h->in_ready[i], 0) != cudaSuccess) {
            rc = SLAB_ERR_CUDA;
            break;
        }
        // the chunk's batch on the caller's stream
        uint8_t* fd = h_found ? h->d_found[i] : nullptr;
        switch (kind) {
            case SLAB_BATCH_INSERT:
                rc = slab_insert_batch(t, h->d_keys[i], values_in ? h->d_values[i] : nullptr, fd, m, stream);
                break;
            case SLAB_BATCH_DELETE:
                rc = slab_delete_batch(t, h->d_keys[i], fd, m, stream);
                break;
            case SLAB_BATCH_SEARCH:
                rc = slab_search_batch(t, h->d_keys[i], h->d_results[i], fd, m, stream);
                break;
            default:
                rc = slab_mixed_batch(t, h->d_ops[i], h->d_keys[i], values_in ? h->d_values[i] : nullptr,
                                      h->d_results[i], fd, m, stream);
        }
        if (rc != SLAB_OK) break;
        // results out, then the set is free again
        if (cudaEventRecord(h->done[i], ks) != cudaSuccess || cudaStreamWaitEvent(h->s_out, h->done[i], 0) != cudaSuccess ||
            (h_results && kind != SLAB_BATCH_INSERT && kind != SLAB_BATCH_DELETE &&
             cudaMemcpyAsync(h_results + off, h->d_results[i], 4ull * m, cudaMemcpyDeviceToHost, h->s_out) != cudaSuccess) ||
            (h_found && cudaMemcpyAsync(h_found + off, h->d_found[i], m, cudaMemcpyDeviceToHost, h->s_out) != cudaSuccess) ||
            cudaEventRecord(h->freed[i], h->s_out) != cudaSuccess) {
            rc = SLAB_ERR_CUDA;
            break;
        }
    }
    if (rc != SLAB_OK) return rc;
    if (done_event) {  // the copies out are in order: the last one queued finishes last
        return cudaEventRecord(reinterpret_cast<cudaEvent_t>(done_event), h->s_out) == cudaSuccess ? SLAB_OK
                                                                                                  : SLAB_ERR_CUDA;
    }
    // otherwise the caller's stream completes once every result is in host memory
    for (int i = 0; i < kSets; ++i)
        if (cudaStreamWaitEvent(ks, h->freed[i], 0) != cudaSuccess) return SLAB_ERR_CUDA;
    return SLAB_OK;
}
