// Serving engine: continuous batching of mixed-op requests on one resident table.
//
// The server owns a fixed number of slots. A slot has its own non-blocking
// stream, an event, and pinned host and device staging for up to
// max_request_ops ops. Work on a slot is one batch: its inputs reach the
// device, one mixed batch runs on the table, a small kernel counts the
// allocated pool slabs, the outputs (results, found flags, slab count) reach
// the host, and the event is recorded. Batches in different slots overlap on
// the device.
//
// How a batch's inputs and outputs move, per direction:
//   staged  packed into / out of the slot's pinned records: one copy each way
//           (any caller memory; the choice for small batches);
//   copy    DMA straight between the caller's page-locked arrays and the slot's
//           device buffers: three copies in, two out, no host memcpy;
//   mapped  (SLAB_SERVER_ZERO_COPY) the kernels read the caller's page-locked,
//           device-mapped arrays and write the results into them in place, over
//           the CPU-GPU link: no copies at all.
//
// slab_server_submit runs each request as its own batch. slab_server_run serves
// an arrival trace with continuous batching: whenever a slot is free it takes
// every request that has arrived and is not yet running, in arrival order, up
// to the slot's capacity and the pool bound, as one batch; requests that arrive
// meanwhile wait for the next free slot. With few requests in flight each gets
// a launch (low latency); under load many share one (high throughput).
//
// Admission by free SlabAlloc memory: a list grows only when its last slab is
// full, so the pool slabs that k inserts link are at most k (a warp holds at
// most one unlinked slab at a time). A batch with k inserts is admitted only if
// measured + reserved + k <= high_water * pool_slabs, where `measured` is the
// largest slab count reported by a finished batch and `reserved` sums the
// inserts of admitted batches whose count has not been folded in. Each count
// starts after its own batch ends, on its stream, and reads the bitmaps through
// L2, so the count that started last sees every allocation of every batch
// folded in before it; allocation never shrinks on this path (deletes leave
// tombstones). The bound therefore always covers the pool in use. With
// SLAB_SERVER_GROW_POOL a request that does not fit while nothing is in flight
// grows the pool (slab_grow_pool) instead of being refused.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/slabhash.h"
#include "slab_device.cuh"
#include "slab_table.cuh"

using slab_host::launch_rc;

namespace {

constexpr int kCountThreads = 512;
constexpr int kCountBlocks = 32;
// Batches of at most this many ops move through the staging records even when
// the caller's arrays are page-locked: one copy each way beats five small ones.
constexpr uint32_t kStageOps = 8192;

// Allocated pool units: popcount of the table's bitmap words. Each block writes
// its partial sum; the last block to finish (ticket) adds them, writes the total
// to *out (device memory or mapped host memory) and re-arms the ticket, so no
// memset is needed between uses. Bitmap reads go through L2 (ld.global.cg)
// because other streams' batches may be setting bits meanwhile; a word read
// mid-update counts either its old or its new bits.
__global__ void __launch_bounds__(kCountThreads) count_allocated_kernel(const uint32_t* words, uint64_t n,
                                                                        unsigned long long* partials,
                                                                        unsigned int* ticket,
                                                                        unsigned long long* out) {
    __shared__ unsigned long long part[kCountThreads / 32];
    __shared__ bool last;
    unsigned long long c = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * kCountThreads + threadIdx.x; i < n; i += (uint64_t)gridDim.x * kCountThreads)
        c += __popc(__ldcg(words + i));
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xFFFFFFFFu, c, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x < 32) {
        c = threadIdx.x < kCountThreads / 32 ? part[threadIdx.x] : 0;
        for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xFFFFFFFFu, c, o);
        if (threadIdx.x == 0) {
            partials[blockIdx.x] = c;
            __threadfence();
            last = atomicAdd(ticket, 1u) == gridDim.x - 1;
        }
    }
    __syncthreads();
    if (last && threadIdx.x < 32) {
        c = threadIdx.x < gridDim.x ? __ldcg(partials + threadIdx.x) : 0;
        for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xFFFFFFFFu, c, o);
        if (threadIdx.x == 0) {
            *out = c;
            *ticket = 0;
        }
    }
}

inline uint64_t up16(uint64_t x) { return (x + 15) & ~uint64_t(15); }

// Input record: keys | values | ops.
struct InLayout {
    uint64_t values, ops, bytes;
    explicit InLayout(uint64_t n) : values(up16(4 * n)), ops(values + up16(4 * n)), bytes(ops + up16(n)) {}
};
// Output record: slab count (u64) | count ticket (u32) | pad | count partials | results | found.
// The count fields sit at fixed offsets whatever the batch size.
constexpr uint64_t kTicketOff = 8, kPartialsOff = 16, kTail = kPartialsOff + 8 * kCountBlocks;
static_assert(kTail % 16 == 0 && kCountBlocks <= 32, "count tail layout");
struct OutLayout {
    uint64_t found, bytes;
    explicit OutLayout(uint64_t n) : found(kTail + up16(4 * n)), bytes(found + up16(n)) {}
};

enum Move { kStaged, kCopy, kMapped };

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    uint8_t *h_in = nullptr, *h_out = nullptr, *d_in = nullptr, *d_out = nullptr;
    unsigned long long* h_out_dev = nullptr;  // device alias of h_out (mapped pinned memory), or null
    bool busy = false;      // holds work (running, or finished and not handed back)
    bool absorbed = false;  // its slab count has been folded into the admission state
    Move out_move = kStaged;
    uint64_t ticket = 0;    // slab_server_submit requests (one per slot)
    uint32_t n = 0;         // ops in the slot
    uint64_t reserved = 0;
    uint64_t r0 = 0, r1 = 0, a = 0;  // slab_server_run batches: requests [r0, r1), first op a
};

}  // namespace

struct slab_server {
    slab_table* table = nullptr;
    uint32_t max_ops = 0;
    uint32_t flags = 0;
    double high_water = 0.9;
    std::vector<Slot> slots;
    uint64_t next_ticket = 1;
    uint64_t measured = 0;
    uint64_t reserved = 0;
    slab_server_stats stats{};
};

namespace {

void release_slot(Slot& s) {
    if (s.stream) cudaStreamSynchronize(s.stream);
    cudaFreeHost(s.h_in);
    cudaFreeHost(s.h_out);
    cudaFree(s.d_in);
    cudaFree(s.d_out);
    if (s.done) cudaEventDestroy(s.done);
    if (s.stream) cudaStreamDestroy(s.stream);
    s = Slot{};
}

bool init_slot(Slot& s, uint32_t n) {
    const InLayout in(n);
    const OutLayout out(n);
    if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaHostAlloc(&s.h_in, in.bytes, cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc(&s.h_out, out.bytes, cudaHostAllocMapped) != cudaSuccess ||
        cudaMalloc(&s.d_in, in.bytes) != cudaSuccess || cudaMalloc(&s.d_out, out.bytes) != cudaSuccess ||
        cudaMemset(s.d_out, 0, kTail) != cudaSuccess)
        return false;
    void* alias = nullptr;
    if (cudaHostGetDevicePointer(&alias, s.h_out, 0) == cudaSuccess) s.h_out_dev = static_cast<unsigned long long*>(alias);
    else cudaGetLastError();  // no mapped alias: the zero-copy path stays off for this slot
    return true;
}

uint64_t bitmap_words(const slab_table* t) { return (uint64_t)t->num_blocks * 32; }

int queue_count(const slab_table* t, const Slot& s, unsigned long long* target) {
    const uint64_t words = bitmap_words(t);
    const uint32_t grid = (uint32_t)std::max<uint64_t>(
        1, std::min<uint64_t>(kCountBlocks, (words + kCountThreads - 1) / kCountThreads));
    count_allocated_kernel<<<grid, kCountThreads, 0, s.stream>>>(
        t->d_bitmaps, words, reinterpret_cast<unsigned long long*>(s.d_out + kPartialsOff),
        reinterpret_cast<unsigned int*>(s.d_out + kTicketOff), target);
    return launch_rc();
}

uint64_t count_inserts(const uint8_t* ops, uint32_t n) {
    uint64_t k = 0;
    for (uint32_t i = 0; i < n; ++i) k += ops[i] == SLAB_OP_INSERT;
    return k;
}

bool fits(const slab_server* sv, uint64_t inserts) {
    return (double)(sv->measured + sv->reserved + inserts) <= sv->high_water * (double)sv->table->pool_slabs;
}

// Fold the slab count of a finished batch into the admission state (once).
void absorb(slab_server* sv, Slot& s) {
    if (s.absorbed) return;
    uint64_t c;
    std::memcpy(&c, s.h_out, 8);
    sv->measured = std::max(sv->measured, c);
    sv->reserved -= s.reserved;
    s.absorbed = true;
}

// Fold in every busy slot whose event has fired; CUDA errors surface here.
int poll(slab_server* sv) {
    for (Slot& s : sv->slots) {
        if (!s.busy || s.absorbed) continue;
        const cudaError_t e = cudaEventQuery(s.done);
        if (e == cudaSuccess) absorb(sv, s);
        else if (e != cudaErrorNotReady) return SLAB_ERR_CUDA;
    }
    return SLAB_OK;
}

Slot* free_slot(slab_server* sv) {
    for (Slot& s : sv->slots)
        if (!s.busy) return &s;
    return nullptr;
}

// One batch's inputs and outputs. Host pointers for kStaged / kCopy; device
// aliases of mapped host memory for kMapped. results / found may be null when
// the caller wants no outputs (then the slot's device buffers take them).
struct Io {
    Move in, out;
    const uint8_t* ops;
    const uint32_t* keys;
    const uint32_t* values;
    uint32_t* results;
    uint8_t* found;
};

// Queue one batch of n ops on slot s (admission already decided).
int launch_ops(slab_server* sv, Slot& s, const Io& io, uint32_t n, uint64_t inserts) {
    slab_table* t = sv->table;
    const InLayout in(n);
    const OutLayout out(n);
    const uint32_t* d_keys = reinterpret_cast<const uint32_t*>(s.d_in);
    const uint32_t* d_values = io.values ? reinterpret_cast<const uint32_t*>(s.d_in + in.values) : nullptr;
    const uint8_t* d_ops = s.d_in + in.ops;
    switch (io.in) {
        case kMapped:
            d_keys = io.keys, d_values = io.values, d_ops = io.ops;
            break;
        case kCopy:
            if (cudaMemcpyAsync(s.d_in, io.keys, 4ull * n, cudaMemcpyHostToDevice, s.stream) != cudaSuccess ||
                (io.values && cudaMemcpyAsync(s.d_in + in.values, io.values, 4ull * n, cudaMemcpyHostToDevice,
                                              s.stream) != cudaSuccess) ||
                cudaMemcpyAsync(s.d_in + in.ops, io.ops, n, cudaMemcpyHostToDevice, s.stream) != cudaSuccess)
                return SLAB_ERR_CUDA;
            break;
        case kStaged:
            std::memcpy(s.h_in, io.keys, 4ull * n);
            if (io.values) std::memcpy(s.h_in + in.values, io.values, 4ull * n);
            std::memcpy(s.h_in + in.ops, io.ops, n);
            if (cudaMemcpyAsync(s.d_in, s.h_in, in.bytes, cudaMemcpyHostToDevice, s.stream) != cudaSuccess)
                return SLAB_ERR_CUDA;
            break;
    }
    uint32_t* d_results = reinterpret_cast<uint32_t*>(s.d_out + kTail);
    uint8_t* d_found = s.d_out + out.found;
    if (io.out == kMapped) {
        if (io.results) d_results = io.results;
        if (io.found) d_found = io.found;
    }
    int rc = slab_mixed_batch(t, d_ops, d_keys, d_values, d_results, d_found, n, s.stream);
    if (rc != SLAB_OK) return rc;
    auto* d_count = reinterpret_cast<unsigned long long*>(s.d_out);
    if ((rc = queue_count(t, s, io.out == kMapped ? s.h_out_dev : d_count)) != SLAB_OK) return rc;
    switch (io.out) {
        case kMapped:
            break;
        case kCopy:
            if ((io.results && cudaMemcpyAsync(io.results, d_results, 4ull * n, cudaMemcpyDeviceToHost, s.stream) !=
                                   cudaSuccess) ||
                (io.found && cudaMemcpyAsync(io.found, d_found, n, cudaMemcpyDeviceToHost, s.stream) != cudaSuccess) ||
                cudaMemcpyAsync(s.h_out, d_count, 8, cudaMemcpyDeviceToHost, s.stream) != cudaSuccess)
                return SLAB_ERR_CUDA;
            break;
        case kStaged:
            if (cudaMemcpyAsync(s.h_out, s.d_out, out.bytes, cudaMemcpyDeviceToHost, s.stream) != cudaSuccess)
                return SLAB_ERR_CUDA;
            break;
    }
    if (cudaEventRecord(s.done, s.stream) != cudaSuccess) return SLAB_ERR_CUDA;
    s.busy = true;
    s.absorbed = false;
    s.out_move = io.out;
    s.ticket = 0;
    s.n = n;
    s.reserved = inserts;
    sv->reserved += inserts;
    sv->stats.batches++;
    return SLAB_OK;
}

// Hand a finished staged batch's outputs to the caller (copy / mapped batches
// wrote them in place).
void copy_out(const Slot& s, uint32_t* results, uint8_t* found) {
    if (s.out_move != kStaged) return;
    const OutLayout out(s.n);
    if (results) std::memcpy(results, s.h_out + kTail, 4ull * s.n);
    if (found) std::memcpy(found, s.h_out + out.found, s.n);
}

void finish(Slot& s) {
    s.busy = false;
    s.ticket = 0;
}

void drain(slab_server* sv) {
    for (Slot& s : sv->slots)
        if (s.busy) cudaStreamSynchronize(s.stream);
}

// Page-locked host memory: whether the device can DMA it, and its device alias
// when it is also mapped (null otherwise). Null pointers count as both.
struct HostMem {
    bool pinned;
    const void* alias;
};
HostMem host_mem(const void* p) {
    if (!p) return {true, nullptr};
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return {false, nullptr};
    }
    if (a.type != cudaMemoryTypeHost) return {false, nullptr};
    return {true, a.devicePointer};
}

// Grow the table's pool (Sec. 5, more super blocks) so that `inserts` more fit
// under the bound: by at least half of the current pool, to keep growth rare.
// Only called with nothing in flight on the server's slots.
int grow_for(slab_server* sv, uint64_t inserts) {
    slab_table* t = sv->table;
    const double need = (double)(sv->measured + sv->reserved + inserts) / sv->high_water - (double)t->pool_slabs;
    const uint64_t extra = std::max<uint64_t>((uint64_t)need + 1, t->pool_slabs / 2);
    const int rc = slab_grow_pool(t, extra);
    if (rc == SLAB_OK) sv->stats.pool_grown++;
    return fits(sv, inserts) ? rc : SLAB_ERR_OUT_OF_SLABS;
}

using Clock = std::chrono::steady_clock;
inline uint64_t ns_since(Clock::time_point t0) {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now() - t0).count();
}

}  // namespace

extern "C" {

int slab_server_create(slab_table* t, uint32_t slots, uint32_t max_request_ops, double pool_high_water,
                       uint32_t flags, slab_server** out) {
    if (!out) return SLAB_ERR_INVALID_ARG;
    *out = nullptr;
    if (!t || slots == 0 || slots > SLAB_SERVER_MAX_SLOTS || max_request_ops == 0 ||
        max_request_ops > SLAB_SERVER_MAX_REQUEST_OPS || !(pool_high_water > 0.0) || pool_high_water > 1.0 ||
        (flags & ~(SLAB_SERVER_ZERO_COPY | SLAB_SERVER_GROW_POOL)))
        return SLAB_ERR_INVALID_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return SLAB_ERR_CUDA;
    if (dev != t->device) return SLAB_ERR_INVALID_ARG;
    slab_server* sv = new (std::nothrow) slab_server();
    if (!sv) return SLAB_ERR_CUDA;
    sv->table = t;
    sv->max_ops = max_request_ops;
    sv->flags = flags;
    sv->high_water = pool_high_water;
    sv->slots.resize(slots);
    for (Slot& s : sv->slots) {
        if (!init_slot(s, max_request_ops)) {
            cudaGetLastError();
            slab_server_destroy(sv);
            return SLAB_ERR_CUDA;
        }
    }
    // the pool in use now (the table may already hold keys)
    Slot& s0 = sv->slots[0];
    auto* d_count = reinterpret_cast<unsigned long long*>(s0.d_out);
    if (queue_count(t, s0, d_count) != SLAB_OK ||
        cudaMemcpyAsync(s0.h_out, d_count, 8, cudaMemcpyDeviceToHost, s0.stream) != cudaSuccess ||
        cudaStreamSynchronize(s0.stream) != cudaSuccess) {
        slab_server_destroy(sv);
        return SLAB_ERR_CUDA;
    }
    std::memcpy(&sv->measured, s0.h_out, 8);
    *out = sv;
    return SLAB_OK;
}

void slab_server_destroy(slab_server* sv) {
    if (!sv) return;
    for (Slot& s : sv->slots) release_slot(s);
    delete sv;
}

int slab_server_submit(slab_server* sv, const uint8_t* h_ops, const uint32_t* h_keys, const uint32_t* h_values,
                       uint32_t n, uint64_t* ticket) {
    if (!sv || !ticket || n == 0 || n > sv->max_ops || !h_ops || !h_keys ||
        (!h_values && sv->table->mode == SLAB_MODE_KEY_VALUE))
        return SLAB_ERR_INVALID_ARG;
    *ticket = 0;
    if (sv->table->mode == SLAB_MODE_KEY_ONLY) h_values = nullptr;
    int rc = poll(sv);
    if (rc != SLAB_OK) return rc;
    Slot* s = free_slot(sv);
    if (!s) {
        sv->stats.deferred_slot++;
        return SLAB_ERR_BUSY;
    }
    const uint64_t k = count_inserts(h_ops, n);
    if (!fits(sv, k)) {
        bool any_busy = false;
        for (const Slot& o : sv->slots) any_busy |= o.busy;
        if (any_busy || !(sv->flags & SLAB_SERVER_GROW_POOL) || grow_for(sv, k) != SLAB_OK) {
            sv->stats.deferred_memory++;
            return SLAB_ERR_OUT_OF_SLABS;
        }
    }
    // the caller may reuse its arrays as soon as this returns: always staged
    const Io io{kStaged, kStaged, h_ops, h_keys, h_values, nullptr, nullptr};
    if ((rc = launch_ops(sv, *s, io, n, k)) != SLAB_OK) return rc;
    s->ticket = sv->next_ticket++;
    sv->stats.submitted++;
    *ticket = s->ticket;
    return SLAB_OK;
}

int slab_server_collect(slab_server* sv, uint64_t ticket, uint32_t* h_results, uint8_t* h_found, int wait) {
    if (!sv || ticket == 0) return SLAB_ERR_INVALID_ARG;
    for (Slot& s : sv->slots) {
        if (!s.busy || s.ticket != ticket) continue;
        const cudaError_t e = wait ? cudaEventSynchronize(s.done) : cudaEventQuery(s.done);
        if (e == cudaErrorNotReady) return SLAB_ERR_BUSY;
        if (e != cudaSuccess) return SLAB_ERR_CUDA;
        absorb(sv, s);
        copy_out(s, h_results, h_found);
        finish(s);
        sv->stats.completed++;
        return SLAB_OK;
    }
    return SLAB_ERR_INVALID_ARG;  // unknown, or already collected
}

int slab_server_get_stats(slab_server* sv, slab_server_stats* out) {
    if (!sv || !out) return SLAB_ERR_INVALID_ARG;
    const int rc = poll(sv);
    *out = sv->stats;
    out->pool_slabs = sv->table->pool_slabs;
    out->pool_measured = sv->measured;
    out->pool_reserved = sv->reserved;
    out->inflight = 0;
    for (const Slot& s : sv->slots) out->inflight += s.busy;
    return rc;
}

int slab_server_run(slab_server* sv, uint64_t n_requests, const uint64_t* h_arrival_ns, const uint64_t* h_op_start,
                    const uint8_t* h_ops, const uint32_t* h_keys, const uint32_t* h_values, uint32_t* h_results,
                    uint8_t* h_found, uint64_t* h_latency_ns, uint64_t* h_wait_ns, uint8_t* h_status,
                    uint64_t* h_makespan_ns) {
    if (!sv || !h_arrival_ns || !h_op_start || !h_status || (n_requests && h_op_start[0] != 0))
        return SLAB_ERR_INVALID_ARG;
    const uint64_t total = h_op_start[n_requests];
    const bool key_only = sv->table->mode == SLAB_MODE_KEY_ONLY;
    if (total && (!h_ops || !h_keys || (!h_values && !key_only))) return SLAB_ERR_INVALID_ARG;
    for (uint64_t r = 0; r < n_requests; ++r) {
        if (h_op_start[r + 1] < h_op_start[r] || h_op_start[r + 1] - h_op_start[r] > sv->max_ops ||
            (r && h_arrival_ns[r] < h_arrival_ns[r - 1]))
            return SLAB_ERR_INVALID_ARG;
    }
    for (const Slot& s : sv->slots)
        if (s.busy) return SLAB_ERR_BUSY;  // tickets from slab_server_submit are still out
    if (key_only) h_values = nullptr;

    std::vector<uint64_t> inserts(n_requests);
    for (uint64_t r = 0; r < n_requests; ++r)
        inserts[r] = count_inserts(h_ops + h_op_start[r], (uint32_t)(h_op_start[r + 1] - h_op_start[r]));

    // how inputs and outputs move: mapped (zero-copy, if asked and possible),
    // else DMA from / to page-locked arrays for large batches, else staged
    const HostMem m_ops = host_mem(h_ops), m_keys = host_mem(h_keys), m_vals = host_mem(h_values);
    const HostMem m_res = host_mem(h_results), m_found = host_mem(h_found);
    bool slots_mapped = true;
    for (const Slot& s : sv->slots) slots_mapped &= s.h_out_dev != nullptr;
    const bool zero_copy = (sv->flags & SLAB_SERVER_ZERO_COPY) && slots_mapped && total;
    const bool in_pinned = m_ops.pinned && m_keys.pinned && m_vals.pinned;
    const bool out_pinned = m_res.pinned && m_found.pinned;
    const bool in_mapped = zero_copy && in_pinned && m_ops.alias && m_keys.alias && (m_vals.alias || !h_values);
    const bool out_mapped = zero_copy && out_pinned && (m_res.alias || !h_results) && (m_found.alias || !h_found);
    auto alias = [](const HostMem& m, const void* base, uint64_t byte_off) -> const uint8_t* {
        return m.alias ? static_cast<const uint8_t*>(m.alias) + byte_off : static_cast<const uint8_t*>(base);
    };

    const Clock::time_point t0 = Clock::now();
    uint64_t next = 0, done = 0, last = 0, held_slot = ~0ull, held_memory = ~0ull;
    int rc = SLAB_OK;
    auto complete = [&](uint64_t r, uint64_t now, uint8_t status) {
        if (h_latency_ns) h_latency_ns[r] = now - h_arrival_ns[r];
        h_status[r] = status;
        last = std::max(last, now);
        ++done;
        if (status == SLAB_OK) sv->stats.completed++;
    };
    while (done < n_requests && rc == SLAB_OK) {
        // retire finished batches
        for (Slot& s : sv->slots) {
            if (!s.busy) continue;
            const cudaError_t e = cudaEventQuery(s.done);
            if (e == cudaErrorNotReady) continue;
            if (e != cudaSuccess) {
                rc = SLAB_ERR_CUDA;
                break;
            }
            const uint64_t now = ns_since(t0);
            absorb(sv, s);
            copy_out(s, h_results ? h_results + s.a : nullptr, h_found ? h_found + s.a : nullptr);
            finish(s);
            for (uint64_t r = s.r0; r < s.r1; ++r) complete(r, now, SLAB_OK);
        }
        if (rc != SLAB_OK) break;
        // continuous batching: every free slot takes all arrived requests that fit
        while (next < n_requests) {
            const uint64_t now = ns_since(t0);
            if (now < h_arrival_ns[next]) break;
            Slot* s = free_slot(sv);
            if (!s) {
                if (held_slot != next) sv->stats.deferred_slot++, held_slot = next;
                break;
            }
            uint64_t r = next, ops = 0, ins = 0;
            while (r < n_requests && h_arrival_ns[r] <= now) {
                const uint64_t n = h_op_start[r + 1] - h_op_start[r];
                if (ops + n > sv->max_ops || !fits(sv, ins + inserts[r])) break;
                ops += n;
                ins += inserts[r];
                ++r;
            }
            if (r == next) {  // the head request does not fit the pool bound
                bool any_busy = false;
                for (const Slot& o : sv->slots) any_busy |= o.busy;
                if (any_busy) {  // reservations come back as batches finish
                    if (held_memory != next) sv->stats.deferred_memory++, held_memory = next;
                    break;
                }
                // nothing in flight: grow the pool if allowed, else the pool cannot
                // take this request now or later
                if ((sv->flags & SLAB_SERVER_GROW_POOL) && grow_for(sv, inserts[next]) == SLAB_OK) continue;
                if (h_wait_ns) h_wait_ns[next] = now - h_arrival_ns[next];
                sv->stats.rejected_memory++;
                complete(next++, now, SLAB_ERR_OUT_OF_SLABS);
                continue;
            }
            for (uint64_t q = next; q < r; ++q)
                if (h_wait_ns) h_wait_ns[q] = now - h_arrival_ns[q];
            sv->stats.submitted += r - next;
            if (ops == 0) {  // only empty requests
                for (uint64_t q = next; q < r; ++q) complete(q, now, SLAB_OK);
                next = r;
                continue;
            }
            const uint64_t a = h_op_start[next];
            Io io;
            io.in = in_mapped ? kMapped : (in_pinned && ops > kStageOps ? kCopy : kStaged);
            io.out = out_mapped ? kMapped : (out_pinned && ops > kStageOps ? kCopy : kStaged);
            const bool in_alias = io.in == kMapped, out_alias = io.out == kMapped;
            io.ops = in_alias ? alias(m_ops, h_ops, a) : h_ops + a;
            io.keys = reinterpret_cast<const uint32_t*>(in_alias ? alias(m_keys, h_keys, 4 * a)
                                                                 : reinterpret_cast<const uint8_t*>(h_keys + a));
            io.values = !h_values ? nullptr
                                  : reinterpret_cast<const uint32_t*>(
                                        in_alias ? alias(m_vals, h_values, 4 * a)
                                                 : reinterpret_cast<const uint8_t*>(h_values + a));
            io.results = !h_results ? nullptr
                                    : reinterpret_cast<uint32_t*>(const_cast<uint8_t*>(
                                          out_alias ? alias(m_res, h_results, 4 * a)
                                                    : reinterpret_cast<const uint8_t*>(h_results + a)));
            io.found = !h_found ? nullptr
                                : const_cast<uint8_t*>(out_alias ? alias(m_found, h_found, a) : h_found + a);
            if (io.out == kCopy && !h_results && !h_found) io.out = kStaged;
            if ((rc = launch_ops(sv, *s, io, (uint32_t)ops, ins)) != SLAB_OK) break;
            s->r0 = next;
            s->r1 = r;
            s->a = a;
            next = r;
        }
    }
    if (rc != SLAB_OK) {
        drain(sv);
        for (Slot& s : sv->slots)
            if (s.busy) {
                absorb(sv, s);
                finish(s);
            }
        return rc;
    }
    if (h_makespan_ns) *h_makespan_ns = last;
    return SLAB_OK;
}

}  // extern "C"
