// The table object behind the opaque slab_table handle, shared by the C-ABI
// translation units.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "../../include/slabhash.h"
#include "slab_device.cuh"

struct slab_host_io;  // staging of batches from host memory (host_batch.cu)

struct slab_table {
    int device = 0;
    int sm_count = 0;
    uint32_t num_buckets = 0;
    int mode = 0;
    uint32_t slab_words = 32;         // words per slab: 32 (128-byte slabs) or 16 (64-byte slabs)
    uint32_t hash_a = 0, hash_b = 0;
    uint64_t fastmod_m = 0;
    uint64_t pool_slabs = 0;
    uint32_t num_blocks = 0;
    uint32_t* d_slabs = nullptr;      // base slabs then pool
    uint32_t* d_bitmaps = nullptr;
    uint32_t* d_misc = nullptr;       // [0] status word, [2..] 8 x u64 counters
    float* d_model = nullptr;         // learned bucket function: root (a, b), then 1024 leaves (a, b)
    uint64_t device_bytes = 0;
    int max_smem_optin = 0;
    int l2_bytes = 0;
    slab_config cfg{};
    uint32_t epoch = 0;
    bool learned = false;             // bucket function in use: learned model or universal hash
    bool model_fitted = false;
    bool dirty = false;               // a batch may have stored keys since create / reset
    bool owns_memory = true;          // false for a table that lives inside a slab_group's arena
    bool multiset = false;            // duplicates allowed (INSERT), deletes empty their slot
    int occupancy[2][4] = {};         // resident blocks per SM by [variant][kernel kind] for cfg; 0 = not yet asked
    slab_host_io* host_io = nullptr;  // device staging of slab_batch_host, made on its first call
};

namespace slab_host {

// Frees the table's staging for batches from host memory (host_batch.cu).
void free_host_io(slab_table* t);

inline unsigned long long* counters(const slab_table* t) {
    return reinterpret_cast<unsigned long long*>(t->d_misc + 2);
}

inline slab::TableView view(slab_table* t) {
    slab::TableView v;
    v.slabs = t->d_slabs;
    v.pool = t->d_slabs + (uint64_t)t->num_buckets * t->slab_words;
    v.bitmaps = t->d_bitmaps;
    v.status = t->d_misc;
    v.model = t->d_model;
    v.fastmod_m = t->fastmod_m;
    v.num_buckets = t->num_buckets;
    v.hash_a = t->hash_a;
    v.hash_b = t->hash_b;
    v.num_blocks = t->num_blocks;
    v.pool_units = (uint32_t)t->pool_slabs;
    v.iter_limit = t->cfg.iter_limit;
    v.random_probes = t->cfg.random_probes;
    v.epoch = ++t->epoch;
    v.prefetch_l2 = (uint64_t)t->num_buckets * t->slab_words * 4ull > (uint64_t)t->l2_bytes / 2;
    v.learned = t->learned ? 1u : 0u;
    v.multiset = t->multiset ? 1u : 0u;
    v.slab_words = t->slab_words;
    return v;
}

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

inline int launch_rc() {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SLAB_OK : SLAB_ERR_CUDA;
}

inline uint32_t util_grid(const slab_table* t, uint64_t work, int tpb) {
    const uint64_t want = (work + tpb - 1) / tpb;
    return (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)t->sm_count * 8));
}

}  // namespace slab_host
