// Warp-cooperative work sharing (WCWS, Sec. 4.1) over slab lists: the two
// kernel families that serve search / replace / delete / mixed batches.
//
//   direct_kernel  the loop of Fig. "alg:search" as written: one op per lane,
//                  the warp serves its queue one op at a time, each step reads
//                  the current slab from global memory.
//   staged_kernel  the same per-op WCWS step, reorganised for sm_103a memory
//                  latency: every lane keeps one pending op in a persistent
//                  window; each round the warp copies all pending ops' current
//                  slabs into its shared-memory stage with cp.async (up to 32
//                  independent 128-byte lines in flight per warp), then serves
//                  the ops one at a time from the stage. Insert CASes are issued
//                  without waiting and checked at the end of the round; a lane
//                  whose op finished takes the next op of the warp's range.
#pragma once
#include "slab_device.cuh"

namespace slab {

// What one WCWS step concluded for the source lane's op (warp-uniform).
enum : uint32_t {
    kResolved = 0,  // done: a = result, b = found
    kAdvance = 1,   // follow the next pointer a
    kMarkDead = 2,  // delete hit at key lane a: write the tombstone, done
    kClaim = 3,     // insert: CAS the pair at key lane a (observed key b, value c)
    kNeedSlab = 4   // insert: slab full and its next pointer empty
};
struct Outcome {
    uint32_t kind, a, b, c;
};

// One WCWS step (Sec. 4.3, Fig. "alg:search" search / replace / delete macros):
// every lane holds word `lane` of the slab; `skey` and `sop` belong to the source
// lane. Ballots find a matching key (or, for insert, the first empty-or-matching
// pair); a miss hands over the address lane's next pointer.
template <bool kKeyOnly>
__device__ __forceinline__ Outcome examine(uint32_t data, uint32_t sop, uint32_t skey) {
    constexpr uint32_t kMask = kKeyOnly ? kKeyLanesKeyOnly : kKeyLanesKV;
    Outcome o;
    if (sop == kOpInsert) {
        uint32_t m = __ballot_sync(kFull, data == kEmptyKey || data == skey) & kMask;
        if (m) {
            int d = __ffs(m) - 1;
            uint32_t ok = __shfl_sync(kFull, data, d);
            uint32_t ov = kKeyOnly ? 0u : __shfl_sync(kFull, data, d + 1);
            if (kKeyOnly && ok == skey) o = Outcome{kResolved, 0u, 1u, 0u};  // already present
            else o = Outcome{kClaim, (uint32_t)d, ok, ov};
        } else {
            uint32_t nx = __shfl_sync(kFull, data, kAddressLane);
            o = nx == kEmptyKey ? Outcome{kNeedSlab, 0u, 0u, 0u} : Outcome{kAdvance, nx, 0u, 0u};
        }
    } else {
        uint32_t m = __ballot_sync(kFull, data == skey) & kMask;
        if (m) {
            int d = __ffs(m) - 1;
            if (sop == kOpSearch) {
                uint32_t v = kKeyOnly ? 0u : __shfl_sync(kFull, data, d + 1);
                o = Outcome{kResolved, v, 1u, 0u};
            } else {
                o = Outcome{kMarkDead, (uint32_t)d, 0u, 0u};
            }
        } else {
            uint32_t nx = __shfl_sync(kFull, data, kAddressLane);
            if (nx == kEmptyKey) o = Outcome{kResolved, sop == kOpSearch ? kNotFound : 0u, 0u, 0u};
            else o = Outcome{kAdvance, nx, 0u, 0u};
        }
    }
    return o;
}

template <int kKind>
__device__ __forceinline__ uint32_t fixed_op() {
    return kKind == kKindSearch ? kOpSearch : kKind == kKindInsert ? kOpInsert : kOpDelete;
}

// Result written for an op that never completes its walk (reserved key, cap, OOM).
__device__ __forceinline__ uint32_t default_result(uint32_t op) {
    return op == kOpSearch ? kNotFound : 0u;
}

// Warp-wide: allocate a slab and link it behind the full slab at `p` (the source
// lane's current slab). Returns the slab to continue with, or kAllocFailed.
// The link is a 32-bit CAS of the empty next pointer (Sec. 4.3.2); a warp that
// loses the race returns its slab to SlabAlloc and follows the winner's.
__device__ __forceinline__ uint32_t grow_list(const TableView& T, AllocCtx& ac, uint32_t warp_gid,
                                              uint32_t* p_src_lane, int s) {
    uint32_t na = warp_allocate(T, ac, warp_gid);
    if (na == kAllocFailed) return kAllocFailed;
    uint32_t old = 0;
    if ((int)lane_id() == s) old = atomicCAS(p_src_lane + kAddressLane, kEmptyKey, na);
    old = __shfl_sync(kFull, old, s);
    if (old == kEmptyKey) return na;
    if ((int)lane_id() == s) deallocate(T, na);
    return old;
}

__device__ __forceinline__ unsigned long long pack_pair(uint32_t key, uint32_t value) {
    return ((unsigned long long)value << 32) | key;
}

// ---------------------------------------------------------------------------
// Paper-structured kernel: Fig. "alg:search" with one op per lane.
// ---------------------------------------------------------------------------
template <int kKind, bool kKeyOnly>
__global__ void direct_kernel(TableView T, BatchArgs A) {
    constexpr bool kReadOnly = kKind == kKindSearch;
    const uint32_t lane = lane_id();
    const uint32_t warp_gid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t ntiles = (A.n + 31u) / 32u;
    AllocCtx ac{kNoBlock, 0u, 0u};

    for (uint32_t tile = warp_gid; tile < ntiles; tile += nwarps) {
        const uint32_t idx = tile * 32u + lane;
        const bool has = idx < A.n;
        uint32_t op = fixed_op<kKind>();
        if constexpr (kKind == kKindMixed) op = has ? ld_stream_u8(A.ops + idx) : 3u;
        const uint32_t key = has ? ld_stream(A.keys + idx) : 0u;
        uint32_t value = 0;
        if ((kKind == kKindInsert || kKind == kKindMixed) && !kKeyOnly && A.values && has)
            value = ld_stream(A.values + idx);
        bool active = has && op <= kOpSearch;
        uint32_t res = default_result(op), fnd = 0;
        if (active && key >= kTombstone) {
            set_flag(T, kFlagReserved);
            active = false;
        }
        const uint32_t bucket = active ? bucket_of(T, key) : 0u;

        uint32_t queue = __ballot_sync(kFull, active);
        int prev = -1;
        uint32_t cur = kEmptyKey, iters = 0;
        while (queue) {
            const int s = __ffs(queue) - 1;
            if (s != prev) {  // the queue changed: start the new source lane at its base slab
                prev = s;
                cur = kEmptyKey;
                iters = 0;
            }
            const uint32_t skey = __shfl_sync(kFull, key, s);
            const uint32_t sb = __shfl_sync(kFull, bucket, s);
            const uint32_t sop = kKind == kKindMixed ? __shfl_sync(kFull, op, s) : op;
            uint32_t* p = slab_ptr(T, sb, cur);
            const uint32_t data = ld_slab<kReadOnly>(p + lane);
            if (++iters > T.iter_limit) {
                if ((int)lane == s) {
                    set_flag(T, kFlagIterLimit);
                    active = false;
                }
            } else {
                const Outcome o = examine<kKeyOnly>(data, sop, skey);
                if (o.kind == kResolved) {
                    if ((int)lane == s) { res = o.a; fnd = o.b; active = false; }
                } else if (o.kind == kAdvance) {
                    if (valid_next(T, o.a)) {
                        cur = o.a;
                    } else if ((int)lane == s) {
                        set_flag(T, kFlagBadPointer);
                        active = false;
                    }
                } else if (o.kind == kMarkDead) {
                    if ((int)lane == s) {
                        st_relaxed(p + o.a, kTombstone);
                        res = 1u; fnd = 1u; active = false;
                    }
                } else if (o.kind == kClaim) {
                    const uint32_t sval = kKeyOnly ? 0u : __shfl_sync(kFull, value, s);
                    if ((int)lane == s) {
                        bool ok;
                        if constexpr (kKeyOnly) {
                            ok = atomicCAS(p + o.a, kEmptyKey, skey) == kEmptyKey;
                        } else {
                            const unsigned long long e = pack_pair(o.b, o.c);
                            ok = atomicCAS(reinterpret_cast<unsigned long long*>(p + o.a), e,
                                           pack_pair(skey, sval)) == e;
                        }
                        if (ok) {  // otherwise re-read the same slab
                            fnd = o.b != kEmptyKey;
                            res = fnd ? 0u : 1u;
                            active = false;
                        }
                    }
                } else {  // kNeedSlab
                    const uint32_t nx = grow_list(T, ac, warp_gid, p, s);
                    if (nx == kAllocFailed) {
                        if ((int)lane == s) {
                            set_flag(T, kFlagOutOfSlabs);
                            active = false;
                        }
                    } else if (valid_next(T, nx)) {
                        cur = nx;
                    } else if ((int)lane == s) {
                        set_flag(T, kFlagBadPointer);
                        active = false;
                    }
                }
            }
            queue = __ballot_sync(kFull, active);
        }
        if (has) {
            if (A.results) A.results[idx] = res;
            if (A.found) A.found[idx] = (uint8_t)fnd;
        }
    }
}

// ---------------------------------------------------------------------------
// GB300 kernel: persistent per-warp op window with shared-memory slab staging.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async_16(uint32_t smem_addr, const void* gptr) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr), "l"(gptr) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

constexpr uint32_t kNoOp = 0xFFFFFFFFu;
constexpr uint32_t kStageWordsPerWarp = 32u * kWordsPerSlab;  // 32 slabs = 4 KB

template <int kKind, bool kKeyOnly>
__global__ void staged_kernel(TableView T, BatchArgs A, uint32_t ops_per_warp) {
    extern __shared__ __align__(16) uint32_t smem[];
    const uint32_t lane = lane_id();
    const uint32_t warp_gid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint32_t* stage = smem + (threadIdx.x >> 5) * kStageWordsPerWarp;
    const uint32_t stage_base = (uint32_t)__cvta_generic_to_shared(stage);

    // This warp's contiguous share of the batch.
    const uint64_t begin64 = (uint64_t)warp_gid * ops_per_warp;
    const uint32_t begin = (uint32_t)min(begin64, (uint64_t)A.n);
    const uint32_t end = (uint32_t)min(begin64 + ops_per_warp, (uint64_t)A.n);
    uint32_t next = begin;

    AllocCtx ac{kNoBlock, 0u, 0u};
    // Per-lane op state.
    uint32_t my = kNoOp, key = 0, value = 0, op = 0, bucket = 0, cur = kEmptyKey, rounds = 0;
    uint32_t res = 0, fnd = 0;
    bool done = false, cas_wait = false, cas_new = false;
    unsigned long long cas_exp = 0, cas_got = 0;
    uint32_t* myp = nullptr;
    const uint32_t lt_mask = (1u << lane) - 1u;

    for (;;) {
        // Refill: lanes without an op take the next ops of the range, in lane order.
        const uint32_t need = __ballot_sync(kFull, my == kNoOp);
        if (need && next < end) {
            const uint32_t i = next + __popc(need & lt_mask);
            if (my == kNoOp && i < end) {
                my = i;
                op = fixed_op<kKind>();
                if constexpr (kKind == kKindMixed) op = ld_stream_u8(A.ops + i);
                key = ld_stream(A.keys + i);
                if ((kKind == kKindInsert || kKind == kKindMixed) && !kKeyOnly && A.values)
                    value = ld_stream(A.values + i);
                res = default_result(op);
                fnd = 0;
                cur = kEmptyKey;
                rounds = 0;
                if (op > kOpSearch) {
                    res = 0;
                    done = true;
                } else if (key >= kTombstone) {
                    set_flag(T, kFlagReserved);
                    done = true;
                } else {
                    bucket = bucket_of(T, key);
                }
            }
            next = min(next + (uint32_t)__popc(need), end);
        }
        const uint32_t pend = __ballot_sync(kFull, my != kNoOp && !done);

        if (pend) {
            // Stage every pending op's current slab: 8 lanes x 16 bytes per slab,
            // 4 slabs per warp instruction.
            const uint32_t u = cur == kEmptyKey ? bucket : T.num_buckets + cur;
            myp = T.slabs + (uint64_t)u * kWordsPerSlab;
            __syncwarp();
#pragma unroll
            for (uint32_t j = 0; j < 8; ++j) {
                const uint32_t s = 4u * j + (lane >> 3);
                const uint32_t us = __shfl_sync(kFull, u, s);
                if ((pend >> s) & 1u) {
                    const uint32_t c = lane & 7u;
                    cp_async_16(stage_base + (s * kWordsPerSlab + c * 4u) * 4u,
                                T.slabs + (uint64_t)us * kWordsPerSlab + c * 4u);
                }
            }
            cp_async_wait_all();
            __syncwarp();

            // Serve the window's ops one at a time (WCWS).
            uint32_t q = pend;
            while (q) {
                const int s = __ffs(q) - 1;
                q &= q - 1u;
                const uint32_t data = stage[s * kWordsPerSlab + lane];
                const uint32_t skey = __shfl_sync(kFull, key, s);
                const uint32_t sop = kKind == kKindMixed ? __shfl_sync(kFull, op, s) : fixed_op<kKind>();
                const Outcome o = examine<kKeyOnly>(data, sop, skey);
                const bool me = (int)lane == s;
                if (o.kind == kResolved) {
                    if (me) { res = o.a; fnd = o.b; done = true; }
                } else if (o.kind == kAdvance) {
                    if (me) {
                        if (valid_next(T, o.a)) {
                            cur = o.a;
                        } else {
                            set_flag(T, kFlagBadPointer);
                            done = true;
                        }
                    }
                } else if (o.kind == kMarkDead) {
                    if (me) {
                        st_relaxed(myp + o.a, kTombstone);
                        res = 1u; fnd = 1u; done = true;
                    }
                } else if (o.kind == kClaim) {
                    if (me) {  // issue now, check after the round
                        if constexpr (kKeyOnly) {
                            cas_exp = kEmptyKey;
                            cas_got = atomicCAS(myp + o.a, kEmptyKey, key);
                        } else {
                            cas_exp = pack_pair(o.b, o.c);
                            cas_got = atomicCAS(reinterpret_cast<unsigned long long*>(myp + o.a),
                                                cas_exp, pack_pair(key, value));
                        }
                        cas_wait = true;
                        cas_new = o.b == kEmptyKey;
                    }
                } else {  // kNeedSlab
                    uint32_t* ps = reinterpret_cast<uint32_t*>(__shfl_sync(kFull, (unsigned long long)myp, s));
                    const uint32_t nx = grow_list(T, ac, warp_gid, ps, s);
                    if (me) {
                        if (nx == kAllocFailed) {
                            set_flag(T, kFlagOutOfSlabs);
                            done = true;
                        } else if (valid_next(T, nx)) {
                            cur = nx;
                        } else {
                            set_flag(T, kFlagBadPointer);
                            done = true;
                        }
                    }
                }
            }
            if (cas_wait) {
                cas_wait = false;
                if (cas_got == cas_exp) {
                    fnd = cas_new ? 0u : 1u;
                    res = cas_new ? 1u : 0u;
                    done = true;
                }  // else: retry this slab next round
            }
            if (my != kNoOp && !done && ++rounds >= T.iter_limit) {
                set_flag(T, kFlagIterLimit);
                done = true;
            }
        }
        if (done) {
            if (A.results) A.results[my] = res;
            if (A.found) A.found[my] = (uint8_t)fnd;
            my = kNoOp;
            done = false;
        }
        if (!pend && next >= end) break;  // nothing pending and the range is used up
    }
}

}  // namespace slab
