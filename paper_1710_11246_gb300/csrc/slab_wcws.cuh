// Warp-cooperative work sharing (WCWS, Sec. 4.1) over slab lists, in the form of
// Fig. "alg:search": one op per lane, the warp serves its queue one op at a time,
// each step reads the source lane's current slab from global memory. This is the
// paper-structured kernel family (direct_kernel); slab_staged.cuh holds the
// pipelined GB300 family built from the same step.
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
__device__ __forceinline__ Outcome examine(uint32_t data, uint32_t sop, uint32_t skey, bool multiset) {
    constexpr uint32_t kMask = kKeyOnly ? kKeyLanesKeyOnly : kKeyLanesKV;
    Outcome o;
    if (sop == kOpInsert) {
        // REPLACE looks for the key or the first empty pair; a multiset INSERT
        // for the first empty pair only (Sec. 3.2)
        uint32_t m = __ballot_sync(kFull, data == kEmptyKey || (!multiset && data == skey)) & kMask;
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
template <uint32_t kW = kWordsPerSlab>
__device__ __forceinline__ uint32_t grow_list(const TableView& T, AllocCtx& ac, uint32_t warp_gid,
                                              uint32_t* p_src_lane, int s) {
    uint32_t na = warp_allocate(T, ac, warp_gid);
    if (na == kAllocFailed) {  // no slab left: follow a slab another op linked meanwhile, if any
        uint32_t nx = kAllocFailed;
        if ((int)lane_id() == s) nx = ld_coherent(p_src_lane + next_word<kW>());
        return __shfl_sync(kFull, nx, s);  // kEmptyKey (= kAllocFailed) while still unlinked
    }
    uint32_t old = 0;
    if ((int)lane_id() == s) old = atomicCAS(p_src_lane + next_word<kW>(), kEmptyKey, na);
    old = __shfl_sync(kFull, old, s);
    if (old == kEmptyKey) return na;
    if ((int)lane_id() == s) deallocate(T, na);
    return old;
}

// Warp-wide, batched: every lane with `need` set links one new slab behind its
// own full slab at `p` (the slab its op last read). The slabs for all such lanes
// come from one batched allocation; each lane then issues its own 32-bit link
// CAS on its slab's next pointer, and a lane that loses (another op linked first)
// returns its slab and follows the winner's. Returns the slab to continue with;
// kAllocRetry where the warp's batch got no slab this time (the op stays on its
// slab and tries again in a later round); kAllocFailed where the pool had no
// slab left. Either way a slab that another op linked meanwhile is followed.
template <uint32_t kW = kWordsPerSlab>
__device__ __forceinline__ uint32_t grow_lists(const TableView& T, AllocCtx& ac, uint32_t warp_gid, uint32_t* p,
                                               bool need) {
    const uint32_t na = warp_allocate_many(T, ac, warp_gid, need, true);
    if (!need) return kAllocFailed;
    if (na >= kAllocRetry) {  // kAllocRetry or kAllocFailed
        const uint32_t nx = ld_coherent(p + next_word<kW>());
        return nx != kEmptyKey ? nx : na;
    }
    const uint32_t old = atomicCAS(p + next_word<kW>(), kEmptyKey, na);
    if (old == kEmptyKey) return na;
    deallocate(T, na);
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
                const Outcome o = examine<kKeyOnly>(data, sop, skey, T.multiset != 0);
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
                        remove_at<kKeyOnly>(T, p, o.a);
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

}  // namespace slab
