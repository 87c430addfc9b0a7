// The GB300 kernel family for slab-hash batches: warp-cooperative work sharing
// (Sec. 4.1) with the slab reads moved off the critical path.
//
// Each warp walks tiles of 32 ops (one per lane) in a persistent grid. Per tile:
//   the tile's 32 base slabs are copied into the warp's shared-memory stage
//   (cp.async, 16 bytes per lane, 4 slabs per warp instruction: the coalesced,
//   warp-cooperative ReadSlab of Sec. 4.3 for 32 ops at once); while they are in
//   flight the warp hashes the next tile's keys (pulling its base slabs into L2
//   for tables much larger than L2) and starts loading the tile after; then the
//   tile is served from the stage.
// Serving a tile: each pending op's own lane scans its staged slab (8 128-bit
// chunk reads) for the lowest key word that holds its key (an insert: its key or
// an empty pair), the position the WCWS ballot of Fig. "alg:search" would give
// the op's source lane. Built with -DSLAB_LANE_MATCH=0 the kernels run that WCWS
// loop itself instead: the warp takes the queued ops in lane order, reads each
// op's staged slab one word per lane, and parks each ballot word in shared
// memory for the source lane. Either way the source lanes then act together: read
// the value (search), write the tombstone (delete) or issue the 64-bit CAS of the
// pair (replace), so the 32 CASes of a tile are in flight together and their
// results are checked once. A claim that lost its race tries the following pair
// of the same slab at once; ops that must follow a next pointer, or that ran off
// their slab, restage just their slabs and go round again; a full list grows
// through SlabAlloc (Sec. 5), by one batched allocation for all of a bulk-insert
// tile's full lists.
//
// Staging just before serving (rather than a tile ahead into a second buffer)
// keeps one 4 KB stage per warp, which leaves room for more resident warps, and
// gives claims a fresh snapshot (an older one makes them lose more races).
//
// Search and delete batches do not restage inside a tile: an op that must go on
// to its list's next slab waits in a per-warp ring and is served later in a
// tile of such ops, 32 at a time, so one long list does not hold the whole warp
// for another stage-and-match round. Mixed batches sort each input tile's ops by
// kind: inserts wait in a per-warp insert queue and are served as insert tiles,
// searches and deletes go to the ring. Insert tiles are served to the end: their
// rounds also claim pairs and grow lists, and measured slower when deferred. On
// tables much larger than L2 (the ones whose slabs are pulled into L2 a tile
// ahead) search and delete restage in the tile and mixed tiles hold all three
// kinds side by side, which measured faster there.
#pragma once
#include "slab_device.cuh"
#include "slab_wcws.cuh"

namespace slab {

template <uint32_t kW>
constexpr uint32_t kTileWords = 32u * kW;  // one slab per lane: 4 KB (128-byte slabs) or 2 KB (64-byte)
constexpr uint32_t kNoOpCode = 0xFFu;
// per warp: the stage, then 32 ballot words, the tile's 32 keys and, for mixed
// batches, 32 alternate keys (below)
template <uint32_t kW>
constexpr uint32_t kServeWordsPerWarp = kTileWords<kW> + 32u + 32u + 32u;
// Search and delete kernels add the ring of deferred ops behind that: op index,
// slab to stage next, key and rounds so far, kDeferSlots of each. Mixed kernels
// keep each ring entry's op code too, and a queue of inserts (op index, key,
// value, bucket); theirs is the largest per-warp layout, kMixedWordsPerWarp.
constexpr uint32_t kDeferSlots = 64u;
template <uint32_t kW>
constexpr uint32_t kStagedWordsPerWarp = kServeWordsPerWarp<kW> + 4u * kDeferSlots;
template <uint32_t kW>
constexpr uint32_t kMixedWordsPerWarp = kServeWordsPerWarp<kW> + 9u * kDeferSlots;

// The second value a mixed op's WCWS step matches besides its key: an empty
// slot for an insert (it may claim one), its key again for a search or delete.
__device__ __forceinline__ uint32_t alt_key(uint32_t key, uint32_t op) {
    return op == kOpInsert ? kEmptyKey : key;
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ void cp_async_16(uint32_t smem_addr, const void* gptr) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr), "l"(gptr) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Stage position of word w of the slab in slot s. The 16-byte chunks of a slot
// are rotated by XOR with a function of s: a warp reading all words of one
// 128-byte slot, or of two adjacent 64-byte slots, hits 32 distinct banks, and
// 32 lanes each reading one word of their own slot hit at most 4 lanes per bank.
// 128-byte slots XOR their 8 chunks with s mod 8; 64-byte slots, two to a bank
// row, XOR their 4 chunks with (s / 2) mod 4.
template <uint32_t kW>
__device__ __forceinline__ uint32_t swz(uint32_t s, uint32_t w) {
    if constexpr (kW == 32u) return s * 32u + ((((w >> 2) ^ (s & 7u)) << 2) | (w & 3u));
    else return s * 16u + ((((w >> 2) ^ ((s >> 1) & 3u)) << 2) | (w & 3u));
}

// Copy, for every lane s in `mask`, the slab with unified index shfl(u, s)
// (base slab b -> b, pool unit a -> B + a) into slot s of the stage at byte
// address `stage`, as 16-byte pieces. 128-byte slabs: lanes 8g..8g+7 move one
// slab, slots g, g + 4, ..., g + 28 in turn; slot 4j + g has (4j + g) mod 8 =
// 4 (j mod 2) + g, so a lane's swizzled destinations take two forms, 512 bytes
// apart per j. 64-byte slabs: lanes 4g..4g+3 move one slab, slots g, g + 8, ...,
// g + 24; slot 8j + g has ((8j + g) / 2) mod 4 = (g / 2) mod 4, one form per lane.
template <uint32_t kW>
__device__ __forceinline__ void stage_slabs(const TableView& T, uint32_t stage, uint32_t u, uint32_t mask,
                                            uint32_t lane) {
    if constexpr (kW == 32u) {
        const uint32_t g = lane >> 3, c = lane & 7u;
        const uint32_t* src = T.slabs + c * 4u;  // this lane's 16-byte piece of slab 0
        const uint32_t dst_even = stage + g * 128u + ((c ^ g) << 4);
        const uint32_t dst_odd = stage + g * 128u + ((c ^ (g | 4u)) << 4);
        const uint32_t mg = mask >> g;
#pragma unroll
        for (uint32_t j = 0; j < 8; ++j) {
            const uint32_t us = __shfl_sync(kFull, u, 4u * j + g);
            if ((mg >> (4u * j)) & 1u)
                cp_async_16(((j & 1u) ? dst_odd : dst_even) + j * 512u, src + (uint64_t)us * 32u);
        }
    } else {
        const uint32_t g = lane >> 2, c = lane & 3u;
        const uint32_t* src = T.slabs + c * 4u;
        const uint32_t dst = stage + g * 64u + ((c ^ ((g >> 1) & 3u)) << 4);
        const uint32_t mg = mask >> g;
#pragma unroll
        for (uint32_t j = 0; j < 4; ++j) {
            const uint32_t us = __shfl_sync(kFull, u, 8u * j + g);
            if ((mg >> (8u * j)) & 1u) cp_async_16(dst + j * 512u, src + (uint64_t)us * 16u);
        }
    }
}

// Where lane reads word `lane` (128-byte slabs) of slot s, or word lane mod 16
// of slot 2i + lane / 16 in step i (64-byte slabs), relative to the slot (pair):
// off[s mod 8] or off[i mod 4] (see swz).
template <uint32_t kW>
__device__ __forceinline__ void stage_offsets(uint32_t lane, uint32_t (&off)[8]) {
#pragma unroll
    for (uint32_t j = 0; j < 8; ++j) {
        if constexpr (kW == 32u) off[j] = (((lane >> 2) ^ j) << 2) | (lane & 3u);
        else off[j] = ((lane >> 4) << 4) | ((((lane >> 2) & 3u) ^ (j & 3u)) << 2) | (lane & 3u);
    }
}

// The WCWS match of one round (Fig. "alg:search"): the warp takes the queued ops
// (bits of `pend`) in lane order; for each op s it compares word `lane` of the
// op's staged slab (slot s) with the op's key from the shared copy of the tile's
// keys (an insert also with EMPTY, a mixed op also with its alternate key) and
// lane 0 stores the ballot. With 64-byte slabs a slab is half a warp wide (the
// slab width the paper ties to the warp's, Sec. 4.2, halved), so one step serves
// two ops: lanes 0-15 match op 2i and lanes 16-31 op 2i + 1, and the step's
// ballot (ballots[i]) holds both, op 2i in its low half. 128-byte slabs store op
// s's ballot in ballots[s]. Three forms of the same loop: all 32 ops queued
// (`full`: keys read and ballots stored four at a time, no branches), `wide`
// (unrolled over the steps, one predicate per step) and a loop over the set bits
// (few ops).
template <int kKind, uint32_t kW>
__device__ __forceinline__ void wcws_ballots(const uint32_t* buf, uint32_t* ballots, const uint32_t* skeys,
                                             const uint32_t* salts, const uint32_t (&off)[8], uint32_t pend,
                                             bool full, bool wide) {
    const uint32_t lane = lane_id();
    auto match = [&](uint32_t data, uint32_t skey, uint32_t salt) {
        bool pred;
        if constexpr (kKind == kKindInsert) {
            pred = data == skey || data == kEmptyKey;
        } else if constexpr (kKind == kKindMixed) {
            pred = data == skey || data == salt;
        } else {
            pred = data == skey;
        }
        return __ballot_sync(kFull, pred);
    };
    if constexpr (kW == 32u) {
        auto step = [&](uint32_t s, uint32_t data) {
            const uint32_t mm = match(data, skeys[s], kKind == kKindMixed ? salts[s] : 0u);
            if (lane == 0) ballots[s] = mm;
        };
        if (full) {
#pragma unroll
            for (uint32_t g = 0; g < 8; ++g) {
                const uint4 k4 = *reinterpret_cast<const uint4*>(skeys + 4u * g);
                const uint4 a4 = kKind == kKindMixed ? *reinterpret_cast<const uint4*>(salts + 4u * g) : k4;
                const uint32_t s0 = 4u * g;
                uint4 b4;
                b4.x = match(buf[(s0 + 0u) * 32u + off[(s0 + 0u) & 7u]], k4.x, a4.x);
                b4.y = match(buf[(s0 + 1u) * 32u + off[(s0 + 1u) & 7u]], k4.y, a4.y);
                b4.z = match(buf[(s0 + 2u) * 32u + off[(s0 + 2u) & 7u]], k4.z, a4.z);
                b4.w = match(buf[(s0 + 3u) * 32u + off[(s0 + 3u) & 7u]], k4.w, a4.w);
                if (lane == 0) *reinterpret_cast<uint4*>(ballots + s0) = b4;
            }
        } else if (wide) {
#pragma unroll
            for (uint32_t s = 0; s < 32; ++s)
                if ((pend >> s) & 1u) step(s, buf[s * 32u + off[s & 7u]]);
        } else {
            for (uint32_t q = pend; q; q &= q - 1u) {
                const uint32_t s = (uint32_t)(__ffs(q) - 1);
                step(s, buf[swz<32u>(s, lane)]);
            }
        }
    } else {
        const uint32_t h = lane >> 4;  // which op of the step's pair this lane serves
        auto step = [&](uint32_t i, uint32_t data) {
            const uint32_t mm = match(data, skeys[2u * i + h], kKind == kKindMixed ? salts[2u * i + h] : 0u);
            if (lane == 0) ballots[i] = mm;
        };
        if (full) {
#pragma unroll
            for (uint32_t g = 0; g < 4; ++g) {  // steps 4g..4g+3: ops 8g..8g+7
                const uint4 ka = *reinterpret_cast<const uint4*>(skeys + 8u * g);
                const uint4 kb = *reinterpret_cast<const uint4*>(skeys + 8u * g + 4u);
                const uint4 aa = kKind == kKindMixed ? *reinterpret_cast<const uint4*>(salts + 8u * g) : ka;
                const uint4 ab = kKind == kKindMixed ? *reinterpret_cast<const uint4*>(salts + 8u * g + 4u) : kb;
                const uint32_t i0 = 4u * g;
                uint4 b4;
                b4.x = match(buf[(i0 + 0u) * 32u + off[(i0 + 0u) & 3u]], h ? ka.y : ka.x, h ? aa.y : aa.x);
                b4.y = match(buf[(i0 + 1u) * 32u + off[(i0 + 1u) & 3u]], h ? ka.w : ka.z, h ? aa.w : aa.z);
                b4.z = match(buf[(i0 + 2u) * 32u + off[(i0 + 2u) & 3u]], h ? kb.y : kb.x, h ? ab.y : ab.x);
                b4.w = match(buf[(i0 + 3u) * 32u + off[(i0 + 3u) & 3u]], h ? kb.w : kb.z, h ? ab.w : ab.z);
                if (lane == 0) *reinterpret_cast<uint4*>(ballots + i0) = b4;
            }
        } else if (wide) {
#pragma unroll
            for (uint32_t i = 0; i < 16; ++i)
                if ((pend >> (2u * i)) & 3u) step(i, buf[i * 32u + off[i & 3u]]);
        } else {
            for (uint32_t q = pend; q;) {
                const uint32_t i = (uint32_t)(__ffs(q) - 1) >> 1;
                q &= ~(3u << (2u * i));
                step(i, buf[i * 32u + off[i & 3u]]);
            }
        }
    }
}

// The source lane's share of the ballots: op `lane`'s ballot over the words of
// its slab, restricted to the key words (Sec. 4.2).
template <bool kKeyOnly, uint32_t kW>
__device__ __forceinline__ uint32_t own_ballot(const uint32_t* ballots, uint32_t lane) {
    if constexpr (kW == 32u) return ballots[lane] & key_words<kKeyOnly, 32u>();
    else return (ballots[lane >> 1] >> ((lane & 1u) * 16u)) & key_words<kKeyOnly, 16u>();
}

// The staged kernels match with the source lane scanning its own op's staged slab
// (SLAB_LANE_MATCH = 1) or with the WCWS ballots above (0). The stage already came
// in as coalesced, warp-cooperative copies of whole slabs, so the per-op compares
// need no warp-wide step: a lane reads its slot as 16-byte chunks (8 lanes of a
// quarter-warp hit 8 distinct chunk positions under the stage's swizzle).
#ifndef SLAB_LANE_MATCH
#define SLAB_LANE_MATCH 1
#endif

#ifndef SLAB_LANE_VALUE
#define SLAB_LANE_VALUE 1
#endif

// One 16-byte chunk of the stage as a single 128-bit shared load. Written out so
// the load stays whole when only some of its words are used: split into 32-bit
// loads, lanes s, s + 8, s + 16 and s + 24 (one chunk position under the swizzle)
// would share banks, four ways; a volatile load is not narrowed to the words
// used. The volatile asm also keeps it after the stage's cp.async wait.
__device__ __forceinline__ uint4 ld_stage_chunk(const uint32_t* p) {
    uint4 r;
    asm volatile("ld.volatile.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "r"((uint32_t)__cvta_generic_to_shared(p)));
    return r;
}

// The lowest key word of slot `lane` that holds `key` or (kAlt) `alt`, as the one
// bit of the mask own_ballot would give it (0: no match). kVal (key-value slabs):
// *val gets the word after that key, its value, from the same 16-byte chunk.
// kWord: *word gets the matched key word itself (the key, or what matched `alt`).
template <bool kKeyOnly, uint32_t kW, bool kAlt, bool kVal = false, bool kWord = false>
__device__ __forceinline__ uint32_t lane_match(const uint32_t* buf, uint32_t lane, uint32_t key, uint32_t alt,
                                               uint32_t* val = nullptr, uint32_t* word = nullptr) {
    static_assert(!(kVal && kKeyOnly), "key-only slabs hold no values");
    constexpr uint32_t kKeys = key_words<kKeyOnly, kW>();
    uint32_t d = 32u, v = 0u, kw = 0u;
#pragma unroll
    for (int c = (int)(kW / 4u) - 1; c >= 0; --c) {  // from the last chunk, so the lowest match stays
        if ((kKeys >> (4 * c)) & 0xFu) {
            const uint4 q = ld_stage_chunk(buf + swz<kW>(lane, 4u * (uint32_t)c));
            const uint32_t w[4] = {q.w, q.z, q.y, q.x};
#pragma unroll
            for (int j = 0; j < 4; ++j) {  // words 4c + 3 down to 4c
                const uint32_t wi = 4u * (uint32_t)c + 3u - (uint32_t)j;
                if ((kKeys >> wi) & 1u) {
                    const bool hit = w[j] == key || (kAlt && w[j] == alt);
                    d = hit ? wi : d;
                    if constexpr (kVal) v = hit ? w[j > 0 ? j - 1 : 0] : v;  // key words are even: j is 1 or 3
                    if constexpr (kWord) kw = hit ? w[j] : kw;
                }
            }
        }
    }
    if constexpr (kVal) *val = v;
    if constexpr (kWord) *word = kw;
    return d < 32u ? 1u << d : 0u;
}

// One WCWS round (Fig. "alg:search") of a search or delete batch for the ops of
// the lanes in `pend`, each of whose current slab (unified index u) is staged in
// slot `lane` of `buf`, with keys in `skeys`: the ballots of wcws_ballots, then
// every source lane acts on its ballot (reads the value, or writes the tombstone). On return
// an op that is done has its result in res / fnd and pending cleared; one that
// goes on has u set to its list's next slab.
// (kKind = kKindMixed: each lane's op is a search or a delete, given by `op`.)
template <int kKind, bool kKeyOnly, uint32_t kW>
__device__ __forceinline__ void read_round(const TableView& T, const uint32_t* buf, uint32_t* ballots,
                                           const uint32_t* skeys, const uint32_t (&off)[8], uint32_t pend,
                                           bool& pending, uint32_t& u, uint32_t& res, uint32_t& fnd,
                                           uint32_t key, uint32_t op = kOpSearch) {
    static_assert(kKind != kKindInsert, "claims serve whole tiles (serve_tile)");
    const uint32_t lane = lane_id();
    uint32_t m, val = 0u;
    // search values come with the match (the value sits in its key's chunk)
    constexpr bool kVal = SLAB_LANE_MATCH && SLAB_LANE_VALUE && !kKeyOnly && kKind != kKindDelete;
    if constexpr (kVal) {
        m = pending ? lane_match<kKeyOnly, kW, false, true>(buf, lane, key, key, &val) : 0u;
    } else if constexpr (SLAB_LANE_MATCH) {
        m = pending ? lane_match<kKeyOnly, kW, false>(buf, lane, key, key) : 0u;
    } else {
        // a search or delete step compares the op's key only
        wcws_ballots<kKindSearch, kW>(buf, ballots, skeys, skeys, off, pend, pend == kFull, __popc(pend) > 8);
        __syncwarp();
        // the source lanes act on their ballots (Sec. 4.3)
        m = pending ? own_ballot<kKeyOnly, kW>(ballots, lane) : 0u;
    }
    if (pending) {
        if (m) {
            const uint32_t d = (uint32_t)(__ffs(m) - 1);
            if (kKind == kKindSearch || (kKind == kKindMixed && op == kOpSearch)) {
                if constexpr (kVal) res = val;
                else res = kKeyOnly ? 0u : buf[swz<kW>(lane, d + 1u)];
            } else {
                remove_at<kKeyOnly>(T, T.slabs + (uint64_t)u * kW, d);
                res = 1u;
            }
            fnd = 1u;
            pending = false;
        } else {
            const uint32_t nx = buf[swz<kW>(lane, next_word<kW>())];
            if (nx == kEmptyKey) {
                pending = false;  // end of the list: not found
            } else if (valid_next(T, nx)) {
                u = T.num_buckets + nx;
            } else {
                set_flag(T, kFlagBadPointer);
                pending = false;
            }
        }
    }
}

// Serve one tile of up to 32 ops, one per lane (op index idx, valid where `has`),
// whose base slabs are staged in slots 0..31 of `buf` (shared byte address
// buf_s), keys in `skeys` and (mixed) alternate keys in `salts`: the WCWS rounds of Fig.
// "alg:search", each op's source-lane action, restaging for ops that move on,
// list growth, and the result writes.
template <int kKind, bool kKeyOnly, uint32_t kW>
__device__ __forceinline__ void serve_tile(const TableView& T, const BatchArgs& A, AllocCtx& ac, uint32_t warp_gid,
                                           const uint32_t* buf, uint32_t buf_s, uint32_t* ballots,
                                           const uint32_t* skeys, const uint32_t* salts, const uint32_t (&off)[8],
                                           uint32_t ck, uint32_t cv, uint32_t co, uint32_t cb, uint32_t idx,
                                           bool has) {
    const uint32_t lane = lane_id();
    bool pending = co <= kOpSearch && ck < kTombstone;
    if (co <= kOpSearch && ck >= kTombstone) set_flag(T, kFlagReserved);

    uint32_t res = default_result(co), fnd = 0, cur = kEmptyKey, rounds = 0;
    bool first = true;
    for (;;) {
        const uint32_t pend = __ballot_sync(kFull, pending);
        if (!pend) break;
        const uint32_t u = cur == kEmptyKey ? cb : T.num_buckets + cur;
        if (!first) {  // restage only the ops that moved on or must retry
            stage_slabs<kW>(T, buf_s, u, pend, lane);
            cp_async_commit();
            cp_async_wait<0>();
            __syncwarp();
        }
        uint32_t m, mw = 0u, mv = 0u;
        if constexpr (SLAB_LANE_MATCH) {
            // each pending op's lane scans its slab for its key (and an insert for
            // EMPTY, a mixed op for its alternate key), keeping the matched pair
            const uint32_t sk = match_key(T, ck, co);
            constexpr bool kClaim = kKind == kKindInsert || kKind == kKindMixed;
            m = pending ? lane_match<kKeyOnly, kW, kClaim, !kKeyOnly, kClaim>(
                              buf, lane, sk, kKind == kKindMixed ? alt_key(ck, co) : kEmptyKey, &mv, &mw)
                        : 0u;
        } else {
            // WCWS: one queued op at a time, lane order (the work-queue loop of Fig. "alg:search").
            wcws_ballots<kKind, kW>(buf, ballots, skeys, salts, off, pend, first && pend == kFull, first);
            __syncwarp();
            // the source lanes act on their ballots (Sec. 4.3)
            m = pending ? own_ballot<kKeyOnly, kW>(ballots, lane) : 0u;
        }
        uint32_t* gslab = T.slabs + (uint64_t)u * kW;
        const uint32_t myop = kKind == kKindMixed ? co : fixed_op<kKind>();
        bool cas_wait = false, cas_new = false, need_slab = false;
        unsigned long long cas_exp = 0, cas_got = 0;
        uint32_t d = 0;
        if (pending) {
            if (m) {
                d = (uint32_t)(__ffs(m) - 1);
                if (myop == kOpSearch) {
                    if constexpr (SLAB_LANE_MATCH) res = kKeyOnly ? 0u : mv;
                    else res = kKeyOnly ? 0u : buf[swz<kW>(lane, d + 1u)];
                    fnd = 1u;
                    pending = false;
                } else if (myop == kOpDelete) {
                    remove_at<kKeyOnly>(T, gslab, d);
                    res = 1u;
                    fnd = 1u;
                    pending = false;
                } else if constexpr (kKeyOnly) {
                    if (!T.multiset && (SLAB_LANE_MATCH ? mw : buf[swz<kW>(lane, d)]) == ck) {  // already present
                        res = 0u;
                        fnd = 1u;
                        pending = false;
                    } else {
                        cas_exp = kEmptyKey;
                        cas_got = atomicCAS(gslab + d, kEmptyKey, ck);
                        cas_wait = true;
                        cas_new = true;
                    }
                } else {
                    uint2 pr;
                    if constexpr (SLAB_LANE_MATCH) pr = make_uint2(mw, mv);  // the matched pair, from the scan
                    else pr = *reinterpret_cast<const uint2*>(buf + swz<kW>(lane, d));
                    cas_exp = pack_pair(pr.x, pr.y);
                    cas_got = atomicCAS(reinterpret_cast<unsigned long long*>(gslab + d), cas_exp,
                                        pack_pair(ck, cv));
                    cas_wait = true;
                    cas_new = pr.x == kEmptyKey;
                }
            } else {
                const uint32_t nx = buf[swz<kW>(lane, next_word<kW>())];
                if (nx == kEmptyKey) {
                    if (myop == kOpInsert) need_slab = true;
                    else pending = false;  // end of the list: not found
                } else if (valid_next(T, nx)) {
                    cur = nx;
                } else {
                    set_flag(T, kFlagBadPointer);
                    pending = false;
                }
            }
        }
        // A claim of an empty pair that lost its race learns from the CAS which key
        // took the pair. If that key is another one, the pair after it is the next
        // empty candidate: slots fill in (slab, lane) order and are never emptied
        // on this path, so every earlier pair of the slab holds a different key and
        // a successful CAS there keeps keys unique. Claims that meet their own key
        // (a replace race) or run off the slab restage and go round again.
        constexpr uint32_t kPairStride = kKeyOnly ? 1u : 2u;
        constexpr uint32_t kLastKeyLane = last_key_word<kKeyOnly, kW>();
        if constexpr (kKind == kKindInsert || kKind == kKindMixed) {
            while (cas_wait) {
                if (cas_got == cas_exp) {
                    fnd = cas_new ? 0u : 1u;
                    res = cas_new ? 1u : 0u;
                    pending = false;
                    break;
                }
                if (!cas_new || ((uint32_t)cas_got == ck && !T.multiset) || d + kPairStride > kLastKeyLane) break;
                d += kPairStride;
                if constexpr (kKeyOnly) {
                    cas_got = atomicCAS(gslab + d, kEmptyKey, ck);
                } else {
                    cas_exp = pack_pair(kEmptyKey, kEmptyKey);
                    cas_got = atomicCAS(reinterpret_cast<unsigned long long*>(gslab + d), cas_exp,
                                        pack_pair(ck, cv));
                }
            }
        }
        // full lists grow by one slab each (SlabAlloc, Sec. 5)
        auto settle = [&](uint32_t nx) {
            if (nx == kAllocRetry) return;  // still pending on the same slab: grow it in a later round
            if (nx == kAllocFailed) {
                set_flag(T, kFlagOutOfSlabs);
                pending = false;
            } else if (valid_next(T, nx)) {
                cur = nx;
            } else {
                set_flag(T, kFlagBadPointer);
                pending = false;
            }
        };
        if constexpr (kKind == kKindInsert) {
            // bulk builds grow many lists at once: lanes whose lists end in the same
            // slab elect one leader, the leaders get their slabs in one batched
            // SlabAlloc round and link them with their own CAS, and the other lanes
            // follow their leader (a warp holds at most one unlinked slab per list)
            if (__any_sync(kFull, need_slab)) {
                const uint32_t peers = __match_any_sync(kFull, need_slab ? (unsigned long long)gslab : 0ull);
                const int leader = __ffs(peers) - 1;
                const uint32_t lead_nx = grow_lists<kW>(T, ac, warp_gid, gslab, need_slab && (int)lane == leader);
                const uint32_t nx = __shfl_sync(kFull, lead_nx, leader);
                if (need_slab) settle(nx);
            }
        } else if constexpr (kKind == kKindMixed) {
            // mixed batches grow a list now and then: one lane at a time
            for (uint32_t q = __ballot_sync(kFull, need_slab); q; q &= q - 1u) {
                const int s = __ffs(q) - 1;
                uint32_t* ps = reinterpret_cast<uint32_t*>(__shfl_sync(kFull, (unsigned long long)gslab, s));
                const uint32_t nx = grow_list<kW>(T, ac, warp_gid, ps, s);
                if ((int)lane == s) settle(nx);
            }
        }
        if (pending && ++rounds >= T.iter_limit) {
            set_flag(T, kFlagIterLimit);
            pending = false;
        }
        first = false;
        __syncwarp();
    }
    if (has) {
        if (A.results) A.results[idx] = res;
        if (A.found) A.found[idx] = (uint8_t)fnd;
    }

}

// Register caps of the staged kernels: more resident warps hide more of each
// tile's staging latency (all kernels) and claim round trip (insert, mixed).
// Mixed kernels hold the claim rounds of their insert tiles and the read rounds
// of their search / delete tiles, and do better with more registers than bulk
// inserts (below 72, the 8 chunk reads of a scan no longer stay in flight
// together).
#ifndef SLAB_READ_MAXNREG
#define SLAB_READ_MAXNREG 72
#endif
#ifndef SLAB_CLAIM_MAXNREG
#define SLAB_CLAIM_MAXNREG 56
#endif
#ifndef SLAB_MIXED_MAXNREG
#define SLAB_MIXED_MAXNREG 72
#endif

template <int kKind>
constexpr bool kClaims = kKind == kKindInsert || kKind == kKindMixed;
// shared memory words per warp of a kind's kernel (the ring only where ops wait in one)
template <int kKind, uint32_t kW>
constexpr uint32_t kWordsPerWarp = kKind == kKindInsert ? kServeWordsPerWarp<kW>
                                   : (kKind == kKindMixed ? kMixedWordsPerWarp<kW> : kStagedWordsPerWarp<kW>);

// kW: words per slab, 32 (128-byte slabs) or 16 (64-byte slabs)
template <int kKind, bool kKeyOnly, uint32_t kW>
__global__ void __maxnreg__(kKind == kKindMixed ? SLAB_MIXED_MAXNREG
                                                : (kClaims<kKind> ? SLAB_CLAIM_MAXNREG : SLAB_READ_MAXNREG))
    staged_kernel(TableView T, BatchArgs A) {
    static_assert(kW == 32u || kW == 16u, "128- or 64-byte slabs");
    extern __shared__ __align__(16) uint32_t smem[];
    constexpr bool kNeedsValue = (kKind == kKindInsert || kKind == kKindMixed) && !kKeyOnly;
    const uint32_t lane = lane_id();
    uint32_t* buf = smem + (threadIdx.x >> 5) * kWordsPerWarp<kKind, kW>;
    uint32_t* ballots = buf + kTileWords<kW>;
    uint32_t* skeys = ballots + 32;
    uint32_t* salts = skeys + 32;
    uint32_t* q_idx = salts + 32;  // the ring (search and delete kernels)
    uint32_t* q_u = q_idx + kDeferSlots;
    uint32_t* q_key = q_u + kDeferSlots;
    uint32_t* q_rounds = q_key + kDeferSlots;
    uint32_t* q_op = q_rounds + kDeferSlots;  // mixed kernels: the ring's op codes, then the insert queue
    const uint32_t buf_s = (uint32_t)__cvta_generic_to_shared(buf);
    const uint32_t warp_gid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t ntiles = (A.n + 31u) / 32u;
    // Launched as a programmatic dependent: touch no memory before the previous
    // kernel on the stream has completed (griddepcontrol.wait below). The next
    // batch's grid is scheduled as our blocks exit; triggering it at our start
    // instead (griddepcontrol.launch_dependents) parks its blocks on the SMs of
    // our tail and measured slower.
    uint32_t t = warp_gid;
    if (t >= ntiles) return;  // warp-uniform

    uint32_t off[8];
    stage_offsets<kW>(lane, off);

    AllocCtx ac{kNoBlock, 0u, 0u};
    asm volatile("griddepcontrol.wait;" ::: "memory");

    auto fetch = [&](uint32_t tt, uint32_t& k, uint32_t& v, uint32_t& o) {
        const uint32_t i = tt * 32u + lane;
        const bool has = tt < ntiles && i < A.n;
        o = kNoOpCode;
        k = 0u;
        v = 0u;
        if (has) {
            o = kKind == kKindMixed ? ld_stream_u8(A.ops + i) : fixed_op<kKind>();
            k = ld_stream(A.keys + i);
            if (kNeedsValue && A.values) v = ld_stream(A.values + i);
        }
    };
    auto walks = [](uint32_t k, uint32_t o) { return o <= kOpSearch && k < kTombstone; };

    // Search / delete ops that must go on to another slab wait in a ring of
    // kDeferSlots entries; qh / qn: its head and count (warp-uniform).
    uint32_t qh = 0u, qn = 0u;
    auto push = [&](bool keep, uint32_t i, uint32_t uu, uint32_t k, uint32_t r, uint32_t op) {
        const uint32_t b = __ballot_sync(kFull, keep);
        if (keep) {
            const uint32_t pos = (qh + qn + __popc(b & ((1u << lane) - 1u))) & (kDeferSlots - 1u);
            q_idx[pos] = i;
            q_u[pos] = uu;
            q_key[pos] = k;
            q_rounds[pos] = r;
            if constexpr (kKind == kKindMixed) q_op[pos] = op;
        }
        qn += __popc(b);
        __syncwarp();
    };
    auto round_done = [&](bool& pending, uint32_t& r) {
        if (pending && ++r >= T.iter_limit) {
            set_flag(T, kFlagIterLimit);
            pending = false;
        }
    };
    // tiles of waiting ops: whenever 32 wait, and (last) after the warp's last
    // tile until the ring is empty
    auto drain = [&](bool last) {
        if constexpr (kKind != kKindInsert) {
            while (qn >= 32u || (last && qn)) {
                const uint32_t take = qn < 32u ? qn : 32u;
                const bool mine = lane < take;
                const uint32_t pos = (qh + lane) & (kDeferSlots - 1u);
                uint32_t i = 0u, uu = 0u, k = 0u, rr = 0u, op = fixed_op<kKind == kKindMixed ? kKindSearch : kKind>();
                if (mine) {
                    i = q_idx[pos];
                    uu = q_u[pos];
                    k = q_key[pos];
                    rr = q_rounds[pos];
                    if constexpr (kKind == kKindMixed) op = q_op[pos];
                }
                qh = (qh + take) & (kDeferSlots - 1u);
                qn -= take;
                const uint32_t pm = take >= 32u ? kFull : (1u << take) - 1u;
                stage_slabs<kW>(T, buf_s, uu, pm, lane);
                cp_async_commit();
                if constexpr (!SLAB_LANE_MATCH) skeys[lane] = match_key(T, k, op);
                cp_async_wait<0>();
                __syncwarp();
                bool more = mine;
                uint32_t rs = default_result(op), fd = 0u;
                read_round<kKind, kKeyOnly, kW>(T, buf, ballots, skeys, off, pm, more, uu, rs, fd, k, op);
                round_done(more, rr);
                if (mine && !more) {
                    if (A.results) A.results[i] = rs;
                    if (A.found) A.found[i] = (uint8_t)fd;
                }
                __syncwarp();
                push(more, i, uu, k, rr, op);
            }
        }
    };

    if constexpr (kKind == kKindMixed) {
        if (!T.prefetch_l2) {
            // Mixed batches on L2-resident tables: each input tile's ops are sorted by
            // kind into two per-warp queues, inserts (served as tiles of the insert
            // kernel's claim rounds) and searches / deletes (the ring, served with
            // read rounds), so that every tile the warp serves holds one kind of op.
            uint32_t* i_idx = q_op + kDeferSlots;
            uint32_t* i_key = i_idx + kDeferSlots;
            uint32_t* i_val = i_key + kDeferSlots;
            uint32_t* i_bkt = i_val + kDeferSlots;
            uint32_t ih = 0u, in = 0u;  // the insert queue's head and count (warp-uniform)
            uint32_t ck, cv, co;
            fetch(t, ck, cv, co);
            for (; t < ntiles; t += nwarps) {
                uint32_t nk, nv, no;
                fetch(t + nwarps, nk, nv, no);
                const uint32_t idx = t * 32u + lane;
                if (co <= kOpSearch && ck >= kTombstone) set_flag(T, kFlagReserved);
                const bool walk = walks(ck, co);
                if (idx < A.n && !walk) {  // reserved keys and unknown op codes
                    if (A.results) A.results[idx] = default_result(co);
                    if (A.found) A.found[idx] = 0u;
                }
                const uint32_t b = walk ? bucket_of(T, ck) : 0u;
                const bool ins = walk && co == kOpInsert;
                const uint32_t im = __ballot_sync(kFull, ins);
                if (ins) {
                    const uint32_t pos = (ih + in + __popc(im & ((1u << lane) - 1u))) & (kDeferSlots - 1u);
                    i_idx[pos] = idx;
                    i_key[pos] = ck;
                    i_val[pos] = cv;
                    i_bkt[pos] = b;
                }
                in += __popc(im);
                push(walk && !ins, idx, b, ck, 0u, co);
                const bool last = t + nwarps >= ntiles;
                while (in >= 32u || (last && in)) {
                    const uint32_t take = in < 32u ? in : 32u;
                    const bool mine = lane < take;
                    const uint32_t pos = (ih + lane) & (kDeferSlots - 1u);
                    uint32_t i = 0u, k = 0u, v = 0u, bk = 0u, o = kNoOpCode;
                    if (mine) {
                        i = i_idx[pos];
                        k = i_key[pos];
                        v = i_val[pos];
                        bk = i_bkt[pos];
                        o = kOpInsert;
                    }
                    ih = (ih + take) & (kDeferSlots - 1u);
                    in -= take;
                    stage_slabs<kW>(T, buf_s, bk, take >= 32u ? kFull : (1u << take) - 1u, lane);
                    cp_async_commit();
                    if constexpr (!SLAB_LANE_MATCH) skeys[lane] = match_key(T, k, o);
                    cp_async_wait<0>();
                    __syncwarp();
                    serve_tile<kKindInsert, kKeyOnly, kW>(T, A, ac, warp_gid, buf, buf_s, ballots, skeys, salts, off, k,
                                                          v, o, bk, i, mine);
                    __syncwarp();
                }
                drain(last);
                ck = nk; cv = nv; co = no;
            }
            return;
        }
    }

    // prologue: this tile hashed (its base slabs pulled into L2 for big tables),
    // the next tile loading
    uint32_t ck, cv, co;
    fetch(t, ck, cv, co);
    uint32_t cb = walks(ck, co) ? bucket_of(T, ck) : 0u;
    if (T.prefetch_l2 && walks(ck, co)) prefetch_l2(T.slabs + (uint64_t)cb * kW);
    uint32_t nk, nv, no;
    fetch(t + nwarps, nk, nv, no);

    // Search and delete batches: an op code is the kind's where the tile has an
    // op and none past the end, recomputed where needed instead of carried along
    // the pipeline (registers for the scan's chunk reads).
    auto opat = [&](uint32_t tt) -> uint32_t {
        return tt < ntiles && tt * 32u + lane < A.n ? fixed_op<kKind == kKindMixed ? kKindSearch : kKind>()
                                                    : (uint32_t)kNoOpCode;
    };
    for (; t < ntiles; t += nwarps) {
        if constexpr (!kClaims<kKind>) co = opat(t);
        // (1) this tile's base slabs start moving into the stage
        stage_slabs<kW>(T, buf_s, cb, __ballot_sync(kFull, walks(ck, co)), lane);
        cp_async_commit();
        // (2) meanwhile: hash the next tile (pulling its slabs into L2 for big
        //     tables), start loading the tile after it, publish this tile's keys
        if constexpr (!kClaims<kKind>) no = opat(t + nwarps);
        const bool nwalk = walks(nk, no);
        const uint32_t nb = nwalk ? bucket_of(T, nk) : 0u;
        if (T.prefetch_l2 && nwalk) prefetch_l2(T.slabs + (uint64_t)nb * kW);
        uint32_t mk, mv, mo;
        fetch(t + 2u * nwarps, mk, mv, mo);
        if constexpr (!SLAB_LANE_MATCH) {  // the WCWS steps read keys four at a time from here
            skeys[lane] = match_key(T, ck, co);
            if constexpr (kKind == kKindMixed) salts[lane] = alt_key(ck, co);
        }
        // (3) serve this tile once its slabs have landed
        cp_async_wait<0>();
        __syncwarp();
        const uint32_t idx = t * 32u + lane;
        if constexpr (kClaims<kKind>) {
            serve_tile<kKind, kKeyOnly, kW>(T, A, ac, warp_gid, buf, buf_s, ballots, skeys, salts, off, ck, cv, co,
                                            cb, idx, idx < A.n);
        } else if (T.prefetch_l2) {
            serve_tile<kKind, kKeyOnly, kW>(T, A, ac, warp_gid, buf, buf_s, ballots, skeys, salts, off, ck, cv, co,
                                            cb, idx, idx < A.n);
        } else {
            // the tile's first round; the ops that go on join the ring
            if (co <= kOpSearch && ck >= kTombstone) set_flag(T, kFlagReserved);
            bool pending = walks(ck, co);
            const uint32_t pend = __ballot_sync(kFull, pending);
            uint32_t res = default_result(co), fnd = 0u, u = cb, r = 0u;
            if (pend) {
                read_round<kKind, kKeyOnly, kW>(T, buf, ballots, skeys, off, pend, pending, u, res, fnd, ck);
                round_done(pending, r);
            }
            if (idx < A.n && !pending) {
                if (A.results) A.results[idx] = res;
                if (A.found) A.found[idx] = (uint8_t)fnd;
            }
            __syncwarp();
            push(pending, idx, u, ck, r, fixed_op<kKind>());
            drain(t + nwarps >= ntiles);
        }
        // (4) rotate the pipeline
        ck = nk; cv = nv; co = no; cb = nb;
        nk = mk; nv = mv; no = mo;
        __syncwarp();
    }
}

}  // namespace slab
