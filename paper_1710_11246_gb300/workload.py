"""Seeded synthetic inputs shaped like the slab-hash paper's workloads (Sec. 6).

This module is shared by the tests, the benchmark and the oracle's callers. It
holds no part of the method's arithmetic: no bucket hash, no slab layout, no
set semantics. It only draws keys, values, op codes and the random hash
parameters that the method consumes as inputs.

Recipe (Sec. 6.1 and 6.3: uniform random 32-bit keys, no external dataset):

* Distinct keys come from one counter per ``KeyStream``. Counter ``c`` maps to
  ``pi((c + offset) mod (2^32 - 2))`` where ``pi`` is the bijective 32-bit
  "lowbias32" integer mixer (two xorshift-multiply rounds, Wellons' hash
  prospector). Outputs that land on the two reserved sentinels
  (0xFFFFFFFE, 0xFFFFFFFF) are re-mixed (cycle walking), which keeps the map
  one-to-one on [0, 2^32 - 3]. Consecutive counter ranges therefore give
  disjoint key sets: stored keys, absent keys and fresh insert keys never
  collide by construction.
* ``value = key XOR 0x9E3779B9``.
* The universal-hash parameters ``a`` in [1, p-1] and ``b`` in [0, p-1]
  (Sec. 3.3) are drawn from ``numpy.random.default_rng(seed)`` and handed
  to both implementations.
* Search batches mix present keys (a random subset of the stored keys) and
  absent keys (fresh counters) at a stated hit rate, shuffled.
* Clustered keys (the learned-bucket workload): draws from 64 Gaussian clusters
  with uniform centres and standard deviations in [2^10, 2^20], rounded, clamped
  and deduplicated; absent keys come from the same clusters.
* Mixed batches (Sec. 6.3) draw fresh inserts, deletes of distinct live keys,
  searches of live keys untouched by the batch and searches of absent keys, in
  stated ratios, shuffled so every op kind can land in one warp. Every key
  appears in at most one op per batch.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

VALUE_XOR = np.uint32(0x9E3779B9)
HASH_PRIME = 4294967291  # 2^32 - 5, the largest prime below 2^32
KEY_LIMIT = 0xFFFFFFFE   # keys must be < this; the two values above are sentinels
OP_INSERT, OP_DELETE, OP_SEARCH = 0, 1, 2

_M32 = np.uint64(0xFFFFFFFF)


def _lowbias32(x: np.ndarray) -> np.ndarray:
    """Bijective 32-bit mixer (xorshift-multiply, constants 0x7feb352d / 0x846ca68b)."""
    x = x.astype(np.uint64)
    x ^= x >> np.uint64(16)
    x = (x * np.uint64(0x7FEB352D)) & _M32
    x ^= x >> np.uint64(15)
    x = (x * np.uint64(0x846CA68B)) & _M32
    x ^= x >> np.uint64(16)
    return x


def _mix_domain(x: np.ndarray) -> np.ndarray:
    """Cycle-walk the mixer until every output is a legal key (< 0xFFFFFFFE)."""
    y = _lowbias32(x)
    bad = y >= np.uint64(KEY_LIMIT)
    while bad.any():
        y[bad] = _lowbias32(y[bad])
        bad = y >= np.uint64(KEY_LIMIT)
    return y.astype(np.uint32)


class KeyStream:
    """Hands out disjoint ranges of distinct uniform keys for one seed."""

    def __init__(self, seed: int = 0):
        self.seed = int(seed)
        rng = np.random.default_rng([self.seed, 0x5EED])
        self._offset = int(rng.integers(0, KEY_LIMIT))
        self._next = 0

    def take(self, n: int) -> np.ndarray:
        n = int(n)
        if self._next + n > KEY_LIMIT:
            raise ValueError("key stream exhausted")
        c = np.arange(self._next, self._next + n, dtype=np.uint64)
        self._next += n
        c = (c + np.uint64(self._offset)) % np.uint64(KEY_LIMIT)
        return _mix_domain(c)


def values_for(keys: np.ndarray) -> np.ndarray:
    return (np.asarray(keys, dtype=np.uint32) ^ VALUE_XOR).astype(np.uint32)


def hash_params(seed: int = 0) -> tuple[int, int]:
    """Random a in [1, p-1], b in [0, p-1] for h(k) = ((a k + b) mod p) mod B."""
    rng = np.random.default_rng([int(seed), 0xA11CE])
    a = int(rng.integers(1, HASH_PRIME))
    b = int(rng.integers(0, HASH_PRIME))
    return a, b


def buckets_for(n: int, beta: float, per_slab: int = 15) -> int:
    """B = ceil(n / (M beta)): the bucket count giving a mean of beta slabs per bucket."""
    return max(1, int(math.ceil(n / (per_slab * beta) - 1e-9)))


@dataclass
class SearchBatch:
    keys: np.ndarray
    present: np.ndarray  # bool, True where the key was drawn from the stored set


def search_batch(stream: KeyStream, stored: np.ndarray, n: int, hit_rate: float,
                 rng: np.random.Generator) -> SearchBatch:
    n_hit = int(round(n * hit_rate))
    n_hit = min(n_hit, len(stored)) if len(stored) else 0
    n_miss = n - n_hit
    hit = stored[rng.choice(len(stored), size=n_hit, replace=False)] if n_hit else \
        np.empty(0, np.uint32)
    miss = stream.take(n_miss)
    keys = np.concatenate([hit, miss]).astype(np.uint32)
    present = np.concatenate([np.ones(n_hit, bool), np.zeros(n_miss, bool)])
    perm = rng.permutation(n)
    return SearchBatch(keys[perm], present[perm])


@dataclass
class MixedBatch:
    ops: np.ndarray     # uint8 op codes
    keys: np.ndarray    # uint32
    values: np.ndarray  # uint32 (inserts: key ^ C; others: 0)


def mixed_batch(stream: KeyStream, live: np.ndarray, n: int,
                ratios: tuple[float, float, float], rng: np.random.Generator,
                ) -> tuple[MixedBatch, np.ndarray]:
    """One batch of n mixed ops; returns the batch and the live key set after it."""
    fi, fd, fs = ratios
    n_ins = int(round(n * fi))
    n_del = min(int(round(n * fd)), len(live))
    n_search = n - n_ins - n_del
    n_sh = min(n_search // 2, max(0, len(live) - n_del))
    n_sm = n_search - n_sh
    pick = rng.choice(len(live), size=n_del + n_sh, replace=False) if len(live) else \
        np.empty(0, np.int64)
    dels = live[pick[:n_del]]
    shit = live[pick[n_del:]]
    ins = stream.take(n_ins)
    smiss = stream.take(n_sm)
    keys = np.concatenate([ins, dels, shit, smiss]).astype(np.uint32)
    ops = np.concatenate([np.full(n_ins, OP_INSERT, np.uint8), np.full(n_del, OP_DELETE, np.uint8),
                          np.full(n_sh + n_sm, OP_SEARCH, np.uint8)])
    vals = np.concatenate([values_for(ins), np.zeros(n - n_ins, np.uint32)]).astype(np.uint32)
    perm = rng.permutation(n)
    keep = np.ones(len(live), bool)
    keep[pick[:n_del]] = False
    new_live = np.concatenate([live[keep], ins]).astype(np.uint32)
    return MixedBatch(ops[perm], keys[perm], vals[perm]), new_live


@dataclass
class BulkWorkload:
    """Sec. 6.1 bulk benchmark: build n pairs, search, delete."""
    num_buckets: int
    hash_a: int
    hash_b: int
    keys: np.ndarray
    values: np.ndarray
    search: SearchBatch
    delete_keys: np.ndarray


def bulk_workload(n: int, beta: float, n_search: int, hit_rate: float, n_delete: int,
                  seed: int = 0, num_buckets: int | None = None, per_slab: int = 15) -> BulkWorkload:
    stream = KeyStream(seed)
    rng = np.random.default_rng([int(seed), 0xB01C])
    keys = stream.take(n)
    a, b = hash_params(seed)
    B = num_buckets if num_buckets is not None else buckets_for(n, beta, per_slab)
    sb = search_batch(stream, keys, n_search, hit_rate, rng)
    dels = keys[rng.choice(n, size=min(n_delete, n), replace=False)] if n_delete else \
        np.empty(0, np.uint32)
    return BulkWorkload(B, a, b, keys, values_for(keys), sb, dels.astype(np.uint32))


def config1(seed: int = 0) -> BulkWorkload:
    """2^16 pairs into 2^16/(15*0.6) buckets, 2^16 searches at 50 % hit, 2^14 deletes."""
    return bulk_workload(1 << 16, 0.6, 1 << 16, 0.5, 1 << 14, seed)


def config2(beta: float = 0.6, hit_rate: float = 0.5, seed: int = 0, per_slab: int = 15) -> BulkWorkload:
    """2^22 pairs, 2^22 searches at the given hit rate, 2^20 deletes; per_slab = M
    (15 pairs per 128-byte slab, 7 per 64-byte slab) sets B = ceil(n / (M beta))."""
    return bulk_workload(1 << 22, beta, 1 << 22, hit_rate, 1 << 20, seed, per_slab=per_slab)


def _cluster_draws(rng, centres, sigmas, count):
    c = rng.integers(0, len(centres), count)
    x = np.rint(centres[c] + sigmas[c] * rng.standard_normal(count))
    return np.clip(x, 0, KEY_LIMIT - 1).astype(np.uint64).astype(np.uint32)


def clustered_keys(n: int, seed: int = 0, clusters: int = 64, sigma_lo: float = 2.0 ** 10,
                   sigma_hi: float = 2.0 ** 20, extra: int = 0):
    """n distinct keys from `clusters` Gaussian clusters (centres uniform in
    [0, 2^32), standard deviations uniform in [sigma_lo, sigma_hi]), rounded,
    clamped to [0, 2^32 - 3] and deduplicated, in random order; plus `extra`
    further distinct keys from the same clusters that are not among the n."""
    rng = np.random.default_rng([int(seed), 0xC1A5])
    centres = rng.uniform(0.0, 2.0 ** 32, clusters)
    sigmas = rng.uniform(sigma_lo, sigma_hi, clusters)
    pool = np.empty(0, np.uint32)
    need = n + extra
    while len(pool) < need:
        pool = np.unique(np.concatenate([pool, _cluster_draws(rng, centres, sigmas, max(1 << 16, need - len(pool)) * 2)]))
    pick = rng.permutation(len(pool))[:need]
    keys = pool[pick]
    return keys[:n].copy(), keys[n:].copy()


def config4(seed: int = 0, n: int = 1 << 22, beta: float = 0.6, hit_rate: float = 0.5) -> BulkWorkload:
    """Clustered keys: n pairs, searches of n keys at the hit rate (absent keys from
    the same clusters), no deletes."""
    n_miss = n - int(round(n * hit_rate))
    keys, absent = clustered_keys(n, seed, extra=n_miss)
    rng = np.random.default_rng([int(seed), 0xC4])
    a, b = hash_params(seed)
    n_hit = n - n_miss
    q = np.concatenate([keys[rng.choice(n, n_hit, replace=False)], absent])
    present = np.concatenate([np.ones(n_hit, bool), np.zeros(n_miss, bool)])
    perm = rng.permutation(n)
    return BulkWorkload(buckets_for(n, beta), a, b, keys, values_for(keys), SearchBatch(q[perm], present[perm]),
                        np.empty(0, np.uint32))


@dataclass
class GroupWorkload:
    """Many independent tables: per-table sizes, buckets and hash parameters, and
    batches concatenated by table (op_start[i] = first op of table i)."""
    sizes: np.ndarray
    num_buckets: np.ndarray
    hash_a: np.ndarray
    hash_b: np.ndarray
    op_start: np.ndarray
    keys: np.ndarray
    values: np.ndarray
    search_start: np.ndarray
    search_keys: np.ndarray
    search_present: np.ndarray


def group_workload(ntables: int, lo: int, hi: int, beta: float = 0.6, hit_rate: float = 0.5,
                   seed: int = 0, sizes=None, per_slab: int = 15) -> GroupWorkload:
    """`ntables` tables with sizes log-uniform in [lo, hi] (or the given sizes), each
    with B = ceil(n / (M beta)) (M = per_slab) and its own hash parameters; one
    search batch per table of n queries at the hit rate."""
    rng = np.random.default_rng([int(seed), 0x6A0])
    if sizes is None:
        sizes = np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi + 1), ntables))).astype(np.int64)
    sizes = np.asarray(sizes, np.int64)
    stream = KeyStream(seed + 0x5000)
    B = np.array([buckets_for(max(int(n), 1), beta, per_slab) for n in sizes], np.uint32)
    ha = rng.integers(1, HASH_PRIME, ntables).astype(np.uint32)
    hb = rng.integers(0, HASH_PRIME, ntables).astype(np.uint32)
    keys, qk, qp = [], [], []
    for n in sizes:
        k = stream.take(int(n))
        keys.append(k)
        sb = search_batch(stream, k, int(n), hit_rate, rng)
        qk.append(sb.keys)
        qp.append(sb.present)
    op_start = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint32)
    allk = np.concatenate(keys).astype(np.uint32) if keys else np.empty(0, np.uint32)
    return GroupWorkload(sizes, B, ha, hb, op_start, allk, values_for(allk), op_start.copy(),
                         np.concatenate(qk).astype(np.uint32), np.concatenate(qp))


@dataclass
class ServingTrace:
    """Requests for one resident table: request r arrives at arrival_ns[r] and owns
    ops [op_start[r], op_start[r + 1]). The table is first loaded with `preload`."""
    num_buckets: int
    hash_a: int
    hash_b: int
    preload: np.ndarray
    arrival_ns: np.ndarray  # uint64, non-decreasing
    op_start: np.ndarray    # uint64, R + 1 entries
    ops: np.ndarray         # uint8
    keys: np.ndarray        # uint32
    values: np.ndarray      # uint32


def request_sizes(n_requests: int, max_size: int, rng: np.random.Generator) -> np.ndarray:
    """Sizes log-uniform on [1, max_size]: floor(exp(U[0, ln(max_size + 1)))."""
    return np.floor(np.exp(rng.uniform(0.0, np.log(max_size + 1), n_requests))).astype(np.int64).clip(1, max_size)


def serving_trace(n_preload: int, n_requests: int, rate_per_s: float | None, beta: float = 0.6,
                  ratios: tuple[float, float, float] = (0.1, 0.1, 0.8), max_size: int = 1 << 16,
                  hit_rate: float = 0.5, seed: int = 0) -> ServingTrace:
    """Poisson arrivals at `rate_per_s` (None: every request at time 0), log-uniform sizes,
    op kinds drawn independently per op in `ratios`. Keys are disjoint across requests
    for every op that changes the table: inserts are fresh keys, deletes take distinct
    preloaded keys in order, searches hit the other preloaded keys (no request deletes
    them) or miss with fresh keys. Every result is therefore independent of the order
    in which requests run."""
    rng = np.random.default_rng([int(seed), 0x5E7])
    stream = KeyStream(seed + 0x7000)
    a, b = hash_params(seed)
    preload = stream.take(n_preload)
    sizes = request_sizes(n_requests, max_size, rng)
    total = int(sizes.sum())
    u = rng.random(total)
    fi, fd, _ = ratios
    ops = np.where(u < fi, OP_INSERT, np.where(u < fi + fd, OP_DELETE, OP_SEARCH)).astype(np.uint8)
    keys = np.empty(total, np.uint32)
    ins, dele, srch = ops == OP_INSERT, ops == OP_DELETE, ops == OP_SEARCH
    n_del = int(dele.sum())
    if n_del >= n_preload:
        raise ValueError("the trace deletes more keys than the table holds")
    keys[ins] = stream.take(int(ins.sum()))
    keys[dele] = preload[:n_del]
    stable = preload[n_del:]
    hit = srch & (rng.random(total) < hit_rate)
    miss = srch & ~hit
    n_hit = int(hit.sum())
    keys[hit] = stable[np.arange(n_hit) % len(stable)]
    keys[miss] = stream.take(int(miss.sum()))
    values = np.where(ins, values_for(keys), np.uint32(0)).astype(np.uint32)
    if rate_per_s is None:
        arrival = np.zeros(n_requests, np.uint64)
    else:
        arrival = np.floor(np.cumsum(rng.exponential(1e9 / rate_per_s, n_requests))).astype(np.uint64)
    op_start = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    return ServingTrace(buckets_for(n_preload, beta), a, b, preload, arrival, op_start, ops, keys, values)


CONFIG3_RATIOS = ((0.5, 0.5, 0.0), (0.2, 0.2, 0.6), (0.05, 0.05, 0.9))
CONFIG2_BETAS = (0.2, 0.4, 0.6, 0.8, 1.0, 2.0)
