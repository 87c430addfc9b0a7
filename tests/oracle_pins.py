"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each ``pin_*`` takes a loaded oracle library and raises AssertionError when the
oracle disagrees with something other than itself: hand-derived golden values
(tests/golden/, each with its citation), closed forms, a brute-force flat-set
model of the Sec. 3.2 operations, invariants, and a statistical law. The same
pins run against deliberately broken builds of the oracle in
test_oracle_mutants.py, to show that each plausible mistake is caught.
"""
from __future__ import annotations

import os
import random

import numpy as np

from oracle.oracle import NOT_FOUND, OracleTable, check_alloc, fit_points, hash_of, learn_model, learned_buckets

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
P = 4294967291


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                yield line.split()


# --------------------------------------------------------------------------- hash
def pin_hash_golden(lib):
    """Sec. 3.3 hash on hand-derived cases (tests/golden/hash_cases.txt)."""
    for a, b, B, k, want in _rows("hash_cases.txt"):
        got = hash_of(int(a), int(b), int(B), int(k), lib=lib)
        assert got == int(want), f"h({k}; a={a}, b={b}) mod {B}: got {got}, want {want}"
    # a table's bucket() is the same function of its own (a, b, B)
    t = OracleTable(10, 3, 7, lib=lib)
    assert [t.bucket(k) for k in (1, 4, P, P + 1)] == [0, 9, 7, 0]


def pin_hash_uniform(lib):
    """Sec. 3.3: a universal hash spreads distinct keys evenly over B buckets.

    With random (a, b) and about 2^16 random distinct keys over B = 512 buckets the bucket
    counts must pass a chi-square test of uniformity (p-value > 1e-4), and no
    bucket may be empty. A transposed or dropped operand collapses the spread.
    """
    from scipy.stats import chisquare
    rng = np.random.default_rng(7)
    for _ in range(3):
        a = int(rng.integers(1, P))
        b = int(rng.integers(0, P))
        B = 512
        t = OracleTable(B, a, b, lib=lib)
        keys = np.unique(rng.integers(0, 0xFFFFFFFE, size=1 << 16, dtype=np.uint64))
        cnt = np.bincount(t.buckets(keys), minlength=B)
        assert cnt.min() > 0
        assert chisquare(cnt).pvalue > 1e-4, "bucket counts are not uniform"


# ------------------------------------------------------------------ set semantics
def pin_worked_example(lib):
    """Hand-derived trace of REPLACE / DELETE / SEARCH (tests/golden/worked_example.txt)."""
    t = OracleTable(1, 1, 0, lib=lib)
    for row in _rows("worked_example.txt"):
        if row[0] == "final":
            _, _, tot = t.stats()
            assert (tot["live"], tot["slots"], tot["slabs"]) == tuple(map(int, row[1:4])), tot
            continue
        op, key, val, _, want_found, want_res, want_lines = row
        code = {"insert": 0, "delete": 1, "search": 2}[op]
        before = t.lines
        res, found = t.mixed(np.array([code], np.uint8), np.array([int(key)], np.uint32),
                             np.array([int(val)], np.uint32))
        want_r = NOT_FOUND if want_res == "NF" else int(want_res)
        assert int(found[0]) == int(want_found), f"{row}: found {found[0]}"
        assert int(res[0]) == want_r, f"{row}: result {res[0]}"
        assert t.lines - before == int(want_lines), f"{row}: lines {t.lines - before}"


def pin_slab_boundaries(lib):
    """Slab layout of Sec. 4.2: slot s lies in slab floor(s / 15) (tests/golden/slab_boundaries.txt)."""
    for n, key, want_lines, want_slabs in _rows("slab_boundaries.txt"):
        n, key = int(n), int(key)
        t = OracleTable(1, 1, 0, lib=lib)
        keys = np.arange(100, 100 + n, dtype=np.uint32)
        t.insert(keys, keys)
        q = np.array([key if key >= 0 else 99], np.uint32)
        before = t.lines
        t.search(q)
        assert t.lines - before == int(want_lines), (n, key, t.lines - before)
        _, slabs, _ = t.stats()
        assert int(slabs[0]) == int(want_slabs), (n, slabs[0])


def pin_slab_boundaries_64(lib):
    """A 64-byte slab keeps 7 pairs or 14 keys (Sec. 4.2's layout at 16 words):
    slot s lies in slab floor(s / M) (tests/golden/slab_boundaries_64.txt)."""
    for mode, n, key, want_lines, want_slabs in _rows("slab_boundaries_64.txt"):
        n, key = int(n), int(key)
        t = OracleTable(1, 1, 0, key_only=mode == "ko", lib=lib, slab_bytes=64)
        keys = np.arange(100, 100 + n, dtype=np.uint32)
        t.insert(keys, keys)
        q = np.array([key if key >= 0 else 99], np.uint32)
        before = t.lines
        t.search(q)
        assert t.lines - before == int(want_lines), (mode, n, key, t.lines - before)
        _, slabs, _ = t.stats()
        assert int(slabs[0]) == int(want_slabs), (mode, n, slabs[0])


class FlatSet:
    """The Sec. 3.2 definitions written over a plain list of pairs, with no buckets."""

    def __init__(self):
        self.S = []

    def replace(self, k, v):
        had = any(x == k for x, _ in self.S)
        self.S = [(x, y) for x, y in self.S if x != k] + [(k, v)]
        return had

    def delete(self, k):
        had = any(x == k for x, _ in self.S)
        self.S = [(x, y) for x, y in self.S if x != k]
        return had

    def search(self, k):
        for x, y in self.S:
            if x == k:
                return y
        return None


def pin_bruteforce_sequences(lib):
    """Random op sequences over a tiny key universe agree with the flat-set model.

    B in {1, 2, 3} and 10 keys force collisions, replaces of present keys,
    deletes of absent keys and re-inserts after deletes.
    """
    rnd = random.Random(1234)
    for trial in range(60):
        B = 1 + trial % 3
        a, b = rnd.randrange(1, P), rnd.randrange(0, P)
        t = OracleTable(B, a, b, lib=lib)
        ref = FlatSet()
        new_inserts = deletes_hit = 0
        for _ in range(120):
            op = rnd.randrange(3)
            k = rnd.randrange(10) * 7919
            v = rnd.randrange(1 << 32)
            res, found = t.mixed(np.array([op], np.uint8), np.array([k], np.uint32),
                                 np.array([v], np.uint32))
            if op == 0:
                had = ref.replace(k, v)
                assert int(found[0]) == int(had) and int(res[0]) == int(not had)
                new_inserts += not had
            elif op == 1:
                had = ref.delete(k)
                assert int(found[0]) == int(had) and int(res[0]) == int(had)
                deletes_hit += had
            else:
                want = ref.search(k)
                assert int(found[0]) == int(want is not None)
                assert int(res[0]) == (NOT_FOUND if want is None else want)
        _, _, tot = t.stats()
        assert tot["live"] == len(ref.S) == new_inserts - deletes_hit
        assert tot["slots"] == new_inserts, "tombstones must not be reused"
        bk, keys, vals = t.export()
        assert sorted(zip(keys.tolist(), vals.tolist())) == sorted(ref.S)
        for bb, kk in zip(bk.tolist(), keys.tolist()):
            assert bb == t.bucket(kk)


def pin_batch_forms_agree(lib):
    """insert/delete/search batches give what the same ops give one at a time."""
    rng = np.random.default_rng(3)
    keys = rng.choice(1 << 20, size=3000, replace=False).astype(np.uint32)
    vals = rng.integers(0, 1 << 32, size=3000, dtype=np.uint64).astype(np.uint32)
    t1 = OracleTable(97, 5, 11, lib=lib)
    t2 = OracleTable(97, 5, 11, lib=lib)
    f1 = t1.insert(keys, vals)
    r2, f2 = t2.mixed(np.zeros(3000, np.uint8), keys, vals)
    assert (f1 == 0).all() and (f2 == 0).all() and (r2 == 1).all()
    d1 = t1.delete(keys[::3])
    r2, d2 = t2.mixed(np.ones(1000, np.uint8), keys[::3], None)
    assert (d1 == 1).all() and (d2 == 1).all() and (r2 == 1).all()
    v1, s1 = t1.search(keys)
    v2, s2 = t2.mixed(np.full(3000, 2, np.uint8), keys, None)
    want_found = np.ones(3000, np.uint8)
    want_found[::3] = 0
    assert (s1 == want_found).all() and (s2 == want_found).all()
    want_v = np.where(want_found == 1, vals, np.uint32(NOT_FOUND))
    assert (v1 == want_v).all() and (v2 == want_v).all()


def pin_invariants(lib):
    """Every live key is found with its latest value; deleted and absent keys are
    not; live = new inserts - deletes that hit; used slots = new inserts."""
    rng = np.random.default_rng(11)
    pool = rng.choice(1 << 31, size=20000, replace=False).astype(np.uint32)
    stored, absent = pool[:12000], pool[12000:]
    t = OracleTable(400, 123456789, 987654321, lib=lib)
    f = t.insert(stored, stored ^ np.uint32(0x9E3779B9))
    assert f.sum() == 0
    f = t.insert(stored[:3000], stored[:3000] + np.uint32(1))  # replaces
    assert f.sum() == 3000
    d = t.delete(stored[5000:9000])
    assert d.sum() == 4000
    d = t.delete(absent[:1000])
    assert d.sum() == 0
    v, found = t.search(stored)
    live = np.ones(12000, bool)
    live[5000:9000] = False
    assert (found.astype(bool) == live).all()
    want = stored ^ np.uint32(0x9E3779B9)
    want[:3000] = stored[:3000] + np.uint32(1)
    assert (v[live] == want[live]).all()
    assert (v[~live] == NOT_FOUND).all()
    v, found = t.search(absent)
    assert found.sum() == 0 and (v == NOT_FOUND).all()
    _, _, tot = t.stats()
    assert tot["live"] == 12000 - 4000
    assert tot["slots"] == 12000


def pin_reserved_keys(lib):
    """The two sentinel keys (Sec. 3.2 footnote) are refused, not stored."""
    t = OracleTable(8, 3, 4, lib=lib)
    keys = np.array([1, 0xFFFFFFFE, 2, 0xFFFFFFFF], np.uint32)
    f = t.insert(keys, keys)
    assert f.tolist() == [0, 0, 0, 0]
    _, _, tot = t.stats()
    assert tot["live"] == 2 and tot["reserved"] == 2
    v, found = t.search(keys)
    assert found.tolist() == [1, 0, 1, 0]
    assert v[1] == NOT_FOUND and v[3] == NOT_FOUND


# ------------------------------------------------------------- slab bookkeeping
def pin_slab_count_closed_form(lib):
    """A bucket with s used slots has max(1, ceil(s / M)) slabs (M = 15 pairs or
    30 keys per 128-byte slab, 7 or 14 per 64-byte slab, Sec. 4.2); the lines of n
    sequential new inserts into one bucket sum to sum_{i<n} (floor(i / M) + 1)."""
    for key_only, M, width in ((False, 15, 128), (True, 30, 128), (False, 7, 64), (True, 14, 64)):
        for n in (0, 1, 6, 7, 8, 13, 14, 15, 16, 29, 30, 31, 44, 45, 46, 100, 451):
            t = OracleTable(1, 1, 0, key_only=key_only, lib=lib, slab_bytes=width)
            keys = np.arange(1, n + 1, dtype=np.uint32)
            t.insert(keys, keys)
            slots, slabs, _ = t.stats()
            assert int(slots[0]) == n
            assert int(slabs[0]) == max(1, -(-n // M)), (key_only, width, n, slabs[0])
            assert t.lines == sum(i // M + 1 for i in range(n)), (key_only, width, n, t.lines)


def pin_max_utilization(lib):
    """Sec. 4.2 / Sec. 6.1: a single full bucket reaches the maximum utilization
    M x / (M x + y) = 120 / 128 (the paper's "94%"), in both modes; a 64-byte slab
    keeps the same 8 bytes of auxiliary word and next pointer, so 56 / 64."""
    for key_only, M in ((False, 15), (True, 30)):
        t = OracleTable(1, 1, 0, key_only=key_only, lib=lib)
        keys = np.arange(1, 15 * M + 1, dtype=np.uint32)
        t.insert(keys, keys)
        assert abs(t.utilization() - 120.0 / 128.0) < 1e-12, t.utilization()
        assert round(100 * t.utilization()) == 94
    for key_only, M in ((False, 7), (True, 14)):
        t = OracleTable(1, 1, 0, key_only=key_only, lib=lib, slab_bytes=64)
        keys = np.arange(1, 9 * M + 1, dtype=np.uint32)
        t.insert(keys, keys)
        assert abs(t.utilization() - 56.0 / 64.0) < 1e-12, t.utilization()


def pin_mean_slabs_binomial(lib):
    """Sec. 3.3: keys spread uniformly, so a bucket's load is Binomial(n, 1/B) and
    its expected slab count is E[max(1, ceil(X / M))]. At n = 2^16 the oracle's
    mean slabs per bucket must match that expectation within 2 %, for every
    beta the bulk benchmark sweeps (B = ceil(n / (M beta))), with M = 15 pairs per
    128-byte slab and 7 per 64-byte slab."""
    from scipy.stats import binom
    rng = np.random.default_rng(5)
    n = 1 << 16
    keys = np.unique(rng.integers(0, 0xFFFFFFFE, size=n, dtype=np.uint64)).astype(np.uint32)
    n = len(keys)
    for M, width in ((15, 128), (7, 64)):
        for beta in (0.2, 0.6, 1.0, 2.0):
            B = int(np.ceil(n / (M * beta)))
            t = OracleTable(B, int(rng.integers(1, P)), int(rng.integers(0, P)), lib=lib, slab_bytes=width)
            t.insert(keys, keys)
            _, slabs, tot = t.stats()
            x = np.arange(0, M * 40)
            pmf = binom.pmf(x, n, 1.0 / B)
            expect = float((pmf * np.maximum(1, -(-x // M))).sum())
            got = tot["slabs"] / B
            assert abs(got - expect) / expect < 0.02, (width, beta, got, expect)


# ------------------------------------------------------------------- SlabAlloc
def pin_alloc_check(lib):
    """Sec. 5 address layout (unit bits [0,10), memory block [10,24), super block
    [24,32)) and bitmap ownership (word w of a block covers units 32w..32w+31),
    on hand-built cases."""
    nb = 4
    bm = np.zeros(nb * 32, np.uint32)
    # block 0: units 0, 1 (word 0 bits 0-1) and unit 1023 (word 31, bit 31)
    bm[0] = 0b11
    bm[31] = 1 << 31
    # block 1, unit 37: word 32 + 1, bit 5
    bm[33] = 1 << 5
    # with 2 blocks per super block, super block 1 / block 1 is linear block 3, unit 64: word 96 + 2
    bm[98] = 1
    addrs = np.array([0, 1, 1023, (1 << 10) | 37, (1 << 24) | (1 << 10) | 64], np.uint32)
    assert check_alloc(addrs, bm, nb, blocks_per_super=2, lib=lib) == (0, 0)
    dup = np.array([0, 1, 1023, (1 << 10) | 37, (1 << 24) | (1 << 10) | 64, 1], np.uint32)
    assert check_alloc(dup, bm, nb, blocks_per_super=2, lib=lib)[0] == 2
    bad = np.array([(2 << 10) | 5], np.uint32)  # block field 2 >= 2 blocks per super block
    assert check_alloc(bad, np.zeros(nb * 32, np.uint32), nb, blocks_per_super=2, lib=lib)[0] == 1
    far = np.array([(2 << 24) | 5], np.uint32)  # super block 2 -> linear block 4 >= 4 blocks
    assert check_alloc(far, np.zeros(nb * 32, np.uint32), nb, blocks_per_super=2, lib=lib)[0] == 1
    bm2 = bm.copy()
    bm2[0] = 0b111
    assert check_alloc(addrs, bm2, nb, blocks_per_super=2, lib=lib) == (3, 0)


# ------------------------------------------------------- learned bucket function
def pin_learned_fit_lines(lib):
    """Least-squares lines through integer points with known answers: collinear
    points give their line exactly; points sharing one x give a flat line at the
    mean; two points give the line through both."""
    assert tuple(fit_points([1, 2, 3], [2, 4, 6], lib=lib)) == (2.0, 0.0)
    assert tuple(fit_points([0, 2], [1, 3], lib=lib)) == (1.0, 1.0)
    assert tuple(fit_points([5, 5], [1, 3], lib=lib)) == (0.0, 2.0)
    assert tuple(fit_points([7], [9], lib=lib)) == (0.0, 9.0)
    assert tuple(fit_points([10, 20, 30, 40], [5, 5, 5, 5], lib=lib)) == (0.0, 5.0)
    a, b = fit_points([0, 1 << 31], [0, 1 << 20], lib=lib)
    assert a == np.float32(2.0 ** -11) and b == 0.0


def pin_learned_tiny_golden(lib):
    """Hand-derived fit and evaluation on four keys (tests/golden/learned_tiny.txt)."""
    rows = list(_rows("learned_tiny.txt"))
    keys = np.array([int(v) for v in rows[0][1:]], np.uint32)
    model, m = learn_model(keys, 1, 8, lib=lib)
    assert m == 4
    for row in rows[1:]:
        if row[0] == "root":
            assert (model[0], model[1]) == (float(row[1]), float(row[2])), model[:2]
        elif row[0] == "leaf":
            j = int(row[1])
            assert (model[2 + 2 * j], model[3 + 2 * j]) == (float(row[2]), float(row[3])), (j, model[2 + 2 * j:4 + 2 * j])
        elif row[0] == "bucket":
            assert int(learned_buckets(model, 8, [int(row[1])], lib=lib)[0]) == int(row[2]), row


def pin_learned_uniform_keys_balance(lib):
    """Evenly spaced keys have a linear CDF, so a model fitted on all of them (in any
    order) spreads them almost perfectly: every bucket receives n / B keys, give or
    take two."""
    n, B = 1 << 16, 4096
    keys = (np.arange(n, dtype=np.uint64) * 65521 + 12345).astype(np.uint32)
    model, _ = learn_model(keys[np.random.default_rng(1).permutation(n)], 1, B, lib=lib)
    load = np.bincount(learned_buckets(model, B, keys, lib=lib), minlength=B)
    assert load.min() >= n // B - 2 and load.max() <= n // B + 2, (load.min(), load.max())


def pin_learned_table_semantics(lib):
    """Set semantics do not depend on the bucket function: a table on a learned model
    agrees with the flat-set model, and chain_profile (sum and max of slabs per
    bucket the keys would form) matches the slabs after inserting those keys."""
    rng = np.random.default_rng(9)
    keys = np.unique(rng.integers(0, 1 << 32, 6000, dtype=np.uint64) % 0xFFFFFFFE).astype(np.uint32)
    B = 300
    model, _ = learn_model(keys, 3, B, lib=lib)
    t = OracleTable(B, 11, 13, lib=lib)
    t.use_model(model)
    sm, mx = t.chain_profile(keys)
    f = t.insert(keys, keys ^ np.uint32(77))
    assert f.sum() == 0
    _, slabs, tot = t.stats()
    assert tot["slabs"] == sm and int(slabs.max()) == mx
    for k, bk in zip(keys[:200].tolist(), t.buckets(keys[:200]).tolist()):
        assert bk == learned_buckets(model, B, [k], lib=lib)[0]
    v, found = t.search(keys)
    assert found.all() and (v == (keys ^ np.uint32(77))).all()
    ref = FlatSet()
    for k in keys[:500].tolist():
        ref.replace(k, k ^ 77)
    d = t.delete(keys[:100])
    assert d.all()
    _, _, tot = t.stats()
    assert tot["live"] == len(keys) - 100
    assert int(learned_buckets(model, B, [0, 0xFFFFFFFD], lib=lib).max()) < B


# ------------------------------------------------------------- multiset and flush
class FlatMultiset:
    """Sec. 3.2 with duplicates allowed, over one flat list in insertion order:
    INSERT appends, DELETE removes the least recent instance, DELETEALL every
    instance, SEARCH returns the least recent, SEARCHALL all in insertion order."""

    def __init__(self):
        self.S = []

    def insert(self, k, v):
        self.S.append((k, v))

    def delete(self, k):
        for i, (x, _) in enumerate(self.S):
            if x == k:
                del self.S[i]
                return True
        return False

    def delete_all(self, k):
        n = sum(1 for x, _ in self.S if x == k)
        self.S = [(x, y) for x, y in self.S if x != k]
        return n

    def search_all(self, k):
        return [y for x, y in self.S if x == k]


def _multiset_table(B, lib, a=7, b=3):
    t = OracleTable(B, a, b, lib=lib)
    t.set_multiset()
    return t


def pin_multiset_golden(lib):
    """Hand-derived INSERT / DELETE / DELETEALL / SEARCH(ALL) / FLUSH sequence on one
    bucket (tests/golden/multiset_flush_example.txt)."""
    t = _multiset_table(1, lib)
    for row in _rows("multiset_flush_example.txt"):
        op, args = row[0], row[1:]
        want = args[args.index("->") + 1:] if "->" in args else None
        args = args[: args.index("->")] if "->" in args else args
        if op == "insert":
            t.insert([int(args[0])], [int(args[1])])
        elif op == "delete":
            assert int(t.delete([int(args[0])])[0]) == int(want[0])
        elif op == "delete_all":
            assert int(t.delete_all([int(args[0])])[0]) == int(want[0])
        elif op == "search":
            v, f = t.search([int(args[0])])
            assert f[0] == 1 and int(v[0]) == int(want[0])
        elif op == "search_all":
            c, vals = t.search_all([int(args[0])], 8)
            assert vals[0, : int(c[0])].tolist() == [int(x) for x in want]
        elif op == "export":
            _, k, v = t.export()
            assert [f"{a}:{b}" for a, b in zip(k.tolist(), v.tolist())] == want
        elif op == "slabs":
            assert t.stats()[2]["slabs"] == int(want[0])
        elif op == "flush":
            assert t.flush() == int(want[0])
        else:
            raise AssertionError(op)


def pin_multiset_insert_lines(lib):
    """Slab reads of multiset INSERT and DELETE, hand-derived on one bucket
    (tests/golden/multiset_insert_lines.txt): an insert that fills a hole reads up
    to the hole's slab, one that appends up to the tail slot's slab."""
    t = _multiset_table(1, lib)
    for row in _rows("multiset_insert_lines.txt"):
        op, args = row[0], row[1:]
        want = int(args[args.index("->") + 1])
        before = t.lines
        if op == "insert":
            t.insert([int(args[0])], [int(args[1])])
        elif op == "delete":
            assert int(t.delete([int(args[0])])[0]) == 1
        else:
            raise AssertionError(op)
        assert t.lines - before == want, (row, t.lines - before)


def pin_multiset_bruteforce(lib):
    """Random INSERT / DELETE / DELETEALL / SEARCH(ALL) sequences over a tiny key
    universe agree with the flat multiset model. Every instance of a key carries the
    same value, so which instance a DELETE removes cannot show; the counts, found
    flags and the live multiset must match exactly."""
    rnd = random.Random(4321)
    for trial in range(50):
        B = 1 + trial % 3
        t = _multiset_table(B, lib, rnd.randrange(1, P), rnd.randrange(0, P))
        ref = FlatMultiset()
        for _ in range(150):
            op = rnd.randrange(5)
            k = rnd.randrange(8) * 104729
            v = k ^ 0x5A5A
            if op <= 1:
                t.insert([k], [v])
                ref.insert(k, v)
            elif op == 2:
                assert int(t.delete([k])[0]) == int(ref.delete(k))
            elif op == 3:
                assert int(t.delete_all([k])[0]) == ref.delete_all(k)
            else:
                c, vals = t.search_all([k], 64)
                want = ref.search_all(k)
                assert int(c[0]) == len(want) and vals[0, : len(want)].tolist() == want
                sv, sf = t.search([k])
                assert int(sf[0]) == int(bool(want)) and (not want or int(sv[0]) == want[0])
        _, _, tot = t.stats()
        assert tot["live"] == len(ref.S)
        _, kk, vv = t.export()
        assert sorted(zip(kk.tolist(), vv.tolist())) == sorted(ref.S)


def pin_multiset_insert_order(lib):
    """With no deletes, list order is insertion order: SEARCH returns the least
    recently inserted value and SEARCHALL returns them in insertion order
    (Sec. 3.2 definitions); duplicates occupy one slot each (slots = inserts)."""
    rng = np.random.default_rng(5)
    t = _multiset_table(13, lib)
    keys = rng.integers(0, 40, 2000).astype(np.uint32)
    vals = np.arange(2000, dtype=np.uint32)
    f = t.insert(keys, vals)
    assert f.sum() == 0
    v, found = t.search(np.arange(40, dtype=np.uint32))
    c, allv = t.search_all(np.arange(40, dtype=np.uint32), 200)
    for k in range(40):
        idx = np.flatnonzero(keys == k)
        assert int(c[k]) == len(idx)
        if len(idx):
            assert found[k] == 1 and int(v[k]) == int(idx[0])
            assert allv[k, : min(len(idx), 200)].tolist() == idx[:200].tolist()
    _, _, tot = t.stats()
    assert tot["slots"] == 2000 and tot["live"] == 2000


def pin_set_table_all_ops(lib):
    """In a set table (unique keys) SEARCHALL finds at most one instance and agrees
    with SEARCH, and DELETEALL does what DELETE does."""
    rng = np.random.default_rng(6)
    keys = rng.choice(1 << 24, 3000, replace=False).astype(np.uint32)
    t1 = OracleTable(101, 9, 4, lib=lib)
    t2 = OracleTable(101, 9, 4, lib=lib)
    for t in (t1, t2):
        t.insert(keys, keys + np.uint32(1))
    q = np.concatenate([keys[:500], rng.choice(1 << 24, 500).astype(np.uint32) | np.uint32(1 << 25)])
    c, vals = t1.search_all(q, 2)
    v, f = t1.search(q)
    assert (c == f).all() and (vals[f == 1, 0] == v[f == 1]).all()
    d1 = t1.delete(keys[::4])
    d2 = t2.delete_all(keys[::4])
    assert (d1 == d2).all()
    assert t1.stats()[2] == t2.stats()[2]
    assert all((x == y).all() for x, y in zip(t1.export(), t2.export()))


def pin_flush_compacts(lib):
    """Sec. 4.3.4 FLUSH: the live elements (and their list order) are unchanged,
    every bucket keeps the minimum number of slabs, max(1, ceil(live / M)), counted
    here from the exported elements, and the released slabs are the difference.
    The flushed table then behaves like a fresh one filled with the export in order."""
    rng = np.random.default_rng(8)
    for key_only, multiset in ((False, False), (True, False), (False, True)):
        M = 30 if key_only else 15
        B = 50
        t = OracleTable(B, 3, 1, key_only=key_only, lib=lib)
        if multiset:
            t.set_multiset()
        keys = rng.choice(1 << 24, 4000, replace=False).astype(np.uint32)
        t.insert(keys, keys ^ np.uint32(3))
        t.delete(keys[rng.permutation(4000)[:2500]])
        before_export = t.export()
        before_slabs = t.stats()[2]["slabs"]
        released = t.flush()
        after = t.export()
        assert all((x == y).all() for x, y in zip(before_export, after))
        live = np.bincount(after[0], minlength=B)
        _, slabs, tot = t.stats()
        assert (slabs == np.maximum(1, (live + M - 1) // M)).all()
        assert tot["slots"] == len(after[0]) and released == before_slabs - tot["slabs"]
        fresh = OracleTable(B, 3, 1, key_only=key_only, lib=lib)
        if multiset:
            fresh.set_multiset()
        fresh.insert(after[1], after[2])
        assert (fresh.stats()[1] == slabs).all() and (fresh.stats()[0] == t.stats()[0]).all()
        more = rng.choice(1 << 24, 800, replace=False).astype(np.uint32) | np.uint32(1 << 25)
        t.insert(more, more)
        fresh.insert(more, more)
        assert all((x == y).all() for x, y in zip(t.export(), fresh.export()))
        assert t.flush() == 0 or not multiset


def pin_flush_noop_and_empty(lib):
    """FLUSH of a table without deletes changes nothing; FLUSH after deleting
    everything leaves every bucket one empty slab."""
    rng = np.random.default_rng(12)
    keys = rng.choice(1 << 24, 1000, replace=False).astype(np.uint32)
    t = OracleTable(20, 5, 6, lib=lib)
    t.insert(keys, keys)
    s0, b0, tot0 = t.stats()
    assert t.flush() == 0
    s1, b1, tot1 = t.stats()
    assert (s0 == s1).all() and (b0 == b1).all() and tot0 == tot1
    t.delete(keys)
    released = t.flush()
    s2, b2, tot2 = t.stats()
    assert (s2 == 0).all() and (b2 == 1).all() and released == tot1["slabs"] - 20


ALL_PINS = [v for k, v in sorted(globals().items()) if k.startswith("pin_")]
