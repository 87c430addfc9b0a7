"""The paper's other operations on the GPU vs the oracle: FLUSH (Sec. 4.3.4),
multiset tables with INSERT / DELETE / SEARCHALL / DELETEALL (Sec. 3.2), and
growing the SlabAlloc pool (Sec. 5).

Slot positions that concurrent inserts of one batch race for are not unique, so
those tests compare per-bucket counts and the multiset of stored elements; list
order is compared exactly wherever it is fixed (one instance of a key per batch
and no emptied slots before the inserts)."""
import numpy as np
import pytest
import torch

from oracle import OracleTable
from paper_1710_11246_gb300 import slabhash as sh
from paper_1710_11246_gb300 import workload as W
from tests.gpu_helpers import VARIANTS, Pair, dev, host, u8

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _lib():
    sh.load_library()


def _i32(n, fill=0):
    return torch.full((n,), fill, dtype=torch.int32, device="cuda")


def _search_all(p, keys, cap):
    n = len(keys)
    counts, vals = _i32(n), _i32(n * cap, -1)
    sh.slab_search_all_batch(p.g.handle, dev(keys), cap, counts, vals)
    return host(counts), host(vals).reshape(n, cap)


def _delete_all(p, keys):
    counts = _i32(len(keys))
    sh.slab_delete_all_batch(p.g.handle, dev(keys), counts)
    return host(counts)


@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("key_only", [False, True])
def test_flush_compacts_like_the_oracle(variant, key_only):
    """Delete most keys of a table with long lists, flush on both sides: the same
    slabs are released, every list has the oracle's slots and slabs, the pool
    bitmaps account exactly for the linked slabs, and later ops agree."""
    n = 1 << 15
    w = W.bulk_workload(n, 2.0, n, 0.5, 0, seed=31)  # beta 2: two slabs per list on average
    p = Pair(w.num_buckets, w.hash_a, w.hash_b, variant=variant, key_only=key_only, n_hint=n)
    try:
        p.insert(w.keys, None if key_only else w.values)
        rng = np.random.default_rng(2)
        p.delete(w.keys[rng.permutation(n)[: 3 * n // 4]])
        before = p.g.stats()
        released = sh.slab_flush(p.g.handle)
        assert released == p.o.flush() > 0
        tot = p.check_structure()
        assert tot["slabs"] == before["slabs"] - released and tot["prefix_violations"] == 0
        assert tot["pool_allocated"] == before["pool_allocated"] - released
        p.search(w.search.keys)
        more = W.KeyStream(77).take(n // 2)
        p.insert(more, None if key_only else W.values_for(more))
        p.delete(more[::3])
        p.check_structure()
        assert sh.slab_flush(p.g.handle) == p.o.flush()
        p.check_structure()
    finally:
        p.close()


def test_flush_edge_cases():
    """Flush of an empty table, of a table without deletes (nothing moves), and
    after deleting every key (one empty slab per list, whole pool free)."""
    w = W.bulk_workload(5000, 1.0, 0, 0.5, 0, seed=5)
    p = Pair(w.num_buckets, w.hash_a, w.hash_b, n_hint=5000)
    try:
        assert sh.slab_flush(p.g.handle) == 0 == p.o.flush()
        p.insert(w.keys, w.values)
        s0 = p.g.stats()
        assert sh.slab_flush(p.g.handle) == 0 == p.o.flush()
        assert p.check_structure() == s0 and s0["prefix_violations"] == 0
        p.delete(w.keys)
        released = sh.slab_flush(p.g.handle)
        assert released == p.o.flush() == s0["linked"]
        tot = p.check_structure()
        assert tot["live"] == 0 and tot["slots"] == 0 and tot["slabs"] == w.num_buckets
        assert tot["pool_allocated"] == 0
    finally:
        p.close()


def _multiset_pair(n_hint, variant="staged", key_only=False, B=None):
    B = B or W.buckets_for(n_hint, 1.0)
    p = Pair(B, 12345, 678, variant=variant, key_only=key_only, n_hint=2 * n_hint)
    sh.slab_set_multiset(p.g.handle)
    p.o.set_multiset()
    assert p.g.info.multiset == 0 and sh.slab_get_info(p.g.handle).multiset == 1
    return p


@pytest.mark.parametrize("variant", list(VARIANTS))
def test_multiset_insert_search_all_delete(variant):
    """Three insert batches re-use keys (each key once per batch): every instance is
    stored, SEARCHALL returns them in batch order, SEARCH the first, DELETE removes
    the first instance (the oracle's choice too) and DELETEALL the rest."""
    ks = W.KeyStream(3)
    base = ks.take(6000)
    rng = np.random.default_rng(4)
    batches = [base, base[rng.permutation(6000)[:4000]], base[rng.permutation(6000)[:2000]]]
    p = _multiset_pair(12000, variant)
    try:
        for j, b in enumerate(batches):
            vals = (b ^ np.uint32(0x1000 * (j + 1))).astype(np.uint32)
            f = p.insert(b, vals)
            assert f.sum() == 0
        p.check_structure()  # set-wise; positions fixed: no emptied slots yet
        q = np.concatenate([base[:3000], ks.take(500)])
        c, v = _search_all(p, q, 4)
        co, vo = p.o.search_all(q, 4)
        assert (c == co).all()
        assert (v == np.where(np.arange(4) < co[:, None], vo, 0xFFFFFFFF)).all()
        p.search(q)
        p.delete(base[:2500])
        p.check_structure(allow_holes=True)
        d = _delete_all(p, base[1000:4000])
        assert (d == p.o.delete_all(base[1000:4000])).all()
        p.check_structure(allow_holes=True)
        c, v = _search_all(p, base, 3)
        co, vo = p.o.search_all(base, 3)
        assert (c == co).all()
        for i in np.flatnonzero(co > 0)[:2000]:
            assert sorted(v[i, : min(co[i], 3)].tolist()) == sorted(vo[i, : min(co[i], 3)].tolist())
    finally:
        p.close()


@pytest.mark.parametrize("key_only", [False, True])
def test_multiset_holes_are_reused_and_flushed(key_only):
    """Deletes empty their slots; the next insert batch fills those slots before
    any list grows (per-bucket slots and slabs equal the oracle's), and a flush
    then compacts the lists. Values are a function of the key here, so which hole
    an instance lands in cannot show."""
    ks = W.KeyStream(9)
    keys = ks.take(20000)
    val = lambda k: (k * np.uint32(2654435761)).astype(np.uint32)  # noqa: E731
    p = _multiset_pair(20000, key_only=key_only)
    try:
        p.insert(keys, None if key_only else val(keys))
        p.insert(keys[:8000], None if key_only else val(keys[:8000]))
        p.delete(keys[5000:15000])
        p.check_structure(allow_holes=True)
        p.insert(keys[10000:16000], None if key_only else val(keys[10000:16000]))
        p.check_structure(allow_holes=True)
        c, _ = _search_all(p, keys, 0)
        co, _ = p.o.search_all(keys, 0)
        assert (c == co).all()
        released = sh.slab_flush(p.g.handle)
        assert released == p.o.flush()
        tot = p.check_structure()
        assert tot["prefix_violations"] == 0
    finally:
        p.close()


@pytest.mark.parametrize("variant", list(VARIANTS))
def test_multiset_mixed_batch(variant):
    """Mixed batches on a multiset table: inserts never report a key as present,
    deletes and searches act on first instances; set-wise parity with the oracle."""
    ks = W.KeyStream(21)
    keys = ks.take(8000)
    p = _multiset_pair(16000, variant)
    try:
        p.insert(keys, keys ^ np.uint32(7))
        rng = np.random.default_rng(22)
        ins = keys[rng.permutation(8000)[:3000]]  # second instances
        dl = np.setdiff1d(keys, ins)[:2000]
        srch = np.concatenate([np.setdiff1d(keys, np.concatenate([ins, dl]))[:2000], ks.take(1000)])
        ops = np.concatenate([np.zeros(3000, np.uint8), np.ones(2000, np.uint8), np.full(3000, 2, np.uint8)])
        kk = np.concatenate([ins, dl, srch])
        vv = np.concatenate([ins ^ np.uint32(7), np.zeros(5000, np.uint32)])
        perm = rng.permutation(len(kk))
        r, f = p.mixed(ops[perm], kk[perm], vv[perm])
        assert (r[ops[perm] == 0] == 1).all() and (f[ops[perm] == 0] == 0).all()
        p.check_structure(allow_holes=True, slabs_fixed=False)
    finally:
        p.close()


def test_set_table_search_all_delete_all():
    """In a set table SEARCHALL finds at most one instance (SEARCH's) and DELETEALL
    does what DELETE does; reserved keys count nothing and raise the flag."""
    w = W.bulk_workload(1 << 14, 0.6, 1 << 14, 0.5, 0, seed=8)
    p = Pair(w.num_buckets, w.hash_a, w.hash_b, n_hint=1 << 14)
    try:
        p.insert(w.keys, w.values)
        c, v = _search_all(p, w.search.keys, 2)
        vo, fo = p.o.search(w.search.keys)
        assert (c == fo).all() and (v[fo == 1, 0] == vo[fo == 1]).all() and (v[:, 1] == 0xFFFFFFFF).all()
        d = _delete_all(p, w.keys[::2])
        assert (d == p.o.delete_all(w.keys[::2])).all() and (d == 1).all()
        p.check_structure()
        _delete_all(p, np.array([0xFFFFFFFE, 5], np.uint32))
        p.o.delete_all(np.array([0xFFFFFFFE, 5], np.uint32))
        rc, flags = p.g.status()
        assert flags == sh.SLAB_FLAG_RESERVED_KEY
    finally:
        p.close()


def test_multiset_only_on_empty_tables():
    t = sh.SlabHash(64, 3, 4, 1024)
    try:
        t.insert(dev(np.arange(10, dtype=np.uint32)), dev(np.arange(10, dtype=np.uint32)))
        with pytest.raises(sh.SlabError):
            sh.slab_set_multiset(t.handle)
        t.reset()
        sh.slab_set_multiset(t.handle)
        sh.slab_set_multiset(t.handle, False)
    finally:
        t.close()


@pytest.mark.parametrize("variant", list(VARIANTS))
def test_grow_pool_keeps_the_table(variant):
    """A pool grown between batches keeps every slab address and allocation; lists
    then grow into the new blocks, and everything agrees with the oracle."""
    n = 40000
    w = W.bulk_workload(n, 2.5, n, 0.5, 0, seed=13)
    p = Pair(w.num_buckets, w.hash_a, w.hash_b, pool_slabs=1024, variant=variant)
    try:
        half = n // 4
        p.insert(w.keys[:half], w.values[:half])
        before = p.check_structure()
        assert before["pool_allocated"] > 0
        sh.slab_grow_pool(p.g.handle, 5000)
        info = sh.slab_get_info(p.g.handle)
        assert info.pool_slabs == 6 * 1024 and info.num_memory_blocks == 6
        assert p.check_structure() == before
        p.insert(w.keys[half:], w.values[half:])
        tot = p.check_structure()
        assert tot["pool_allocated"] > 1024
        p.search(w.search.keys)
        with pytest.raises(sh.SlabError):
            sh.slab_grow_pool(p.g.handle, 0)
    finally:
        p.close()
