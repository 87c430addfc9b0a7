"""Tables of 64-byte slabs (slab_create_width) against the oracle at the same width.

A 64-byte slab keeps Sec. 4.2's layout at 16 words: 7 pairs (or 14 keys), the
auxiliary word and the next pointer; the staged kernels serve two ops per warp
step on half-warps. Every test compares results, found flags, per-bucket slot
and slab counts and the exported table with an oracle of M = 7 (or 14) element
by element, through the C ABI.
"""
import numpy as np
import pytest
import torch

from paper_1710_11246_gb300 import slabhash as sh
from paper_1710_11246_gb300 import workload as W
from tests.gpu_helpers import Pair, dev, host, u8

pytestmark = pytest.mark.gpu

M64 = 7  # pairs per 64-byte slab


@pytest.fixture(autouse=True, scope="module")
def _lib():
    sh.load_library()


def _pair(B, a, b, **kw):
    return Pair(B, a, b, slab_bytes=64, **kw)


def test_info_reports_the_width():
    t = sh.SlabHash(100, 3, 4, 1024, slab_bytes=64)
    k = sh.SlabHash(100, 3, 4, 1024, mode=sh.SLAB_MODE_KEY_ONLY, slab_bytes=64)
    try:
        assert t.info.slab_bytes == 64 and t.info.elements_per_slab == 7
        assert k.info.slab_bytes == 64 and k.info.elements_per_slab == 14
        assert t.info.device_bytes >= (100 + 1024) * 64
    finally:
        t.close()
        k.close()


@pytest.mark.parametrize("key_only", [False, True])
def test_small_workload(key_only):
    """2^16 pairs at beta 0.6 in 64-byte slabs, 2^16 searches at 50 % hit, 2^14 deletes."""
    per = 14 if key_only else M64
    w = W.bulk_workload(1 << 16, 0.6, 1 << 16, 0.5, 1 << 14, seed=0, per_slab=per)
    p = _pair(w.num_buckets, w.hash_a, w.hash_b, key_only=key_only, n_hint=len(w.keys))
    try:
        vals = None if key_only else w.values
        assert p.insert(w.keys, vals).sum() == 0
        p.check_structure()
        _, found = p.search(w.search.keys)
        assert (found.astype(bool) == w.search.present).all()
        assert p.delete(w.delete_keys).all()
        p.search(w.search.keys)
        p.insert(w.keys[:5000], vals[:5000] if vals is not None else None)  # replaces and re-inserts
        p.check_structure()
    finally:
        p.close()


@pytest.mark.parametrize("n", [0, 1, 31, 33, 1000, 4097])
def test_ragged_sizes(n):
    ks = W.KeyStream(n + 3)
    keys = ks.take(n)
    absent = ks.take(n)
    a, b = W.hash_params(n)
    for B in (1, 3, max(1, n // 4)):
        p = _pair(B, a, b, n_hint=n)
        try:
            p.insert(keys, W.values_for(keys))
            p.search(np.concatenate([keys, absent]))
            p.delete(keys[::2])
            p.search(keys)
            p.check_structure()
        finally:
            p.close()


@pytest.mark.parametrize("key_only", [False, True])
@pytest.mark.parametrize("B,n", [(1, 6), (1, 7), (1, 8), (1, 13), (1, 14), (1, 15), (1, 29), (1, 2000), (3, 46)])
def test_slab_boundaries_and_long_chains(key_only, B, n):
    keys = W.KeyStream(B * 1000 + n).take(n)
    p = _pair(B, 5, 9, key_only=key_only, n_hint=n)
    try:
        vals = None if key_only else W.values_for(keys)
        p.insert(keys, vals)
        p.search(keys)
        p.delete(keys[1::3])
        p.search(keys)
        p.insert(keys[: n // 2], vals[: n // 2] if vals is not None else None)
        p.check_structure()
    finally:
        p.close()


def test_mixed_batches():
    """Preload 2^16 pairs, then batches of 2^14 mixed ops in each concurrent-benchmark ratio."""
    ks = W.KeyStream(5)
    keys = ks.take(1 << 16)
    a, b = W.hash_params(5)
    p = _pair(W.buckets_for(1 << 16, 0.6, M64), a, b, n_hint=1 << 18)
    rng = np.random.default_rng(5)
    try:
        p.insert(keys, W.values_for(keys))
        live = keys
        for ratios in W.CONFIG3_RATIOS:
            for _ in range(3):
                mb, live = W.mixed_batch(ks, live, 1 << 14, ratios, rng)
                p.mixed(mb.ops, mb.keys, mb.values)
        p.search(live[:5000])
        p.check_structure()
    finally:
        p.close()


def test_repeated_keys_follow_a_serial_order():
    """A key repeated in one batch: one of its two inserts reports it new, the stored
    value is one of the two written, and keys stay unique."""
    ks = W.KeyStream(41)
    pre = ks.take(3000)
    new = ks.take(2000)
    p = _pair(W.buckets_for(5000, 0.6, M64), 17, 23, n_hint=8000)
    try:
        p.insert(pre, W.values_for(pre))
        v1, v2 = (new * np.uint32(3)).astype(np.uint32), (new * np.uint32(5)).astype(np.uint32)
        keys = np.concatenate([new, new]).astype(np.uint32)
        vals = np.concatenate([v1, v2]).astype(np.uint32)
        perm = np.random.default_rng(42).permutation(len(keys))
        fd = torch.empty(len(keys), dtype=torch.uint8, device="cuda")
        p.g.insert(dev(keys[perm]), dev(vals[perm]), fd)
        f = np.empty(len(keys), np.uint8)
        f[perm] = u8(fd)
        assert ((f[:2000] + f[2000:]) == 1).all()
        fd2 = torch.empty(2000, dtype=torch.uint8, device="cuda")
        now = host(p.g.search(dev(new), found=fd2))
        assert (u8(fd2) == 1).all() and ((now == v1) | (now == v2)).all()
        tot = p.g.stats()
        assert tot["live"] == 5000 and tot["prefix_violations"] == 0
    finally:
        p.close()


def test_pool_exhaustion_reports_and_stays_consistent():
    """One memory block (1024 64-byte slabs) cannot hold 2^14 pairs in one bucket."""
    keys = W.KeyStream(11).take(1 << 14)
    p = _pair(1, 5, 6, pool_slabs=1024, iter_limit=1 << 20)
    try:
        res = host(p.g.mixed(torch.zeros(len(keys), dtype=torch.uint8, device="cuda"), dev(keys),
                             dev(W.values_for(keys))))
        rc, flags = p.g.status()
        assert rc == sh.SLAB_ERR_OUT_OF_SLABS and flags & sh.SLAB_FLAG_OUT_OF_SLABS
        ok = res == 1
        assert 0 < ok.sum() <= M64 * 1025
        fd = torch.empty(len(keys), dtype=torch.uint8, device="cuda")
        v = host(p.g.search(dev(keys), found=fd))
        hit = u8(fd).astype(bool)
        assert (hit == ok).all() and (v[hit] == W.values_for(keys)[hit]).all()
        tot = p.g.stats()
        assert tot["live"] == ok.sum() and tot["prefix_violations"] == 0
        assert tot["pool_allocated"] == tot["linked"] and 1000 <= tot["linked"] <= 1024
    finally:
        p.close()


def test_iteration_cap_ends_ops_with_a_status():
    keys = W.KeyStream(12).take(64)
    p = _pair(1, 5, 6, iter_limit=1)
    try:
        p.g.insert(dev(keys), dev(W.values_for(keys)))
        rc, flags = p.g.status()
        assert rc == sh.SLAB_ERR_ITER_LIMIT and flags == sh.SLAB_FLAG_ITER_LIMIT
        tot = p.g.stats()
        assert tot["live"] < 64 and tot["prefix_violations"] == 0
    finally:
        p.close()


def test_reset_and_reuse():
    ks = W.KeyStream(8)
    keys = ks.take(20000)
    p = _pair(W.buckets_for(20000, 1.5, M64), 3, 5, n_hint=40000)
    try:
        p.insert(keys, W.values_for(keys))
        p.g.reset()
        p.o.close()
        from oracle import OracleTable
        p.o = OracleTable(p.B, 3, 5, slab_bytes=64)
        tot = p.g.stats()
        assert tot["live"] == 0 and tot["pool_allocated"] == 0
        more = ks.take(20000)
        p.insert(more, W.values_for(more))
        p.search(np.concatenate([keys[:5000], more[:5000]]))
        p.check_structure()
    finally:
        p.close()


@pytest.mark.parametrize("tpb,bps", [(32, 1), (256, 0), (512, 1)])
def test_launch_shapes(tpb, bps):
    w = W.bulk_workload(20000, 0.8, 20000, 0.5, 5000, seed=4, per_slab=M64)
    p = _pair(w.num_buckets, w.hash_a, w.hash_b, n_hint=20000, threads_per_block=tpb, blocks_per_sm=bps)
    try:
        p.insert(w.keys, w.values)
        p.search(w.search.keys)
        p.delete(w.delete_keys)
        p.check_structure()
    finally:
        p.close()


def test_unsupported_calls_are_refused():
    """64-byte tables run the staged kernels only; the paper-structured variant,
    multiset tables, SEARCHALL / DELETEALL and FLUSH are refused."""
    t = sh.SlabHash(64, 3, 4, 1024, slab_bytes=64)
    try:
        with pytest.raises(sh.SlabError):
            t.configure(variant=sh.SLAB_VARIANT_DIRECT)
        with pytest.raises(sh.SlabError):
            sh.slab_set_multiset(t.handle, 1)
        keys = dev(np.arange(10, dtype=np.uint32))
        counts = torch.empty(10, dtype=torch.int32, device="cuda")
        with pytest.raises(sh.SlabError):
            sh.slab_delete_all_batch(t.handle, keys, counts)
        with pytest.raises(sh.SlabError):
            sh.slab_flush(t.handle)
        with pytest.raises(sh.SlabError):
            sh.slab_create_width(64, sh.SLAB_MODE_KEY_VALUE, 96, 3, 4, 1024)
    finally:
        t.close()


def test_chain_histogram_noalloc_at_64_bytes():
    keys = W.KeyStream(3).take(1 << 14)
    p = _pair(W.buckets_for(1 << 14, 1.0, M64), 7, 9, n_hint=1 << 15)
    try:
        p.insert(keys, W.values_for(keys))
        _, slabs, tot = p.g.stats(per_bucket=True)
        per_bucket = host(slabs).astype(np.int64)
        want = np.bincount(np.minimum(per_bucket, 6) - 1, minlength=6).astype(np.uint64)
        hist, totals = sh.slab_chain_histogram_noalloc(p.g.handle, 6)
        assert (hist == want).all() and totals == tot
        _, oslabs, _ = p.o.stats()
        assert (per_bucket == oslabs).all()
    finally:
        p.close()


def test_full_size_step_matches_the_oracle():
    """2^22 pairs in 64-byte slabs at beta 0.6 (B = ceil(n / (7 beta))), 2^22
    searches at 50 % hit, 2^20 deletes and 2^20 mixed ops at (0.2, 0.2, 0.6), in the
    benchmark's launch configuration: every output and the final table agree."""
    w = W.config2(0.6, 0.5, seed=0, per_slab=M64)
    ks = W.KeyStream(0)
    ks.take(len(w.keys) + (len(w.search.keys) - int(round(len(w.search.keys) * 0.5))))
    rng = np.random.default_rng([0, 0x3333])
    live = np.setdiff1d(w.keys, w.delete_keys, assume_unique=True)
    mb, _ = W.mixed_batch(ks, live, 1 << 20, (0.2, 0.2, 0.6), rng)
    p = _pair(w.num_buckets, w.hash_a, w.hash_b, pool_slabs=1 << 21)
    try:
        assert p.insert(w.keys, w.values).sum() == 0
        _, found = p.search(w.search.keys)
        assert (found.astype(bool) == w.search.present).all()
        assert p.delete(w.delete_keys).all()
        p.mixed(mb.ops, mb.keys, mb.values)
        p.check_structure()
    finally:
        p.close()


def test_full_size_concurrent_batches_match_the_oracle():
    w = W.config2(0.6, 0.5, seed=3, per_slab=M64)
    ks = W.KeyStream(3)
    ks.take(len(w.keys) + len(w.search.keys))
    rng = np.random.default_rng(3)
    p = _pair(w.num_buckets, w.hash_a, w.hash_b, pool_slabs=1 << 22)
    try:
        assert p.insert(w.keys, w.values).sum() == 0
        live = w.keys
        for ratios in W.CONFIG3_RATIOS:
            mb, live = W.mixed_batch(ks, live, 1 << 20, ratios, rng)
            p.mixed(mb.ops, mb.keys, mb.values)
        p.search(live[: 1 << 20])
        p.check_structure()
    finally:
        p.close()


def test_group_of_64_byte_tables_matches_single_tables():
    """A group at 64-byte width against each table's own oracle."""
    from oracle import OracleTable
    gw = W.group_workload(40, 1 << 6, 1 << 12, seed=9, per_slab=M64)
    pools = np.full(40, 1 << 12, np.uint64)
    g = sh.slab_group_create(gw.num_buckets, gw.hash_a, gw.hash_b, pools, slab_bytes=64)
    try:
        start = dev(gw.op_start)
        fd = torch.empty(len(gw.keys), dtype=torch.uint8, device="cuda")
        sh.slab_group_insert(g, start, dev(gw.keys), dev(gw.values), fd)
        vals = torch.empty(len(gw.search_keys), dtype=torch.int32, device="cuda")
        sf = torch.empty(len(gw.search_keys), dtype=torch.uint8, device="cuda")
        sh.slab_group_search(g, dev(gw.search_start), dev(gw.search_keys), vals, sf)
        rc, flags = sh.slab_group_status(g)
        assert flags == 0
        gv, gf = host(vals), u8(sf)
        for i in range(40):
            lo, hi = int(gw.op_start[i]), int(gw.op_start[i + 1])
            o = OracleTable(int(gw.num_buckets[i]), int(gw.hash_a[i]), int(gw.hash_b[i]), slab_bytes=64)
            assert (o.insert(gw.keys[lo:hi], gw.values[lo:hi]) == u8(fd)[lo:hi]).all()
            ov, of = o.search(gw.search_keys[lo:hi])
            assert (ov == gv[lo:hi]).all() and (of == gf[lo:hi]).all()
            t = sh.slab_group_table(g, i)
            slabs = torch.empty(int(gw.num_buckets[i]), dtype=torch.int32, device="cuda")
            sh.slab_stats(t, None, slabs)
            _, oslabs, _ = o.stats()
            assert (host(slabs) == oslabs).all()
            o.close()
    finally:
        sh.slab_group_destroy(g)
