"""Groups of tables in one persistent launch vs per-table oracles and per-table launches."""
import numpy as np
import pytest
import torch

from oracle import OracleTable
from paper_1710_11246_gb300 import slabhash as sh
from paper_1710_11246_gb300 import workload as W
from tests.gpu_helpers import dev, host, u8

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _lib():
    sh.load_library()


def _group(w, pool_factor=4):
    pools = np.maximum(1024, pool_factor * w.sizes // 15 + 64).astype(np.uint64)
    return sh.slab_group_create(w.num_buckets, w.hash_a, w.hash_b, pools)


def _seg(a, start, i):
    return a[start[i]:start[i + 1]]


def test_group_parity_with_oracles():
    """Every table of a group, served by one launch per batch, agrees with its own
    oracle: insert flags, search values and flags, delete flags, mixed results,
    per-bucket slots and slabs."""
    sizes = np.array([0, 1, 5, 31, 32, 33, 200, 1000, 4097, 3, 0, 777, 15, 16, 2000, 64])
    w = W.group_workload(len(sizes), 1, 1, sizes=sizes, seed=3)
    g = _group(w)
    try:
        st = torch.from_numpy(w.op_start.view(np.int32)).cuda()
        fd = torch.full((len(w.keys),), 7, dtype=torch.uint8, device="cuda")
        sh.slab_group_insert(g, st, dev(w.keys), dev(w.values), fd)
        vo = torch.empty(len(w.search_keys), dtype=torch.int32, device="cuda")
        fs = torch.full((len(w.search_keys),), 7, dtype=torch.uint8, device="cuda")
        sh.slab_group_search(g, torch.from_numpy(w.search_start.view(np.int32)).cuda(), dev(w.search_keys), vo, fs)
        dels = [_seg(w.keys, w.op_start, i)[::3] for i in range(len(sizes))]
        dstart = np.concatenate([[0], np.cumsum([len(d) for d in dels])]).astype(np.uint32)
        dk = np.concatenate(dels).astype(np.uint32)
        fdel = torch.full((len(dk),), 7, dtype=torch.uint8, device="cuda")
        sh.slab_group_delete(g, torch.from_numpy(dstart.view(np.int32)).cuda(), dev(dk), fdel)
        rc, flags = sh.slab_group_status(g)
        assert rc == sh.SLAB_OK and flags == 0
        fd, vo, fs, fdel = u8(fd), host(vo), u8(fs), u8(fdel)
        for i in range(len(sizes)):
            o = OracleTable(int(w.num_buckets[i]), int(w.hash_a[i]), int(w.hash_b[i]))
            assert (_seg(fd, w.op_start, i) == o.insert(_seg(w.keys, w.op_start, i), _seg(w.values, w.op_start, i))).all()
            v, f = o.search(_seg(w.search_keys, w.search_start, i))
            assert (_seg(vo, w.search_start, i) == v).all() and (_seg(fs, w.search_start, i) == f).all()
            assert (_seg(fdel, dstart, i) == o.delete(dels[i])).all()
            t = sh.slab_group_table(g, i)
            slots = torch.empty(int(w.num_buckets[i]), dtype=torch.int32, device="cuda")
            slabs = torch.empty_like(slots)
            tot = sh.slab_stats(t, slots, slabs)
            os_, ob, otot = o.stats()
            assert (host(slots) == os_).all() and (host(slabs) == ob).all()
            assert tot["live"] == otot["live"] and tot["prefix_violations"] == 0
            assert tot["pool_allocated"] == tot["linked"]
    finally:
        sh.slab_group_destroy(g)


def test_group_equals_separate_tables_mixed():
    """A mixed batch through the group gives the same results as the same ops issued
    table by table through slab_create tables."""
    sizes = np.array([300, 64, 1500, 9, 0, 700])
    w = W.group_workload(len(sizes), 1, 1, sizes=sizes, seed=8)
    g = _group(w)
    singles = []
    try:
        st = torch.from_numpy(w.op_start.view(np.int32)).cuda()
        sh.slab_group_insert(g, st, dev(w.keys), dev(w.values))
        rng = np.random.default_rng(2)
        batches = []
        ks = W.KeyStream(77)
        for i in range(len(sizes)):
            live = _seg(w.keys, w.op_start, i)
            mb, _ = W.mixed_batch(ks, live, max(1, len(live) // 2), (0.3, 0.3, 0.4), rng) if len(live) else \
                (W.MixedBatch(np.empty(0, np.uint8), np.empty(0, np.uint32), np.empty(0, np.uint32)), None)
            batches.append(mb)
        mstart = np.concatenate([[0], np.cumsum([len(b.keys) for b in batches])]).astype(np.uint32)
        ops = np.concatenate([b.ops for b in batches]).astype(np.uint8)
        keys = np.concatenate([b.keys for b in batches]).astype(np.uint32)
        vals = np.concatenate([b.values for b in batches]).astype(np.uint32)
        res = torch.empty(len(keys), dtype=torch.int32, device="cuda")
        fnd = torch.empty(len(keys), dtype=torch.uint8, device="cuda")
        sh.slab_group_mixed(g, torch.from_numpy(mstart.view(np.int32)).cuda(), torch.from_numpy(ops).cuda(),
                            dev(keys), dev(vals), res, fnd)
        res, fnd = host(res), u8(fnd)
        for i in range(len(sizes)):
            t = sh.SlabHash(int(w.num_buckets[i]), int(w.hash_a[i]), int(w.hash_b[i]), 4096)
            singles.append(t)
            t.insert(dev(_seg(w.keys, w.op_start, i)), dev(_seg(w.values, w.op_start, i)))
            b = batches[i]
            if len(b.keys) == 0:
                continue
            f1 = torch.empty(len(b.keys), dtype=torch.uint8, device="cuda")
            r1 = host(t.mixed(torch.from_numpy(b.ops).cuda(), dev(b.keys), dev(b.values), found=f1))
            assert (r1 == _seg(res, mstart, i)).all() and (u8(f1) == _seg(fnd, mstart, i)).all()
    finally:
        for t in singles:
            t.close()
        sh.slab_group_destroy(g)


def test_group_in_cuda_graph():
    """reset + insert + search of a group captured once in a CUDA graph and replayed
    give the same results as the eager calls."""
    w = W.group_workload(40, 8, 4096, seed=12)
    g = _group(w)
    try:
        st = torch.from_numpy(w.op_start.view(np.int32)).cuda()
        qs = torch.from_numpy(w.search_start.view(np.int32)).cuda()
        k, v, q = dev(w.keys), dev(w.values), dev(w.search_keys)
        out = torch.empty(len(w.search_keys), dtype=torch.int32, device="cuda")
        fnd = torch.empty(len(w.search_keys), dtype=torch.uint8, device="cuda")
        sh.slab_group_reset(g)
        sh.slab_group_insert(g, st, k, v)
        sh.slab_group_search(g, qs, q, out, fnd)
        torch.cuda.synchronize()
        want_v, want_f = host(out).copy(), u8(fnd).copy()
        s = torch.cuda.Stream()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            sh.slab_group_reset(g, s)  # warm the launch paths outside the capture
            sh.slab_group_insert(g, st, k, v, stream=s)
            sh.slab_group_search(g, qs, q, out, fnd, stream=s)
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=s):
            sh.slab_group_reset(g, s)
            sh.slab_group_insert(g, st, k, v, stream=s)
            sh.slab_group_search(g, qs, q, out, fnd, stream=s)
        for _ in range(2):
            out.fill_(0)
            graph.replay()
            torch.cuda.synchronize()
            assert (host(out) == want_v).all() and (u8(fnd) == want_f).all()
        rc, _ = sh.slab_group_status(g)
        assert rc == sh.SLAB_OK
    finally:
        sh.slab_group_destroy(g)


def test_autotuner_searches_slab_width():
    """The autotuner times every (slab width, beta, launch shape) candidate on the
    group's own step and returns the fastest; the chosen configuration, rebuilt,
    still matches each table's oracle at its width."""
    from oracle import OracleTable
    from paper_1710_11246_gb300 import autotune as AT
    gw = W.group_workload(24, 1 << 6, 1 << 12, seed=12)
    best, cands = AT.tune_group(gw, betas=(0.6, 1.0), threads=(64, 128), blocks=(0,), widths=(128, 64), reps=1)
    assert {c.slab_bytes for c in cands} == {128, 64} and len(cands) == 8
    assert best.mops == max(c.mops for c in cands) and all(c.ms > 0 for c in cands)
    g = AT.create_group(gw, best.beta, best.slab_bytes)
    try:
        cfg = sh.slab_group_get_config(g)
        cfg.threads_per_block, cfg.blocks_per_sm = best.threads_per_block, best.blocks_per_sm
        sh.slab_group_set_config(g, cfg)
        st, k, v, qs, q = AT._arrays(gw, "cuda")
        out = torch.empty(len(gw.search_keys), dtype=torch.int32, device="cuda")
        fnd = torch.empty(len(gw.search_keys), dtype=torch.uint8, device="cuda")
        AT.group_step(g, (st, k, v, qs, q), out, fnd, None)
        torch.cuda.synchronize()
        gv, gf = sh.to_host_u32(out), fnd.cpu().numpy()
        per = (best.slab_bytes // 4 - 2) // 2
        for i in range(24):
            lo, hi = int(gw.op_start[i]), int(gw.op_start[i + 1])
            o = OracleTable(W.buckets_for(max(int(gw.sizes[i]), 1), best.beta, per), int(gw.hash_a[i]),
                            int(gw.hash_b[i]), slab_bytes=best.slab_bytes)
            o.insert(gw.keys[lo:hi], gw.values[lo:hi])
            ov, of = o.search(gw.search_keys[lo:hi])
            assert (ov == gv[lo:hi]).all() and (of == gf[lo:hi]).all()
            o.close()
    finally:
        sh.slab_group_destroy(g)
