"""Serving loop (continuous batching on one resident table) vs the oracle.

Traces keep every mutated key private to one request, so each request's results
are independent of what runs beside it: the oracle applies the served requests
one after another and must agree op by op with the concurrent run, and each
request replayed alone on a freshly loaded table must give the same bits."""
import numpy as np
import pytest
import torch

from paper_1710_11246_gb300 import slabhash as sh
from paper_1710_11246_gb300 import workload as W
from tests.gpu_helpers import Pair, dev

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _lib():
    sh.load_library()


def _loaded_pair(tr, pool_slabs=None):
    p = Pair(tr.num_buckets, tr.hash_a, tr.hash_b, pool_slabs=pool_slabs, n_hint=len(tr.preload) * 2)
    p.insert(tr.preload, W.values_for(tr.preload))
    torch.cuda.synchronize()
    return p


def _served_ops(tr, served):
    idx = np.concatenate([np.arange(tr.op_start[r], tr.op_start[r + 1]) for r in np.flatnonzero(served)] or
                         [np.empty(0, np.int64)]).astype(np.int64)
    return idx


def _check_against_oracle(p, tr, out, served):
    idx = _served_ops(tr, served)
    ro, fo = p.o.mixed(tr.ops[idx], tr.keys[idx], tr.values[idx])
    assert (out["found"][idx] == fo).all(), np.flatnonzero(out["found"][idx] != fo)[:8]
    assert (out["results"][idx] == ro).all(), np.flatnonzero(out["results"][idx] != ro)[:8]
    p.check_structure()


@pytest.mark.parametrize("slots,rate,capacity,pinned,zero_copy", [
    (1, None, 1 << 12, False, False), (4, None, 1 << 14, False, False), (8, 2e5, 1 << 14, False, False),
    (4, None, 1 << 15, True, False), (2, 5e4, 1 << 12, True, False), (4, None, 1 << 15, True, True),
    (8, 2e5, 1 << 14, True, True), (3, None, 1 << 14, False, True)])
def test_trace_matches_oracle(slots, rate, capacity, pinned, zero_copy):
    """Continuous batching over a trace, from pageable or page-locked host arrays,
    copied (staged or DMA) or read in place (zero-copy): every request's results
    equal the oracle's serial run of the trace."""
    tr = W.serving_trace(1 << 16, 300, rate, max_size=1 << 12, seed=slots)
    p = _loaded_pair(tr)
    sv = sh.slab_server_create(p.g.handle, slots, capacity, flags=sh.SLAB_SERVER_ZERO_COPY if zero_copy else 0)
    arrays = [tr.ops, tr.keys, tr.values]
    if pinned:
        arrays = [sh.pinned_copy(a) for a in arrays]
    try:
        out = sh.slab_server_run(sv, tr.arrival_ns, tr.op_start, *arrays, pinned_outputs=pinned)
        assert (out["status"] == sh.SLAB_OK).all()
        lat, wait = out["latency_ns"].astype(np.int64), out["wait_ns"].astype(np.int64)
        assert (lat >= wait).all() and (wait >= 0).all() and (lat > 0).all()
        assert out["makespan_ns"] == int((tr.arrival_ns + out["latency_ns"]).max())
        st = sh.slab_server_get_stats(sv)
        assert st["submitted"] == st["completed"] == 300 and st["inflight"] == 0 and st["pool_reserved"] == 0
        assert 1 <= st["batches"] <= 300
        if rate is None and capacity > 1 << 12:
            assert st["batches"] < 300  # queued requests share launches
        _check_against_oracle(p, tr, out, np.ones(300, bool))
        # the largest count a batch reported bounds the final allocation from above
        # (a count may land while another batch holds a slab it frees after losing
        # an append race)
        tot = p.g.stats()
        assert st["pool_measured"] >= tot["pool_allocated"]
    finally:
        sh.slab_server_destroy(sv)
        p.close()


@pytest.mark.parametrize("zero_copy", [False, True])
def test_key_only_table_serving(zero_copy):
    """A key-only table behind the server: values are ignored, results are the
    key-only ones (search 0 / NOT_FOUND, insert and delete 1 / 0), all equal to the
    oracle's."""
    tr = W.serving_trace(1 << 15, 150, None, max_size=1 << 11, seed=33)
    p = Pair(tr.num_buckets, tr.hash_a, tr.hash_b, key_only=True, n_hint=1 << 16)
    p.insert(tr.preload)
    arrays = [sh.pinned_copy(tr.ops), sh.pinned_copy(tr.keys), None]
    sv = sh.slab_server_create(p.g.handle, 4, 1 << 13, flags=sh.SLAB_SERVER_ZERO_COPY if zero_copy else 0)
    try:
        out = sh.slab_server_run(sv, tr.arrival_ns, tr.op_start, *arrays, pinned_outputs=zero_copy)
        assert (out["status"] == sh.SLAB_OK).all()
        ro, fo = p.o.mixed(tr.ops, tr.keys, None)
        assert (out["results"] == ro).all() and (out["found"] == fo).all()
        p.check_structure()
    finally:
        sh.slab_server_destroy(sv)
        p.close()


def test_each_request_same_alone_and_in_the_mix():
    """Results of requests served eight at a time equal, bit for bit, the results
    of the same requests each run alone on a freshly loaded table."""
    tr = W.serving_trace(1 << 16, 200, None, max_size=1 << 12, seed=21)
    p = _loaded_pair(tr)
    sv = sh.slab_server_create(p.g.handle, 8, 1 << 12)
    try:
        mix = sh.slab_server_run(sv, tr.arrival_ns, tr.op_start, tr.ops, tr.keys, tr.values)
    finally:
        sh.slab_server_destroy(sv)
    p.close()
    sizes = np.diff(tr.op_start)
    picks = [int(np.argmax(sizes)), int(np.argmin(sizes))] + list(np.random.default_rng(0).choice(200, 6, replace=False))
    for r in picks:
        a, b = int(tr.op_start[r]), int(tr.op_start[r + 1])
        q = _loaded_pair(tr)
        sv = sh.slab_server_create(q.g.handle, 2, 1 << 12)
        try:
            rc, ticket = sh.slab_server_submit(sv, tr.ops[a:b], tr.keys[a:b], tr.values[a:b])
            assert rc == sh.SLAB_OK
            res, found = sh.slab_server_collect(sv, ticket, b - a)
            assert (res == mix["results"][a:b]).all() and (found == mix["found"][a:b]).all(), r
        finally:
            sh.slab_server_destroy(sv)
            q.close()


def test_admission_by_free_pool_memory():
    """A pool that cannot take every insert of the trace: requests whose inserts
    would not fit are held back while others run and refused once nothing runs;
    no op ever finds the pool empty, and the served requests agree with the oracle."""
    tr = W.serving_trace(1 << 16, 200, None, ratios=(0.6, 0.1, 0.3), max_size=1 << 12, seed=5)
    # slabs the preload needs, and what serving every request would need (oracle)
    from oracle import OracleTable
    o = OracleTable(tr.num_buckets, tr.hash_a, tr.hash_b)
    o.insert(tr.preload, W.values_for(tr.preload))
    base = o.stats()[2]["slabs"] - tr.num_buckets
    o.mixed(tr.ops, tr.keys, tr.values)
    need_all = o.stats()[2]["slabs"] - tr.num_buckets
    o.close()
    pool = 1024 * max(1, (base + need_all) // 2048)  # a whole number of memory blocks
    assert base < 0.95 * pool < need_all
    p = _loaded_pair(tr, pool_slabs=pool)
    assert p.g.info.pool_slabs == pool
    sv = sh.slab_server_create(p.g.handle, 8, 1 << 12, pool_high_water=0.95)
    try:
        out = sh.slab_server_run(sv, tr.arrival_ns, tr.op_start, tr.ops, tr.keys, tr.values)
        st = sh.slab_server_get_stats(sv)
        served = out["status"] == sh.SLAB_OK
        assert (served | (out["status"] == sh.SLAB_ERR_OUT_OF_SLABS)).all()
        assert st["rejected_memory"] == int((~served).sum()) > 0
        # a refused request touched nothing, so the oracle sees only the served ones
        _check_against_oracle(p, tr, out, served)
        assert p.g.stats()["pool_allocated"] <= 0.95 * pool
    finally:
        sh.slab_server_destroy(sv)
        p.close()


def test_pool_grows_instead_of_refusing():
    """With SLAB_SERVER_GROW_POOL the same trace that overflowed the pool is served
    in full: the pool grows between batches, nothing is refused, and every request
    agrees with the oracle."""
    tr = W.serving_trace(1 << 16, 200, None, ratios=(0.6, 0.1, 0.3), max_size=1 << 12, seed=5)
    p = _loaded_pair(tr, pool_slabs=2048)
    sv = sh.slab_server_create(p.g.handle, 8, 1 << 12, pool_high_water=0.95, flags=sh.SLAB_SERVER_GROW_POOL)
    try:
        out = sh.slab_server_run(sv, tr.arrival_ns, tr.op_start, tr.ops, tr.keys, tr.values)
        st = sh.slab_server_get_stats(sv)
        assert (out["status"] == sh.SLAB_OK).all() and st["rejected_memory"] == 0
        assert st["pool_grown"] >= 1 and sh.slab_get_info(p.g.handle).pool_slabs > 2048
        _check_against_oracle(p, tr, out, np.ones(200, bool))
        # submit grows too, with nothing in flight
        big = np.arange(1, 40001, dtype=np.uint32) | np.uint32(1 << 30)
        before = sh.slab_get_info(p.g.handle).pool_slabs
        rc, ticket = sh.slab_server_submit(sv, np.zeros(4000, np.uint8), big[:4000], big[:4000])
        assert rc == sh.SLAB_OK
        sh.slab_server_collect(sv, ticket, 4000)
        assert sh.slab_get_info(p.g.handle).pool_slabs >= before
    finally:
        sh.slab_server_destroy(sv)
        p.close()


def test_submit_collect_slots_and_errors():
    tr = W.serving_trace(1 << 12, 4, None, max_size=300, seed=9)
    p = _loaded_pair(tr)
    sv = sh.slab_server_create(p.g.handle, 2, 300)
    try:
        seg = [(int(tr.op_start[r]), int(tr.op_start[r + 1])) for r in range(4)]
        tickets = []
        for a, b in seg[:2]:
            rc, t = sh.slab_server_submit(sv, tr.ops[a:b], tr.keys[a:b], tr.values[a:b])
            assert rc == sh.SLAB_OK
            tickets.append(t)
        a, b = seg[2]
        rc, t = sh.slab_server_submit(sv, tr.ops[a:b], tr.keys[a:b], tr.values[a:b])
        assert rc == sh.SLAB_ERR_BUSY and t == 0
        assert sh.slab_server_get_stats(sv)["deferred_slot"] == 1
        # run refuses while tickets are out
        with pytest.raises(sh.SlabError):
            sh.slab_server_run(sv, tr.arrival_ns, tr.op_start, tr.ops, tr.keys, tr.values)
        outs = [sh.slab_server_collect(sv, t, b - a) for t, (a, b) in zip(tickets, seg)]
        with pytest.raises(sh.SlabError):
            sh.slab_server_collect(sv, tickets[0], 1)  # already collected
        with pytest.raises(sh.SlabError):  # more ops than a slot holds
            sh.slab_server_submit(sv, np.zeros(301, np.uint8), np.arange(301, dtype=np.uint32),
                                  np.zeros(301, np.uint32))
        ro, fo = p.o.mixed(tr.ops[: seg[1][1]], tr.keys[: seg[1][1]], tr.values[: seg[1][1]])
        got_r = np.concatenate([o[0] for o in outs])
        got_f = np.concatenate([o[1] for o in outs])
        assert (got_r == ro).all() and (got_f == fo).all()
        p.check_structure()
    finally:
        sh.slab_server_destroy(sv)
        p.close()


def test_full_size_serving_table_sampled():
    """The serving workload's table (2^26 pairs) under a Poisson trace of
    log-uniform 1..2^16-op requests: every request served, and 64 sampled
    requests checked op by op against the oracle's table loaded the same way
    (no other request touches their keys, so the loaded state decides them)."""
    from oracle import OracleTable
    n = 1 << 26
    tr = W.serving_trace(n, 256, 5e4, seed=2)
    B = tr.num_buckets
    t = sh.SlabHash(B, tr.hash_a, tr.hash_b, 1 << 22)
    sv = None
    try:
        t.insert(dev(tr.preload), dev(W.values_for(tr.preload)))
        sv = sh.slab_server_create(t.handle, 8, 1 << 16)
        out = sh.slab_server_run(sv, tr.arrival_ns, tr.op_start, tr.ops, tr.keys, tr.values)
        assert (out["status"] == sh.SLAB_OK).all()
        rc, flags = t.status()
        assert rc == sh.SLAB_OK and flags == 0
        tot = t.stats()
        n_ins = int((tr.ops == W.OP_INSERT).sum())
        n_del = int((tr.ops == W.OP_DELETE).sum())
        assert tot["live"] == n + n_ins - n_del and tot["prefix_violations"] == 0
    finally:
        if sv:
            sh.slab_server_destroy(sv)
        t.close()
    o = OracleTable(B, tr.hash_a, tr.hash_b)
    try:
        o.insert(tr.preload, W.values_for(tr.preload))
        picks = np.sort(np.random.default_rng(1).choice(256, 64, replace=False))
        idx = np.concatenate([np.arange(tr.op_start[r], tr.op_start[r + 1]) for r in picks]).astype(np.int64)
        ro, fo = o.mixed(tr.ops[idx], tr.keys[idx], tr.values[idx])
        assert (out["found"][idx] == fo).all() and (out["results"][idx] == ro).all()
    finally:
        o.close()
