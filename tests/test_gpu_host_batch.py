"""slab_batch_host: batches whose arrays live in host memory, through the C ABI,
against the oracle and against the device-array calls: page-locked and pageable
arrays, one chunk and many (ragged last chunk), both modes and both slab widths,
the completion event, and the argument checks."""
import numpy as np
import pytest
import torch

from oracle import OracleTable
from paper_1710_11246_gb300 import slabhash as sh
from paper_1710_11246_gb300 import workload as W

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _lib():
    sh.load_library()


def _host(a, pinned):
    t = torch.from_numpy(np.ascontiguousarray(a).view(np.int32 if a.dtype == np.uint32 else a.dtype))
    return t.pin_memory() if pinned else t.clone()


def _u32(t):
    return t.numpy().view(np.uint32)


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("chunk", [0, 999])
@pytest.mark.parametrize("key_only,slab_bytes", [(False, 128), (True, 128), (False, 64)])
def test_host_batches_match_the_oracle(pinned, chunk, key_only, slab_bytes):
    per = (slab_bytes // 4 - 2) // (1 if key_only else 2)
    w = W.bulk_workload(20000, 0.8, 20000, 0.5, 5000, seed=6, per_slab=per)
    mode = sh.SLAB_MODE_KEY_ONLY if key_only else sh.SLAB_MODE_KEY_VALUE
    t = sh.SlabHash(w.num_buckets, w.hash_a, w.hash_b, 1 << 14, mode=mode, slab_bytes=slab_bytes)
    o = OracleTable(w.num_buckets, w.hash_a, w.hash_b, key_only=key_only, slab_bytes=slab_bytes)
    s = torch.cuda.Stream()
    try:
        n, q = len(w.keys), len(w.search.keys)
        kf = _host(np.zeros(n, np.uint8), pinned)
        sh.slab_batch_host(t.handle, sh.SLAB_BATCH_INSERT, _host(w.keys, pinned),
                           values=None if key_only else _host(w.values, pinned), found=kf, chunk=chunk, stream=s)
        s.synchronize()
        assert (kf.numpy() == o.insert(w.keys, None if key_only else w.values)).all()
        res = _host(np.zeros(q, np.uint32), pinned)
        fnd = _host(np.zeros(q, np.uint8), pinned)
        ev = torch.cuda.Event()
        sh.slab_batch_host(t.handle, sh.SLAB_BATCH_SEARCH, _host(w.search.keys, pinned), results=res, found=fnd,
                           chunk=chunk, stream=s, done_event=ev)
        ev.synchronize()
        vo, fo = o.search(w.search.keys)
        assert (_u32(res) == vo).all() and (fnd.numpy() == fo).all()
        df = _host(np.zeros(len(w.delete_keys), np.uint8), pinned)
        sh.slab_batch_host(t.handle, sh.SLAB_BATCH_DELETE, _host(w.delete_keys, pinned), found=df, chunk=chunk,
                           stream=s)
        s.synchronize()
        assert (df.numpy() == o.delete(w.delete_keys)).all()
        live = np.setdiff1d(w.keys, w.delete_keys)
        mb, _ = W.mixed_batch(W.KeyStream(77), live, 7777, (0.2, 0.2, 0.6), np.random.default_rng(7))
        mr = _host(np.zeros(len(mb.keys), np.uint32), pinned)
        mf = _host(np.zeros(len(mb.keys), np.uint8), pinned)
        sh.slab_batch_host(t.handle, sh.SLAB_BATCH_MIXED, _host(mb.keys, pinned), ops=_host(mb.ops, pinned),
                           values=_host(mb.values, pinned), results=mr, found=mf, chunk=chunk, stream=s)
        s.synchronize()
        ro, fo = o.mixed(mb.ops, mb.keys, None if key_only else mb.values)
        assert (_u32(mr) == ro).all() and (mf.numpy() == fo).all()
        rc, flags = t.status()
        assert flags == 0
        tot = t.stats()
        assert tot["live"] == o.stats()[2]["live"] and tot["prefix_violations"] == 0
    finally:
        t.close()
        o.close()


def test_host_batch_overlaps_and_equals_the_device_path():
    """Back-to-back host batches with completion events, the stream never waiting on
    the copies back: the final host results equal the device-array path's."""
    w = W.config2(0.6, 0.5, seed=2)
    t = sh.SlabHash(w.num_buckets, w.hash_a, w.hash_b, 1 << 20)
    s = torch.cuda.Stream()
    try:
        hk, hv, hq = _host(w.keys, True), _host(w.values, True), _host(w.search.keys, True)
        res = _host(np.zeros(len(w.search.keys), np.uint32), True)
        fnd = _host(np.zeros(len(w.search.keys), np.uint8), True)
        evs = []
        for _ in range(3):
            sh.slab_reset(t.handle, s)
            sh.slab_batch_host(t.handle, sh.SLAB_BATCH_INSERT, hk, values=hv, stream=s)
            ev = torch.cuda.Event()
            sh.slab_batch_host(t.handle, sh.SLAB_BATCH_SEARCH, hq, results=res, found=fnd, stream=s, done_event=ev)
            evs.append(ev)
        evs[-1].synchronize()
        dv = torch.empty(len(w.search.keys), dtype=torch.int32, device="cuda")
        df = torch.empty(len(w.search.keys), dtype=torch.uint8, device="cuda")
        sh.slab_search_batch(t.handle, sh.as_device_u32(w.search.keys), dv, df, stream=s)
        s.synchronize()
        assert (_u32(res) == sh.to_host_u32(dv)).all() and (fnd.numpy() == df.cpu().numpy()).all()
        assert int(fnd.numpy().sum()) == int(w.search.present.sum())
    finally:
        t.close()


def test_host_batch_argument_checks():
    t = sh.SlabHash(64, 3, 4, 1024)
    try:
        keys = np.arange(10, dtype=np.uint32)
        with pytest.raises(sh.SlabError):
            sh.slab_batch_host(t.handle, 7, keys)
        with pytest.raises(sh.SlabError):  # key-value inserts need values
            sh.slab_batch_host(t.handle, sh.SLAB_BATCH_INSERT, keys)
        with pytest.raises(sh.SlabError):  # a search needs somewhere to put values
            sh.slab_batch_host(t.handle, sh.SLAB_BATCH_SEARCH, keys)
        sh.slab_batch_host(t.handle, sh.SLAB_BATCH_SEARCH, keys[:0], results=keys[:0], n=0)  # n = 0: no-op
    finally:
        t.close()
