"""slab_chain_histogram_noalloc: the statistics entry point that allocates no device memory.

It exists for callers that cannot call cudaMalloc when they need table statistics
(with the device memory held by another allocator, or on a path that cannot take
an allocation's synchronization). Its counters live in a fixed device array
compiled into the library. These checks compare it, through the C ABI, with the
allocating path (slab_stats per-bucket slab counts binned on the host) on two
calls in a row, so a second call must not see the first call's counts; check that
repeated calls leave the device's free memory unchanged; and check that a
capturing stream is refused without breaking the capture. The file is named to
be collected last.
"""
import numpy as np
import pytest

from paper_1710_11246_gb300 import slabhash as sh
from paper_1710_11246_gb300 import workload as W
from tests.gpu_helpers import dev, host

pytestmark = pytest.mark.gpu


def _table(num_buckets, n, seed, pool):
    keys = W.KeyStream(seed).take(n)
    a, b = W.hash_params(seed)
    t = sh.SlabHash(num_buckets, a, b, pool)
    t.insert(dev(keys), dev(W.values_for(keys)))
    t.delete(dev(keys[::5]))
    return t


@pytest.mark.parametrize("num_buckets,n,n_bins", [
    (W.buckets_for(1 << 16, 0.6), 1 << 16, 8),     # short lists, several bins
    (W.buckets_for(1 << 16, 2.0), 1 << 16, 3),     # lists longer than the last bin
    (1, 600, 1024),                                 # one 40-slab list, widest histogram
])
def test_noalloc_histogram_matches_stats(num_buckets, n, n_bins):
    t = _table(num_buckets, n, seed=n_bins, pool=1 << 14)
    try:
        _, slabs, tot = t.stats(per_bucket=True)
        per_bucket = host(slabs).astype(np.int64)
        want = np.bincount(np.minimum(per_bucket, n_bins) - 1, minlength=n_bins).astype(np.uint64)
        for _ in range(2):  # the array keeps the last call's counts; each call must clear it
            hist, totals = sh.slab_chain_histogram_noalloc(t.handle, n_bins)
            assert (hist == want).all(), (hist[:8], want[:8])
            assert totals == tot
            assert int(hist.sum()) == num_buckets
    finally:
        t.close()


def test_noalloc_histogram_rejects_too_many_bins():
    t = _table(64, 1000, seed=3, pool=1024)
    try:
        with pytest.raises(sh.SlabError) as e:
            sh.slab_chain_histogram_noalloc(t.handle, 1025)
        assert e.value.rc == sh.SLAB_ERR_INVALID_ARG
        with pytest.raises(sh.SlabError):
            sh.slab_chain_histogram_noalloc(t.handle, 0)
        hist, _ = sh.slab_chain_histogram_noalloc(t.handle, 1024)  # the limit itself is accepted
        assert int(hist.sum()) == 64
    finally:
        t.close()


def test_noalloc_histogram_takes_no_device_memory():
    """The property the entry point exists for: after one call, further calls leave
    the device's free memory exactly where it was."""
    import torch
    t = _table(W.buckets_for(1 << 14, 0.6), 1 << 14, seed=5, pool=1 << 12)
    try:
        sh.slab_chain_histogram_noalloc(t.handle, 16)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        for _ in range(20):
            sh.slab_chain_histogram_noalloc(t.handle, 16)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, (free0, free1)
    finally:
        t.close()


def test_noalloc_histogram_refuses_a_capturing_stream():
    """Inside stream capture the call returns SLAB_ERR_INVALID_ARG without enqueueing
    anything, and the capture still ends and replays."""
    import torch
    t = _table(64, 1000, seed=7, pool=1024)
    try:
        x = torch.zeros(4, device="cuda")
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            x.add_(1)
            with pytest.raises(sh.SlabError) as e:
                sh.slab_chain_histogram_noalloc(t.handle, 8, stream=s)
            assert e.value.rc == sh.SLAB_ERR_INVALID_ARG
        g.replay()
        torch.cuda.synchronize()
        assert x.tolist() == [1.0] * 4
        hist, _ = sh.slab_chain_histogram_noalloc(t.handle, 8)  # usable again outside capture
        assert int(hist.sum()) == 64
    finally:
        t.close()
