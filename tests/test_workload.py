"""Host-side input generators: the serving trace keeps every mutated key private to
one request, so any interleaving of its requests gives the same per-op results."""
import numpy as np

from paper_1710_11246_gb300 import workload as W


def test_request_sizes_log_uniform():
    rng = np.random.default_rng(0)
    s = W.request_sizes(200000, 1 << 16, rng)
    assert s.min() == 1 and s.max() <= 1 << 16
    # log-uniform: each octave [2^j, 2^(j+1)) holds about 1/16 of the draws
    octave = np.floor(np.log2(s)).astype(int)
    frac = np.bincount(octave, minlength=17)[:16] / len(s)
    assert np.allclose(frac, 1 / 16, atol=0.01), frac


def test_serving_trace_structure():
    tr = W.serving_trace(1 << 14, 400, 1e5, max_size=1 << 10, seed=3)
    sizes = np.diff(tr.op_start.astype(np.int64))
    assert tr.op_start[0] == 0 and (sizes >= 1).all() and (sizes <= 1 << 10).all()
    assert len(tr.ops) == len(tr.keys) == len(tr.values) == tr.op_start[-1]
    assert (np.diff(tr.arrival_ns.astype(np.int64)) >= 0).all()
    frac = np.bincount(tr.ops, minlength=3) / len(tr.ops)
    assert np.allclose(frac, [0.1, 0.1, 0.8], atol=0.01)
    ins, dele, srch = tr.ops == W.OP_INSERT, tr.ops == W.OP_DELETE, tr.ops == W.OP_SEARCH
    # mutated keys: distinct across the whole trace and never searched
    mut = tr.keys[ins | dele]
    assert len(np.unique(mut)) == len(mut)
    assert not np.isin(tr.keys[srch], mut).any()
    assert not np.isin(tr.keys[ins], tr.preload).any() and np.isin(tr.keys[dele], tr.preload).all()
    # within one request every key appears once
    for r in range(len(sizes)):
        k = tr.keys[tr.op_start[r]:tr.op_start[r + 1]]
        assert len(np.unique(k)) == len(k)
    # values: key ^ constant for inserts, zero elsewhere
    assert (tr.values[ins] == W.values_for(tr.keys[ins])).all() and (tr.values[~ins] == 0).all()
    # about half the searches hit the loaded keys
    hit = np.isin(tr.keys[srch], tr.preload).mean()
    assert abs(hit - 0.5) < 0.02


def test_serving_trace_rate_changes_arrivals_only():
    a = W.serving_trace(1 << 12, 50, None, max_size=256, seed=1)
    b = W.serving_trace(1 << 12, 50, 1e4, max_size=256, seed=1)
    assert (a.arrival_ns == 0).all() and b.arrival_ns[-1] > 0
    for f in ("op_start", "ops", "keys", "values", "preload"):
        assert (getattr(a, f) == getattr(b, f)).all()
    # Poisson: mean gap near 1 / rate
    c = W.serving_trace(1 << 12, 4000, 1e4, max_size=4, seed=2)
    gaps = np.diff(np.concatenate([[0], c.arrival_ns.astype(np.int64)]))
    assert abs(gaps.mean() / 1e5 - 1) < 0.05


def test_mixed_batch_keys_once_each_and_the_live_set_follows():
    """Concurrent-benchmark batches (Sec. 6.3): every key appears in at most one op of
    a batch, so every outcome is fixed; inserts take fresh keys, deletes take live
    keys, half of the searches hit live keys that the batch does not delete, the
    op counts follow the ratios, no key is a sentinel, and the returned live set
    is the old one minus the deletes plus the inserts."""
    for ratios in W.CONFIG3_RATIOS:
        ks = W.KeyStream(11)
        live = ks.take(50000)
        rng = np.random.default_rng(11)
        for _ in range(3):
            n = 20000
            mb, new_live = W.mixed_batch(ks, live, n, ratios, rng)
            assert len(mb.keys) == len(mb.ops) == len(mb.values) == n
            assert len(np.unique(mb.keys)) == n
            assert (mb.keys < 0xFFFFFFFE).all()
            ins = mb.keys[mb.ops == W.OP_INSERT]
            dels = mb.keys[mb.ops == W.OP_DELETE]
            srch = mb.keys[mb.ops == W.OP_SEARCH]
            assert len(ins) == round(n * ratios[0]) and len(dels) == round(n * ratios[1])
            assert not np.isin(ins, live).any() and np.isin(dels, live).all()
            hits = np.isin(srch, live)
            assert hits.sum() == len(srch) // 2 and not np.isin(srch[hits], dels).any()
            assert (mb.values[mb.ops == W.OP_INSERT] == W.values_for(ins)).all()
            assert (mb.values[mb.ops != W.OP_INSERT] == 0).all()
            want = np.union1d(np.setdiff1d(live, dels), ins)
            assert len(new_live) == len(want) and (np.sort(new_live) == want).all()
            live = new_live


def test_bulk_workload_shapes():
    """The bulk benchmark's inputs (Sec. 6.1) at the small size: distinct
    non-sentinel keys, value = key XOR the fixed constant, B = ceil(n / (15 beta)),
    searches whose `present` flags are exactly membership in the stored keys at
    the stated hit rate, and distinct deletes of stored keys."""
    w = W.config1()
    n = len(w.keys)
    assert n == 1 << 16 and len(np.unique(w.keys)) == n and (w.keys < 0xFFFFFFFE).all()
    assert (w.values == (w.keys ^ np.uint32(0x9E3779B9))).all()
    assert w.num_buckets == int(np.ceil(n / (15 * 0.6))) == 7282
    q = w.search.keys
    assert len(q) == 1 << 16 and (w.search.present == np.isin(q, w.keys)).all()
    assert w.search.present.sum() == len(q) // 2 and len(np.unique(q)) == len(q)
    d = w.delete_keys
    assert len(d) == 1 << 14 and len(np.unique(d)) == len(d) and np.isin(d, w.keys).all()
