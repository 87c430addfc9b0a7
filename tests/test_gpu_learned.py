"""Learned bucket function on the GPU vs the oracle's independent fit, bit for bit."""
import numpy as np
import pytest
import torch

from oracle import OracleTable, learn_model, learned_buckets
from paper_1710_11246_gb300 import slabhash as sh
from paper_1710_11246_gb300 import workload as W
from tests.gpu_helpers import VARIANTS, Pair, dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _lib():
    sh.load_library()


def _fit_both(keys, B, stride, policy=sh.SLAB_LEARN_ALWAYS, variant="staged", a=5, b=7, slab_bytes=128):
    p = Pair(B, a, b, variant=variant, n_hint=len(keys), slab_bytes=slab_bytes)
    rep = sh.slab_learn_buckets(p.g.handle, dev(keys), stride, policy)
    model_g, in_use = sh.slab_get_model(p.g.handle)
    model_o, m = learn_model(keys, stride, B)
    return p, rep, model_g, in_use, model_o, m


@pytest.mark.parametrize("n,stride", [(1 << 16, 100), (1 << 16, 1), (5000, 3), (1000, 1000), (1 << 12, 7)])
def test_model_bits_match_oracle_fit(n, stride):
    keys, _ = W.clustered_keys(n, seed=n + stride)
    B = W.buckets_for(n, 0.6)
    p, rep, model_g, in_use, model_o, m = _fit_both(keys, B, stride)
    try:
        assert rep["sample_size"] == m and in_use and rep["use_learned"] == 1
        assert model_g.view(np.uint32).tolist() == model_o.view(np.uint32).tolist(), \
            np.flatnonzero(model_g.view(np.uint32) != model_o.view(np.uint32))[:8]
        got = host(p.g.buckets_of(dev(keys)))
        want = learned_buckets(model_o, B, keys)
        assert (got == want).all(), np.flatnonzero(got != want)[:8]
    finally:
        p.close()


@pytest.mark.parametrize("variant", list(VARIANTS))
def test_learned_table_parity(variant):
    """A table on the learned model (GPU fit) agrees op by op with the oracle on its
    own fit: inserts, searches of present and absent clustered keys, deletes, mixed."""
    w = W.config4(seed=3, n=1 << 16)
    p, rep, model_g, _, model_o, _ = _fit_both(w.keys, w.num_buckets, 100, variant=variant)
    try:
        p.o.use_model(model_o)
        p.insert(w.keys, w.values)
        _, found = p.search(w.search.keys)
        assert (found.astype(bool) == w.search.present).all()
        p.delete(w.keys[::5])
        rng = np.random.default_rng(4)
        live = np.setdiff1d(w.keys, w.keys[::5])
        mb, _ = W.mixed_batch(W.KeyStream(99), live, 1 << 13, (0.2, 0.2, 0.6), rng)
        p.mixed(mb.ops, mb.keys, mb.values)
        p.check_structure()
    finally:
        p.close()


def test_learned_table_parity_at_64_bytes():
    """The learned bucket function on a table of 64-byte slabs: the GPU fit equals the
    oracle's, and every op and the table structure agree with an oracle of 7 pairs
    per slab on that model."""
    w = W.config4(seed=5, n=1 << 16, beta=0.6)
    B = W.buckets_for(len(w.keys), 0.6, 7)
    p, rep, model_g, _, model_o, _ = _fit_both(w.keys, B, 100, slab_bytes=64)
    try:
        assert model_g.view(np.uint32).tolist() == model_o.view(np.uint32).tolist()
        p.o.use_model(model_o)
        p.insert(w.keys, w.values)
        _, found = p.search(w.search.keys)
        assert (found.astype(bool) == w.search.present).all()
        p.delete(w.keys[::3])
        p.check_structure()
    finally:
        p.close()


def test_chain_report_matches_oracle_and_policy():
    """The reported mean / max slabs per bucket of both bucket functions equal the
    oracle's counts, and SLAB_LEARN_AUTO picks the model exactly when neither is worse."""
    n = 1 << 16
    keys, _ = W.clustered_keys(n, seed=11)
    B = W.buckets_for(n, 0.6)
    a, b = W.hash_params(11)
    for policy in (sh.SLAB_LEARN_AUTO, sh.SLAB_LEARN_MEASURE, sh.SLAB_LEARN_ALWAYS):
        p, rep, _, in_use, model_o, _ = _fit_both(keys, B, 100, policy=policy, a=a, b=b)
        try:
            ou = OracleTable(B, a, b)
            sum_u, max_u = ou.chain_profile(keys)
            ol = OracleTable(B, a, b)
            ol.use_model(model_o)
            sum_l, max_l = ol.chain_profile(keys)
            assert rep["max_slabs_universal"] == max_u and rep["max_slabs_learned"] == max_l
            assert rep["mean_slabs_universal"] == sum_u / B and rep["mean_slabs_learned"] == sum_l / B
            better = sum_l <= sum_u and max_l <= max_u
            want = {sh.SLAB_LEARN_AUTO: better, sh.SLAB_LEARN_MEASURE: False, sh.SLAB_LEARN_ALWAYS: True}[policy]
            assert bool(rep["use_learned"]) == want == in_use
            # buckets follow the chosen function
            got = host(p.g.buckets_of(dev(keys[:4096])))
            ref = ol if want else ou
            assert (got == ref.buckets(keys[:4096])).all()
        finally:
            p.close()


def test_fit_refused_on_a_table_holding_keys():
    keys, _ = W.clustered_keys(4096, seed=5)
    t = sh.SlabHash(300, 3, 4, 4096)
    try:
        t.insert(dev(keys), dev(W.values_for(keys)))
        with pytest.raises(sh.SlabError):
            sh.slab_learn_buckets(t.handle, dev(keys), 10)
        t.reset()
        rep = sh.slab_learn_buckets(t.handle, dev(keys), 10, sh.SLAB_LEARN_ALWAYS)
        assert rep["use_learned"] == 1
    finally:
        t.close()


def test_full_size_clustered_model_and_report():
    """2^22 clustered keys, 1 % sample: model bits, chain report and a 2^20-key slice of
    searches against the oracle."""
    w = W.config4(seed=0)
    B = w.num_buckets
    p, rep, model_g, _, model_o, m = _fit_both(w.keys, B, 100, policy=sh.SLAB_LEARN_AUTO, a=w.hash_a, b=w.hash_b)
    try:
        assert m == (len(w.keys) + 99) // 100
        assert model_g.view(np.uint32).tolist() == model_o.view(np.uint32).tolist()
        ou = OracleTable(B, w.hash_a, w.hash_b)
        sum_u, max_u = ou.chain_profile(w.keys)
        ol = OracleTable(B, w.hash_a, w.hash_b)
        ol.use_model(model_o)
        sum_l, max_l = ol.chain_profile(w.keys)
        assert (rep["max_slabs_learned"], rep["max_slabs_universal"]) == (max_l, max_u)
        if rep["use_learned"]:
            p.o.use_model(model_o)
        p.insert(w.keys, w.values)
        q = w.search.keys[: 1 << 20]
        p.search(q)
        tot = p.g.stats()
        assert tot["live"] == len(w.keys) and tot["prefix_violations"] == 0
    finally:
        p.close()


@pytest.mark.parametrize("n,stride,slab_bytes", [(1 << 26, 100, 128), (3 << 20, 3, 128), (1 << 20, 100, 64)])
def test_fit_scales_to_the_serving_table(n, stride, slab_bytes):
    """The multi-block sort and fit at the serving table's size (2^26 keys, a 1 %
    sample of 671,089 keys padded to 2^20), at the largest sample the call takes
    (2^20 keys: a 3 x 2^20-key set at stride 3) and on a 64-byte table: the model
    and its chain profile match the oracle's bit for bit."""
    keys = W.KeyStream(n + stride).take(n)
    B = W.buckets_for(n, 0.6, (slab_bytes // 4 - 2) // 2)
    t = sh.SlabHash(B, 5, 7, 1024, slab_bytes=slab_bytes)
    try:
        rep = sh.slab_learn_buckets(t.handle, dev(keys), stride, sh.SLAB_LEARN_MEASURE)
        model_g, in_use = sh.slab_get_model(t.handle)
        model_o, m = learn_model(keys, stride, B)
        assert rep["sample_size"] == m and not in_use
        assert model_g.view(np.uint32).tolist() == model_o.view(np.uint32).tolist(), \
            np.flatnonzero(model_g.view(np.uint32) != model_o.view(np.uint32))[:8]
        o = OracleTable(B, 5, 7, slab_bytes=slab_bytes)
        o.use_model(model_o)
        s, mx = o.chain_profile(keys)
        assert rep["max_slabs_learned"] == mx and abs(rep["mean_slabs_learned"] - s / B) < 1e-12
        o.close()
    finally:
        t.close()
