"""GPU slab hash vs the CPU oracle, element by element, through the C ABI."""
import numpy as np
import pytest
import torch

from oracle import OracleTable, hash_of
from paper_1710_11246_gb300 import slabhash as sh
from paper_1710_11246_gb300 import workload as W
from tests.gpu_helpers import VARIANTS, Pair, dev, host, u8

pytestmark = pytest.mark.gpu

P = W.HASH_PRIME


@pytest.fixture(autouse=True, scope="module")
def _lib():
    sh.load_library()


def test_bucket_hash_matches_oracle():
    rng = np.random.default_rng(0)
    keys = np.concatenate([
        np.array([0, 1, 2, P - 1, P, P + 1, P + 2, 0xFFFFFFFD], np.uint32),
        rng.integers(0, 0xFFFFFFFE, 20000, dtype=np.uint64).astype(np.uint32)])
    for a, b, B in [(1, 0, 1), (1, 0, 7282), (P - 1, P - 1, 466034), (2, 3, 1 << 20),
                    (int(rng.integers(1, P)), int(rng.integers(0, P)), 1398102)]:
        t = sh.SlabHash(B, a, b, 1024)
        got = host(t.buckets_of(dev(keys)))
        want = np.array([hash_of(a, b, B, int(k)) for k in keys], np.uint32)
        t.close()
        assert (got == want).all(), (a, b, B, np.flatnonzero(got != want)[:5])


@pytest.mark.parametrize("variant", list(VARIANTS))
def test_config1(variant):
    """2^16 pairs, B = 7282, 2^16 searches at 50 % hit, 2^14 deletes (seed 0)."""
    w = W.config1()
    p = Pair(w.num_buckets, w.hash_a, w.hash_b, variant=variant, n_hint=len(w.keys))
    try:
        f = p.insert(w.keys, w.values)
        assert f.sum() == 0
        p.check_structure()
        _, found = p.search(w.search.keys)
        assert (found.astype(bool) == w.search.present).all()
        d = p.delete(w.delete_keys)
        assert d.all()
        p.search(w.search.keys)
        p.search(w.delete_keys)
        p.check_structure()
    finally:
        p.close()


@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("n", [0, 1, 31, 33, 1000, 4097])
def test_ragged_sizes(variant, n):
    ks = W.KeyStream(n + 3)
    keys = ks.take(n)
    absent = ks.take(n)
    a, b = W.hash_params(n)
    for B in (1, 3, max(1, n // 9)):
        p = Pair(B, a, b, variant=variant, n_hint=n)
        try:
            p.insert(keys, W.values_for(keys))
            p.search(np.concatenate([keys, absent]))
            p.delete(keys[::2])
            p.search(keys)
            p.check_structure()
        finally:
            p.close()


@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("B,n", [(1, 2000), (2, 1500), (3, 46), (1, 15), (1, 16), (1, 30), (1, 31), (1, 45)])
def test_long_chains_and_slab_boundaries(variant, B, n):
    keys = W.KeyStream(B * 1000 + n).take(n)
    a, b = W.hash_params(7)
    p = Pair(B, a, b, variant=variant, n_hint=n)
    try:
        p.insert(keys, W.values_for(keys))
        p.insert(keys[: n // 2], W.values_for(keys[: n // 2]) + np.uint32(1))  # replaces
        p.search(keys)
        p.delete(keys[1::3])
        p.insert(keys[1::3], W.values_for(keys[1::3]))  # re-insert after delete: new slots
        p.search(keys)
        p.check_structure()
    finally:
        p.close()


@pytest.mark.parametrize("variant", list(VARIANTS))
def test_value_equal_to_not_found_marker(variant):
    key = np.array([0x61C88646, 5, 6], np.uint32)  # 0x61C88646 ^ 0x9E3779B9 = 0xFFFFFFFF
    vals = W.values_for(key)
    assert vals[0] == 0xFFFFFFFF
    p = Pair(4, 3, 5, variant=variant)
    try:
        p.insert(key, vals)
        v, f = p.search(key)
        assert f.tolist() == [1, 1, 1] and v[0] == 0xFFFFFFFF
    finally:
        p.close()


@pytest.mark.parametrize("variant", list(VARIANTS))
def test_reserved_keys_are_refused(variant):
    keys = np.array([10, 0xFFFFFFFE, 11, 0xFFFFFFFF, 12], np.uint32)
    p = Pair(2, 9, 4, variant=variant)
    try:
        p.insert(keys, keys)
        p.search(keys)
        p.delete(keys)
        ops = np.array([0, 1, 2, 0, 2], np.uint8)
        p.mixed(ops, keys, keys)
        p.check_structure(expect_flags=sh.SLAB_FLAG_RESERVED_KEY)
    finally:
        p.close()


@pytest.mark.parametrize("variant", list(VARIANTS))
def test_key_only_mode(variant):
    ks = W.KeyStream(99)
    keys = ks.take(5000)
    absent = ks.take(2000)
    a, b = W.hash_params(99)
    p = Pair(200, a, b, variant=variant, key_only=True, n_hint=5000)
    try:
        p.insert(keys, None)
        p.insert(keys[:100], None)  # already present
        p.search(np.concatenate([keys, absent]))
        p.delete(keys[::4])
        p.search(keys)
        rng = np.random.default_rng(3)
        live = np.setdiff1d(keys, keys[::4])
        mb, _ = W.mixed_batch(ks, live, 3000, (0.3, 0.3, 0.4), rng)
        p.mixed(mb.ops, mb.keys, None)
        p.check_structure()
    finally:
        p.close()


@pytest.mark.parametrize("variant", list(VARIANTS))
def test_mixed_batches(variant):
    """Sec. 6.3 workload at reduced scale: preload 2^16, then batches of 2^14 in each ratio."""
    ks = W.KeyStream(5)
    keys = ks.take(1 << 16)
    a, b = W.hash_params(5)
    B = W.buckets_for(1 << 16, 0.6)
    p = Pair(B, a, b, variant=variant, n_hint=1 << 18)
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


def _kind_runs(kind, n, rng):
    """Op codes for n ops: one kind only, alternating, or in long runs of one kind
    (the first third inserts, then deletes, then searches), with unknown codes
    sprinkled in where `kind` says so."""
    if kind in (0, 1, 2):
        return np.full(n, kind, np.uint8)
    if kind == "alternate":
        return (np.arange(n) % 3).astype(np.uint8)
    if kind == "runs":
        return np.minimum(np.arange(n) * 3 // max(n, 1), 2).astype(np.uint8)
    ops = rng.integers(0, 3, n).astype(np.uint8)  # "unknown": a few codes past search
    odd = rng.random(n) < 0.1
    ops[odd] = rng.integers(3, 256, int(odd.sum())).astype(np.uint8)
    return ops


@pytest.mark.parametrize("n", [1, 31, 33, 100, 4097])
@pytest.mark.parametrize("kind", [0, 1, 2, "alternate", "runs", "unknown"])
@pytest.mark.parametrize("tpb", [128, 32])
def test_mixed_batches_of_one_kind_and_ragged_sizes(n, kind, tpb):
    """Staged mixed kernels sort each tile's ops into a queue of inserts and a ring
    of searches and deletes, and serve each as tiles of their own: batches of one
    kind only, of alternating kinds and of long runs of one kind, at ragged sizes
    (so both queues end in partial tiles), with unknown op codes, and on the
    smallest grid (each warp then serves many tiles and both queues wrap), agree
    with the oracle. Keys are distinct within a batch."""
    ks = W.KeyStream(1000 + n)
    pre = ks.take(2 * n)
    a, b = W.hash_params(n + 11)
    rng = np.random.default_rng(n)
    for B in (1, 3, max(1, n // 9)):
        p = Pair(B, a, b, n_hint=4 * n, threads_per_block=tpb, blocks_per_sm=1 if tpb == 32 else 0)
        try:
            p.insert(pre, W.values_for(pre))
            ops = _kind_runs(kind, n, rng)
            # inserts take fresh keys; deletes and searches take preloaded keys
            # (half of the searches miss)
            fresh = ks.take(n)
            keys = np.where(ops == 0, fresh, pre[rng.permutation(2 * n)[:n]]).astype(np.uint32)
            miss = (ops == 2) & (rng.random(n) < 0.5)
            keys[miss] = ks.take(int(miss.sum()))
            p.mixed(ops, keys, W.values_for(keys))
            p.search(np.concatenate([pre, fresh]))
            p.check_structure()
        finally:
            p.close()


@pytest.mark.parametrize("variant", list(VARIANTS))
def test_pool_exhaustion_reports_and_stays_consistent(variant):
    """One memory block (1024 slabs) cannot hold 2^15 pairs in one bucket: some inserts
    must fail with OUT_OF_SLABS; the rest land, and nothing hangs."""
    keys = W.KeyStream(11).take(1 << 15)
    p = Pair(1, 5, 6, pool_slabs=1024, variant=variant, iter_limit=1 << 20)
    try:
        res = host(p.g.mixed(torch.zeros(len(keys), dtype=torch.uint8, device="cuda"), dev(keys),
                             dev(W.values_for(keys))))
        rc, flags = p.g.status()
        assert rc == sh.SLAB_ERR_OUT_OF_SLABS and flags & sh.SLAB_FLAG_OUT_OF_SLABS
        ok = res == 1
        assert 0 < ok.sum() <= 15 * 1025
        fd = torch.empty(len(keys), dtype=torch.uint8, device="cuda")
        v = host(p.g.search(dev(keys), found=fd))
        hit = fd.cpu().numpy().astype(bool)
        assert (hit == ok).all()
        assert (v[hit] == W.values_for(keys)[hit]).all()
        tot = p.g.stats()
        assert tot["live"] == ok.sum() and tot["prefix_violations"] == 0
        # every allocated slab is linked; slabs freed by lost link races may stay free
        assert tot["pool_allocated"] == tot["linked"] and 1000 <= tot["linked"] <= 1024
    finally:
        p.close()


@pytest.mark.parametrize("variant", list(VARIANTS))
def test_iteration_cap_ends_ops_with_a_status(variant):
    """With a cap of one slab read per op, ops that must walk past the base slab stop
    with ITER_LIMIT instead of finishing (B = 1, 64 keys need 5 slabs)."""
    keys = W.KeyStream(12).take(64)
    p = Pair(1, 5, 6, variant=variant, iter_limit=1)
    try:
        fd = torch.empty(64, dtype=torch.uint8, device="cuda")
        p.g.insert(dev(keys), dev(W.values_for(keys)), fd)
        rc, flags = p.g.status()
        assert rc == sh.SLAB_ERR_ITER_LIMIT and flags == sh.SLAB_FLAG_ITER_LIMIT
        tot = p.g.stats()
        assert tot["live"] < 64 and tot["prefix_violations"] == 0
    finally:
        p.close()


@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("key_only", [False, True])
def test_iteration_cap_counts_slab_reads_across_the_ring(variant, key_only):
    """One bucket filled one slab per batch (five slabs). With a cap of two slab reads
    per op, searches and deletes of keys in the first two slabs finish (in the staged
    kernels the second slab is read when the op's turn in the warp's ring comes) and
    the others stop with ITER_LIMIT and report not found; with the cap lifted, the
    table agrees with the oracle."""
    per = 30 if key_only else 15
    keys = W.KeyStream(91).take(5 * per)
    vals = None if key_only else W.values_for(keys)
    p = Pair(1, 5, 6, variant=variant, key_only=key_only, n_hint=5 * per)
    try:
        for j in range(5):
            p.insert(keys[j * per:(j + 1) * per], None if key_only else vals[j * per:(j + 1) * per])
        tot = p.check_structure()
        assert tot["slabs"] == 5
        cap = sh.slab_get_config(p.g.handle).iter_limit
        p.g.configure(iter_limit=2)
        fd = torch.full((len(keys),), 7, dtype=torch.uint8, device="cuda")
        got = host(p.g.search(dev(keys), found=fd))
        rc, flags = p.g.status()
        assert rc == sh.SLAB_ERR_ITER_LIMIT and flags == sh.SLAB_FLAG_ITER_LIMIT
        f = u8(fd)
        assert (f[:2 * per] == 1).all() and (f[2 * per:] == 0).all()
        if not key_only:
            assert (got[:2 * per] == vals[:2 * per]).all()
        dk = keys[::2]
        fd = torch.full((len(dk),), 7, dtype=torch.uint8, device="cuda")
        p.g.delete(dev(dk), fd)
        rc, flags = p.g.status()
        assert flags & sh.SLAB_FLAG_ITER_LIMIT
        in_first_two = np.isin(dk, keys[:2 * per])
        assert (u8(fd) == in_first_two).all()
        p.o.delete(dk[in_first_two])
        p.g.configure(iter_limit=cap)
        p.search(keys)
        p.check_structure()
    finally:
        p.close()


@pytest.mark.parametrize("variant,tpb,bps", [("staged", 32, 1), ("staged", 128, 2), ("staged", 256, 0),
                                             ("staged", 512, 1), ("staged", 576, 1), ("direct", 32, 1),
                                             ("direct", 128, 2), ("direct", 512, 0), ("direct", 1024, 1)])
def test_launch_shapes(variant, tpb, bps):
    w = W.bulk_workload(20000, 0.8, 20000, 0.5, 5000, seed=4)
    p = Pair(w.num_buckets, w.hash_a, w.hash_b, variant=variant, n_hint=20000,
             threads_per_block=tpb, blocks_per_sm=bps)
    try:
        p.insert(w.keys, w.values)
        p.search(w.search.keys)
        p.delete(w.delete_keys)
        p.check_structure()
    finally:
        p.close()


@pytest.mark.parametrize("variant", list(VARIANTS))
def test_largest_accepted_block_runs(variant):
    """configure() refuses a block the kernels cannot launch (register caps bound
    the staged kernels below 1024 threads); the largest block it accepts runs."""
    w = W.bulk_workload(20000, 0.8, 20000, 0.5, 5000, seed=6)
    p = Pair(w.num_buckets, w.hash_a, w.hash_b, variant=variant, n_hint=20000)
    try:
        for tpb in range(1024, 0, -32):
            try:
                p.g.configure(threads_per_block=tpb, blocks_per_sm=1)
                break
            except sh.SlabError:
                continue
        assert tpb >= 512
        p.insert(w.keys, w.values)
        p.search(w.search.keys)
        p.delete(w.delete_keys)
        p.check_structure()
    finally:
        p.close()


@pytest.mark.parametrize("variant", list(VARIANTS))
def test_invalid_launch_configs_are_rejected(variant):
    """Block sizes that are not whole warps or exceed 1024 threads, occupancy targets
    above 64 blocks per SM and a zero iteration cap are refused; the table keeps its
    previous configuration."""
    t = sh.SlabHash(16, 3, 4, 1024)
    try:
        t.configure(variant=VARIANTS[variant], threads_per_block=512)
        before = t.config()
        for bad in (dict(threads_per_block=48), dict(threads_per_block=2048), dict(threads_per_block=0),
                    dict(blocks_per_sm=65), dict(iter_limit=0), dict(variant=7)):
            with pytest.raises(sh.SlabError):
                t.configure(**bad)
            assert t.config() == before
    finally:
        t.close()


@pytest.mark.parametrize("variant", list(VARIANTS))
def test_reset_after_use_empties_the_table(variant):
    """slab_reset refills the base slabs and the allocated pool slabs only; a table
    reset after long chains and stray allocations behaves like a new one."""
    from oracle import OracleTable
    keys = W.KeyStream(21).take(3000)
    a, b = W.hash_params(21)
    p = Pair(2, a, b, variant=variant, n_hint=3000)
    try:
        p.insert(keys, W.values_for(keys))
        p.delete(keys[::7])
        stray = torch.empty(100, dtype=torch.int32, device="cuda")
        sh.slab_alloc_batch(p.g.handle, stray)
        p.g.reset()
        tot = p.g.stats()
        assert tot["live"] == 0 and tot["slots"] == 0 and tot["slabs"] == 2
        assert tot["pool_allocated"] == 0 and tot["linked"] == 0
        assert (host(p.g.bitmaps()) == 0).all()
        p.o.close()
        p.o = OracleTable(2, a, b)
        p.insert(keys[::2], W.values_for(keys[::2]))
        p.search(keys)
        p.check_structure()
    finally:
        p.close()


def test_side_stream():
    w = W.bulk_workload(30000, 0.6, 30000, 0.5, 3000, seed=8)
    s = torch.cuda.Stream()
    p = Pair(w.num_buckets, w.hash_a, w.hash_b, n_hint=30000)
    try:
        with torch.cuda.stream(s):
            p.insert(w.keys, w.values)
            p.search(w.search.keys)
        p.check_structure()
    finally:
        p.close()


@pytest.mark.parametrize("variant", list(VARIANTS))
def test_slab_alloc_microbench_state(variant):
    """Sec. 5 SlabAlloc, one request per lane served one at a time (direct) or all
    32 of a warp together (staged): n single-slab allocations give n distinct valid
    addresses, the bitmaps mark exactly those units, and freeing them all clears
    every bit."""
    from oracle import check_alloc
    t = sh.SlabHash(8, 3, 4, pool_slabs=1 << 17)
    try:
        n = 100000
        addrs = torch.empty(n, dtype=torch.int32, device="cuda")
        t.configure(random_probes=64, variant=VARIANTS[variant])
        sh.slab_alloc_batch(t.handle, addrs)
        rc, flags = t.status()
        assert rc == sh.SLAB_OK, flags
        a = host(addrs)
        bm = host(t.bitmaps())
        assert check_alloc(a, bm, t.info.num_memory_blocks) == (0, 0)
        sh.slab_free_batch(t.handle, addrs)
        assert (host(t.bitmaps()) == 0).all()
        # more requests than units: the surplus fails with OUT_OF_SLABS, nothing hangs
        m = (1 << 17) + 5000
        addrs = torch.empty(m, dtype=torch.int32, device="cuda")
        sh.slab_alloc_batch(t.handle, addrs)
        rc, flags = t.status()
        assert rc == sh.SLAB_ERR_OUT_OF_SLABS
        a = host(addrs)
        good = a != 0xFFFFFFFF
        assert good.sum() <= 1 << 17
        assert check_alloc(a[good], host(t.bitmaps()), t.info.num_memory_blocks) == (0, 0)
    finally:
        t.close()


def test_create_seeded_uses_the_seeded_parameters():
    """slab_create_seeded draws (a, b) with slab_hash_params and reports them; a table
    built that way agrees with the oracle on those parameters."""
    w = W.config1(seed=0)
    h = sh.slab_create_seeded(w.num_buckets, sh.SLAB_MODE_KEY_VALUE, 1234, 4096)
    try:
        info = sh.slab_get_info(h)
        assert (info.hash_a, info.hash_b) == sh.slab_hash_params(1234)
        o = OracleTable(w.num_buckets, info.hash_a, info.hash_b)
        fd = torch.empty(len(w.keys), dtype=torch.uint8, device="cuda")
        sh.slab_insert_batch(h, dev(w.keys), dev(w.values), fd)
        o.insert(w.keys, w.values)
        vals = torch.empty(len(w.search.keys), dtype=torch.int32, device="cuda")
        found = torch.empty(len(w.search.keys), dtype=torch.uint8, device="cuda")
        sh.slab_search_batch(h, dev(w.search.keys), vals, found)
        vo, fo = o.search(w.search.keys)
        assert (host(vals) == vo).all() and (u8(found) == fo).all()
        o.close()
    finally:
        sh.slab_destroy(h)


@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("key_only", [False, True])
def test_repeated_keys_in_one_batch_follow_a_serial_order(variant, key_only):
    """Ops of one batch are concurrent; with a key repeated, every outcome must be one
    that some serial order of the ops produces: keys stay unique, exactly one of a
    new key's inserts reports it new, the stored value is one the batch wrote, and
    searches see the key's value before or after the batch's writes."""
    ks = W.KeyStream(41)
    pre = ks.take(6000)
    new = ks.take(3000)
    B = W.buckets_for(9000, 0.6)
    p = Pair(B, 17, 23, variant=variant, key_only=key_only, n_hint=12000)
    try:
        p.insert(pre, None if key_only else W.values_for(pre))
        rng = np.random.default_rng(42)
        gone = pre[:2000]
        ops = np.concatenate([np.full(3000, 0, np.uint8), np.full(3000, 0, np.uint8), np.full(3000, 2, np.uint8),
                              np.full(2000, 1, np.uint8), np.full(2000, 2, np.uint8)])
        keys = np.concatenate([new, new, new, gone, gone]).astype(np.uint32)
        v1, v2 = (new * np.uint32(3)).astype(np.uint32), (new * np.uint32(5)).astype(np.uint32)
        vals = np.concatenate([v1, v2, np.zeros(7000, np.uint32)]).astype(np.uint32)
        perm = rng.permutation(len(keys))
        fd = torch.empty(len(keys), dtype=torch.uint8, device="cuda")
        res = host(p.g.mixed(torch.from_numpy(ops[perm]).cuda(), dev(keys[perm]),
                             None if key_only else dev(vals[perm]), found=fd))
        fnd = u8(fd)
        r, f = np.empty_like(res), np.empty_like(fnd)
        r[perm], f[perm] = res, fnd
        rc, flags = p.g.status()
        assert flags == 0
        # the two inserts of each new key: exactly one found it absent
        f_ins = f[:3000] + f[3000:6000]
        assert (f_ins == 1).all() and ((r[:3000] + r[3000:6000]) == 1).all()
        # deletes of preloaded keys all hit
        assert (f[9000:11000] == 1).all() and (r[9000:11000] == 1).all()
        # searches: before or after the batch's writes
        s_new, sf_new = r[6000:9000], f[6000:9000]
        if key_only:
            assert ((s_new == 0) | (s_new == sh.SLAB_NOT_FOUND)).all()
        else:
            assert ((sf_new == 0) & (s_new == sh.SLAB_NOT_FOUND) | (sf_new == 1) & ((s_new == v1) | (s_new == v2))).all()
        s_gone, sf_gone = r[11000:], f[11000:]
        want = 0 if key_only else W.values_for(gone)
        assert ((sf_gone == 0) & (s_gone == sh.SLAB_NOT_FOUND) | (sf_gone == 1) & (s_gone == want)).all()
        # afterwards: new keys once each with a value the batch wrote, deleted keys gone
        fd2 = torch.empty(3000, dtype=torch.uint8, device="cuda")
        vals_now = host(p.g.search(dev(new), found=fd2))
        assert (u8(fd2) == 1).all()
        if not key_only:
            assert ((vals_now == v1) | (vals_now == v2)).all()
        fd3 = torch.empty(2000, dtype=torch.uint8, device="cuda")
        p.g.search(dev(gone), found=fd3)
        assert (u8(fd3) == 0).all()
        tot = p.g.stats()
        assert tot["live"] == 6000 - 2000 + 3000 and tot["prefix_violations"] == 0
    finally:
        p.close()


@pytest.mark.parametrize("key_only", [False, True])
def test_deferred_ops_cycle_through_long_lists(key_only):
    """Staged kernels park ops that need another slab and serve them later, 32 at a
    time. Lists of ~8 slabs and the smallest grid (one 32-thread block per SM, so
    each warp serves many tiles) send every op round that ring several times and
    wrap it over and over: inserts, replaces, searches, deletes and mixed batches
    all agree with the oracle."""
    n = 1 << 16
    ks = W.KeyStream(41)
    keys = ks.take(n)
    a, b = W.hash_params(41)
    per = 30 if key_only else 15
    B = max(1, n // (8 * per))
    p = Pair(B, a, b, key_only=key_only, n_hint=2 * n, threads_per_block=32, blocks_per_sm=1)
    vals = None if key_only else W.values_for(keys)
    try:
        p.insert(keys, vals)
        p.insert(keys[::2], None if key_only else vals[::2] + np.uint32(3))
        p.search(np.concatenate([keys[::3], ks.take(n // 4)]))
        p.delete(keys[1::4])
        rng = np.random.default_rng(41)
        live = np.setdiff1d(keys, keys[1::4])
        for ratios in W.CONFIG3_RATIOS:
            mb, live = W.mixed_batch(ks, live, n // 2, ratios, rng)
            p.mixed(mb.ops, mb.keys, None if key_only else mb.values)
        p.search(live[: n // 2])
        tot = p.check_structure()
        assert tot["slabs"] >= 4 * B
    finally:
        p.close()


@pytest.mark.parametrize("variant", list(VARIANTS))
def test_growth_burst_in_a_tight_pool(variant):
    """One batch whose ops all start together and pile onto 64 lists (~45 per
    list, each list growing to 3-5 slabs): for a moment many more ops want a new
    slab than the 1024-slab pool holds, though the table needs ~200. An op that
    finds no free slab follows the slab another op linked meanwhile, so nothing
    fails and the table matches the oracle."""
    n = 64 * 45
    keys = W.KeyStream(77).take(n)
    a, b = W.hash_params(77)
    p = Pair(64, a, b, pool_slabs=1024, variant=variant)
    try:
        p.insert(keys, W.values_for(keys))
        tot = p.check_structure()
        assert tot["pool_allocated"] < 400
        p.search(keys)
    finally:
        p.close()


@pytest.mark.parametrize("variant,key_only", [("staged", False), ("staged", True), ("direct", False)])
def test_long_lists_in_a_table_larger_than_l2(variant, key_only):
    """Search, delete and mixed batches on a table whose base slabs (2^20 x 128 B =
    134 MB) are far larger than half the L2, the case where those kernels restage
    an op's next slab inside its tile (and pull slabs into L2 ahead) instead of
    parking the op. With
    h(k) = k mod B (a = 1, b = 0) the keys bucket + j * B fill 1000 lists with 60
    keys each (4 slabs in key-value mode, 2 in key-only mode); hits, misses and
    deletes along the lists agree with the oracle. The one batch of inserts also
    makes ~45 ops per list want a new slab at the same moment, in a pool about
    three times the table's need."""
    B = 1 << 20
    j = np.arange(90, dtype=np.uint64)
    keys = (np.arange(1000, dtype=np.uint64)[:, None] + j[None, :] * B).astype(np.uint32)
    stored = keys[:, :60].ravel()
    absent = keys[:, 60:].ravel()
    rng = np.random.default_rng(7)
    stored = stored[rng.permutation(len(stored))]
    p = Pair(B, 1, 0, variant=variant, key_only=key_only, n_hint=len(stored))
    try:
        p.insert(stored, None if key_only else W.values_for(stored))
        p.search(np.concatenate([stored[::2], absent[::3]]))
        p.delete(stored[::3])
        p.search(np.concatenate([stored, absent[::5]]))
        tot = p.check_structure()
        assert tot["slabs"] == B + (1000 if key_only else 3000)
        if variant == "staged":
            # one mixed batch along the same lists: deletes and hits of stored keys,
            # misses and inserts of absent ones (the inserts grow some lists again)
            live = np.setdiff1d(stored, stored[::3])
            ins, miss = absent[1::5][:4000], absent[2::5]
            keys = np.concatenate([ins, live[:6000], live[6000:20000], miss]).astype(np.uint32)
            ops = np.concatenate([np.zeros(len(ins), np.uint8), np.ones(6000, np.uint8),
                                  np.full(len(keys) - len(ins) - 6000, 2, np.uint8)])
            perm = rng.permutation(len(keys))
            p.mixed(ops[perm], keys[perm], W.values_for(keys[perm]))
            p.search(np.concatenate([live, ins]))
            p.check_structure()
    finally:
        p.close()


def test_full_size_step_matches_the_oracle():
    """The benchmark's step at full size, in its launch configuration (staged
    kernels, default block size and occupancy): 2^22 pairs built at beta 0.6, 2^22
    searches at 50 % hit, 2^20 deletes, then 2^20 mixed ops at (0.2, 0.2, 0.6).
    The oracle runs the same 10.5 M ops; every result, found flag, per-bucket slot
    and slab count and the exported table agree element by element."""
    w = W.config2(0.6, 0.5, seed=0)
    ks = W.KeyStream(0)
    ks.take(len(w.keys) + (len(w.search.keys) - int(round(len(w.search.keys) * 0.5))))
    rng = np.random.default_rng([0, 0x3333])
    live = np.setdiff1d(w.keys, w.delete_keys, assume_unique=True)
    mb, _ = W.mixed_batch(ks, live, 1 << 20, (0.2, 0.2, 0.6), rng)
    p = Pair(w.num_buckets, w.hash_a, w.hash_b, pool_slabs=1 << 20)
    try:
        assert p.insert(w.keys, w.values).sum() == 0
        _, found = p.search(w.search.keys)
        assert (found.astype(bool) == w.search.present).all()
        assert p.delete(w.delete_keys).all()
        p.mixed(mb.ops, mb.keys, mb.values)
        p.check_structure()
    finally:
        p.close()


@pytest.mark.parametrize("beta", [0.2, 2.0])
def test_full_size_betas_and_hit_rates_match_the_oracle(beta):
    """2^22 pairs at the smallest and largest mean fill of the bulk sweep (beta 0.2:
    1.4 M one-slab lists; beta 2.0: 2.45 slabs per list, so many searches and
    deletes go on through the ring), 2^22 searches at 100 % and at 0 % hit, 2^20
    deletes: every output and the final table agree with the oracle."""
    w1 = W.config2(beta, 1.0, seed=0)
    w0 = W.config2(beta, 0.0, seed=0)
    assert (w1.keys == w0.keys).all()
    p = Pair(w1.num_buckets, w1.hash_a, w1.hash_b, pool_slabs=1 << 21)
    try:
        assert p.insert(w1.keys, w1.values).sum() == 0
        _, f1 = p.search(w1.search.keys)
        _, f0 = p.search(w0.search.keys)
        assert f1.all() and not f0.any()
        assert p.delete(w1.delete_keys).all()
        p.search(w1.search.keys[: 1 << 20])
        p.check_structure()
    finally:
        p.close()


def test_slab_alloc_full_size():
    """The SlabAlloc microbenchmark's size (Sec. 5): 2^24 single-slab allocations
    from a pool of 2^25 units in one launch give 2^24 distinct valid addresses that
    the bitmaps mark exactly; freeing them all clears every bit."""
    from oracle import check_alloc
    t = sh.SlabHash(8, 3, 4, pool_slabs=1 << 25)
    try:
        n = 1 << 24
        addrs = torch.empty(n, dtype=torch.int32, device="cuda")
        sh.slab_alloc_batch(t.handle, addrs)
        rc, flags = t.status()
        assert rc == sh.SLAB_OK, flags
        a = host(addrs)
        assert check_alloc(a, host(t.bitmaps()), t.info.num_memory_blocks) == (0, 0)
        sh.slab_free_batch(t.handle, addrs)
        assert (host(t.bitmaps()) == 0).all()
    finally:
        t.close()


def test_full_size_concurrent_batches_match_the_oracle():
    """The concurrent benchmark's sizes (Sec. 6.3): 2^22 pairs preloaded at beta 0.6,
    then batches of 2^20 mixed ops at each of (0.5, 0.5, 0), (0.2, 0.2, 0.6) and
    (0.05, 0.05, 0.9), three batches per ratio here (the benchmark runs 64): every
    result and found flag and the final table agree with the oracle."""
    w = W.config2(0.6, 0.5, seed=3)
    ks = W.KeyStream(3)
    ks.take(len(w.keys) + len(w.search.keys))
    rng = np.random.default_rng(3)
    p = Pair(w.num_buckets, w.hash_a, w.hash_b, pool_slabs=1 << 21)
    try:
        assert p.insert(w.keys, w.values).sum() == 0
        live = w.keys
        for ratios in W.CONFIG3_RATIOS:
            for _ in range(3):
                mb, live = W.mixed_batch(ks, live, 1 << 20, ratios, rng)
                p.mixed(mb.ops, mb.keys, mb.values)
        p.search(live[: 1 << 20])
        p.check_structure()
    finally:
        p.close()
