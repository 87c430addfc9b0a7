"""Shared pieces of the GPU parity tests: one table on the GPU and one oracle table,
driven with the same seeded inputs and compared element by element."""
from __future__ import annotations

import numpy as np
import torch

from oracle import OracleTable
from paper_1710_11246_gb300 import slabhash as sh

VARIANTS = {"staged": sh.SLAB_VARIANT_STAGED, "direct": sh.SLAB_VARIANT_DIRECT}


def dev(a) -> torch.Tensor:
    return sh.as_device_u32(a)


def host(t: torch.Tensor) -> np.ndarray:
    return sh.to_host_u32(t)


def u8(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy()


class Pair:
    """A GPU table and its oracle twin, fed the same batches."""

    def __init__(self, num_buckets, a, b, pool_slabs=None, variant="staged", key_only=False,
                 n_hint=0, slab_bytes=128, **cfg):
        self.B = int(num_buckets)
        per = (slab_bytes // 4 - 2) // (1 if key_only else 2)  # elements per slab
        pool = pool_slabs if pool_slabs is not None else max(1024, 2 * n_hint // per + 2048)
        mode = sh.SLAB_MODE_KEY_ONLY if key_only else sh.SLAB_MODE_KEY_VALUE
        self.g = sh.SlabHash(self.B, a, b, pool, mode=mode, slab_bytes=slab_bytes)
        self.g.configure(variant=VARIANTS[variant], **cfg)
        self.o = OracleTable(self.B, a, b, key_only=key_only, slab_bytes=slab_bytes)
        self.key_only = key_only

    def close(self):
        self.g.close()
        self.o.close()

    def insert(self, keys, values=None):
        n = len(keys)
        fd = torch.full((n,), 7, dtype=torch.uint8, device="cuda")
        self.g.insert(dev(keys), None if values is None else dev(values), fd)
        fo = self.o.insert(keys, values)
        got = u8(fd)
        assert (got == fo).all(), f"insert found: {np.flatnonzero(got != fo)[:10]}"
        return fo

    def delete(self, keys):
        n = len(keys)
        fd = torch.full((n,), 7, dtype=torch.uint8, device="cuda")
        self.g.delete(dev(keys), fd)
        fo = self.o.delete(keys)
        got = u8(fd)
        assert (got == fo).all(), f"delete found: {np.flatnonzero(got != fo)[:10]}"
        return fo

    def search(self, keys):
        n = len(keys)
        fd = torch.full((n,), 7, dtype=torch.uint8, device="cuda")
        vg = host(self.g.search(dev(keys), found=fd))
        vo, fo = self.o.search(keys)
        assert (u8(fd) == fo).all(), f"search found: {np.flatnonzero(u8(fd) != fo)[:10]}"
        assert (vg == vo).all(), f"search values: {np.flatnonzero(vg != vo)[:10]}"
        return vo, fo

    def mixed(self, ops, keys, values):
        n = len(keys)
        fd = torch.full((n,), 7, dtype=torch.uint8, device="cuda")
        rg = host(self.g.mixed(torch.from_numpy(np.ascontiguousarray(ops, np.uint8)).cuda(), dev(keys),
                               None if values is None else dev(values), found=fd))
        ro, fo = self.o.mixed(ops, keys, values)
        assert (u8(fd) == fo).all(), f"mixed found: {np.flatnonzero(u8(fd) != fo)[:10]}"
        assert (rg == ro).all(), f"mixed results: {np.flatnonzero(rg != ro)[:10]}"
        return ro, fo

    def check_structure(self, expect_flags=0, allow_holes=False, slabs_fixed=True):
        """Per-bucket used slots and slab counts, live multiset, bucket membership,
        allocator bitmaps and status all agree with the oracle / invariants.
        allow_holes: multiset tables after deletes (used slots need not be a
        prefix of the list); slabs_fixed=False skips the per-bucket slab counts
        (a multiset batch mixing inserts and deletes does not fix them)."""
        rc, flags = self.g.status()
        assert flags == expect_flags, (rc, flags)
        slots, slabs, tot = self.g.stats(per_bucket=True)
        oslots, oslabs, otot = self.o.stats()
        gs, gb = host(slots), host(slabs)
        assert (gs == oslots).all(), f"slots differ in buckets {np.flatnonzero(gs != oslots)[:10]}"
        assert tot["live"] == otot["live"] and tot["slots"] == otot["slots"]
        if slabs_fixed:
            assert (gb == oslabs).all(), f"slabs differ in buckets {np.flatnonzero(gb != oslabs)[:10]}"
            assert tot["slabs"] == otot["slabs"]
        if not allow_holes:
            assert tot["prefix_violations"] == 0
        assert tot["pool_allocated"] == tot["linked"], "allocated slabs must all be linked"
        b, k, v = self.g.export()
        ob, ok, ov = self.o.export()
        gk = np.lexsort((host(v), host(k), host(b)))
        okk = np.lexsort((ov, ok, ob))
        assert (host(b)[gk] == ob[okk]).all() and (host(k)[gk] == ok[okk]).all()
        assert (host(v)[gk] == ov[okk]).all()
        return tot
