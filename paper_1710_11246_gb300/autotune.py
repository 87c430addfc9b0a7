"""Autotuner for groups of tables: picks the slab width (128 or 64 bytes), buckets
per key (beta), threads per block and resident blocks per SM by timing the
group's own step on the device.

A step is reset + bulk insert of every table + one search batch per table, all
through the group calls of libslabhash.so. Each candidate (width, beta) needs its
own group (the width and B change the tables' layout); launch parameters are
switched on one group with slab_group_set_config. beta is the mean number of
slabs per bucket at the candidate's width: B = ceil(n / (M beta)) with M = 15
pairs per 128-byte slab or 7 per 64-byte slab.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np
import torch

from . import slabhash as sh
from . import workload as W


@dataclass
class GroupCandidate:
    slab_bytes: int
    beta: float
    threads_per_block: int
    blocks_per_sm: int
    ms: float
    mops: float


def _arrays(w: W.GroupWorkload, device):
    as_i32 = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).to(device)  # noqa: E731
    return (as_i32(w.op_start), sh.as_device_u32(w.keys, device), sh.as_device_u32(w.values, device),
            as_i32(w.search_start), sh.as_device_u32(w.search_keys, device))


def group_step(g: int, arrays, out, found, stream):
    st, k, v, qs, q = arrays
    sh.slab_group_reset(g, stream)
    sh.slab_group_insert(g, st, k, v, stream=stream)
    sh.slab_group_search(g, qs, q, out, found, stream=stream)


def time_group(g: int, arrays, out, found, stream, reps: int = 3) -> float:
    """Best of `reps` step times in ms (CUDA events on `stream`, after one warm-up)."""
    best = float("inf")
    for r in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            group_step(g, arrays, out, found, stream)
            e1.record(stream)
        torch.cuda.synchronize()
        if r:
            best = min(best, e0.elapsed_time(e1))
    rc, flags = sh.slab_group_status(g, stream)
    if rc != sh.SLAB_OK:
        raise RuntimeError(f"group step reported rc={rc} flags={flags}")
    return best


def create_group(w: W.GroupWorkload, beta: float, slab_bytes: int = 128):
    per = (slab_bytes // 4 - 2) // 2  # pairs per slab
    B = np.array([W.buckets_for(max(int(n), 1), beta, per) for n in w.sizes], np.uint32)
    pools = np.maximum(1024, 2 * w.sizes // per + 1024).astype(np.uint64)
    return sh.slab_group_create(B, w.hash_a, w.hash_b, pools, slab_bytes=slab_bytes)


def tune_group(w: W.GroupWorkload, betas=(0.5, 0.6, 0.75), threads=(64, 128, 256), blocks=(0, 4, 8),
               widths=(128, 64), reps: int = 3, device="cuda"):
    """All candidates timed; returns (best, every candidate)."""
    arrays = _arrays(w, device)
    out = torch.empty(len(w.search_keys), dtype=torch.int32, device=device)
    found = torch.empty(len(w.search_keys), dtype=torch.uint8, device=device)
    stream = torch.cuda.Stream()
    ops = 2 * int(w.sizes.sum())
    results = []
    for width, beta in itertools.product(widths, betas):
        g = create_group(w, beta, width)
        try:
            for tpb, bps in itertools.product(threads, blocks):
                cfg = sh.slab_group_get_config(g)
                cfg.threads_per_block, cfg.blocks_per_sm = tpb, bps
                try:
                    sh.slab_group_set_config(g, cfg)
                except sh.SlabError:  # a launch shape this width's kernels cannot take
                    continue
                ms = time_group(g, arrays, out, found, stream, reps)
                results.append(GroupCandidate(width, beta, tpb, bps, ms, ops / (ms * 1e3)))
        finally:
            sh.slab_group_destroy(g)
    return max(results, key=lambda c: c.mops), results
