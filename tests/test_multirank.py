"""The bench's multi-rank path on CPU: two gloo ranks. Replicas run the same
workload, the slowest rank's timed total is the job's time, the whole-job rate
counts every rank's ops, and the reference arm does its work on rank 0 only."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = [3.0, 5.5][rank]
        got = bench.slowest_rank_ms(local, world)
        w, mb = bench.make_step_inputs(0)
        digest = torch.tensor([int(w.keys[:1000].sum()), int(mb.keys[:1000].sum())], dtype=torch.int64)
        gathered = [torch.zeros_like(digest) for _ in range(world)]
        dist.all_gather(gathered, digest)
        out[rank] = (got, all((g == gathered[0]).all() for g in gathered))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_time_and_inputs():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0] == out[1] == (5.5, True)
    # whole-job rate: both ranks' ops over the slowest rank's time
    ms_step = 5.5 / 10
    assert bench.job_value(ms_step, world) == pytest.approx(2 * bench.OPS_PER_STEP / (ms_step * 1e3))


def test_single_rank_needs_no_process_group():
    assert bench.slowest_rank_ms(4.25, 1) == 4.25
    assert bench.job_value(1.0, 1) == pytest.approx(bench.OPS_PER_STEP / 1e3)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    class Args:
        steps, warmup, seed = 1, 1, 0
    assert bench.reference_arm(Args(), rank=1, world=2) is None
    assert capsys.readouterr().out == ""
