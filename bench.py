"""Benchmark of the slab hash hot path on GB300.

One step = one pass of the whole hot path over one batch of the 2^22-key bulk
workload (Sec. 6.1, beta = 0.6, 50 % search hits) followed by one concurrent
batch (Sec. 6.3): reset the table, bulk-build 2^22 pairs, search 2^22 keys,
delete 2^20 keys, run 2^20 mixed ops (insert/delete/search = 0.2/0.2/0.6).
Inputs are resident in HBM before the timed region; L2 is flushed (a 256 MiB
write) before every step. Prints one JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --sweep   # extra lines: beta sweep, hit rates, SlabAlloc, probes
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1710_11246_gb300 import workload as W  # noqa: E402

METRIC = "Mops/s search/insert/delete/mixed at 2^22 keys; % of random-128B-line roofline"
N_KEYS = 1 << 22
N_SEARCH = 1 << 22
N_DELETE = 1 << 20
N_MIXED = 1 << 20
BETA = 0.6
HIT = 0.5
SERVING_KEYS, SERVING_REQUESTS, SERVING_POOL, SERVING_SLOT_OPS = 1 << 26, 8192, 1 << 22, 1 << 20
MIXED_RATIOS = (0.2, 0.2, 0.6)
POOL_SLABS = 1 << 20
OPS_PER_STEP = N_KEYS + N_SEARCH + N_DELETE + N_MIXED
PHASES = ("reset", "build", "search", "delete", "mixed")

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the staged
# build kernel from one ncu capture of this workload. They describe the kernel
# sources they were taken from (the headers that define the staged kernels' device
# code) and are dropped as soon as those sources change.
KERNEL_SOURCES = ("slab_device.cuh", "slab_wcws.cuh", "slab_staged.cuh")
NCU_TRAFFIC = {"sources_sha256": "0c96e2eb2dd3c7e8", "build": 103.46e6}


def ncu_traffic(phase: str):
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1710_11246_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return NCU_TRAFFIC.get(phase) if h.hexdigest()[:16] == NCU_TRAFFIC["sources_sha256"] else None


def make_step_inputs(seed: int = 0, per_slab: int = 15):
    """The step's batches (deterministic for a seed); per_slab = M sets the bucket
    count B = ceil(n / (M beta)) (15 pairs per 128-byte slab, 7 per 64-byte slab)."""
    w = W.config2(BETA, HIT, seed, per_slab=per_slab)
    stream = W.KeyStream(seed)
    stream.take(N_KEYS + (N_SEARCH - int(round(N_SEARCH * HIT))))  # skip keys the bulk workload used
    rng = np.random.default_rng([seed, 0x3333])
    live = np.setdiff1d(w.keys, w.delete_keys, assume_unique=True)
    mb, _ = W.mixed_batch(stream, live, N_MIXED, MIXED_RATIOS, rng)
    return w, mb


def config_dict(extra=None):
    d = {"workload": f"bulk build 2^22 pairs (beta={BETA}, B=ceil(n/(15*beta))), search 2^22 at "
                     f"{int(HIT * 100)}% hit, delete 2^20, mixed 2^20 ops {MIXED_RATIOS}",
         "num_keys": N_KEYS, "beta": BETA, "num_buckets": W.buckets_for(N_KEYS, BETA),
         "ops_per_step": OPS_PER_STEP, "l2": "flushed before every step (256 MiB write)",
         "parallelism": "replicas"}
    if extra:
        d.update(extra)
    return d


# ---------------------------------------------------------------- CPU oracle
def run_oracle_step(w, mb, slab_bytes: int = 128):
    """One step on the CPU oracle; returns (seconds, lines touched per phase, slabs
    linked per phase). The seconds cover the four batches only."""
    from oracle import OracleTable
    o = OracleTable(w.num_buckets, w.hash_a, w.hash_b, slab_bytes=slab_bytes)
    lines, linked, dt = {}, {}, 0.0
    slabs = o.stats()[2]["slabs"]
    batches = (("build", lambda: o.insert(w.keys, w.values)), ("search", lambda: o.search(w.search.keys)),
               ("delete", lambda: o.delete(w.delete_keys)), ("mixed", lambda: o.mixed(mb.ops, mb.keys, mb.values)))
    for name, fn in batches:
        o.lines = 0
        t0 = time.perf_counter()
        fn()
        dt += time.perf_counter() - t0
        lines[name] = o.lines
        now = o.stats()[2]["slabs"]
        linked[name], slabs = now - slabs, now
    o.close()
    return dt, lines, linked


def host_cpu() -> str:
    """CPU model and logical core count of this host (best effort)."""
    model = ""
    try:
        import subprocess
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu model")):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return f"{model or 'unknown CPU'}, {os.cpu_count()} logical cores"


def cpu_baseline(w, mb, budget_s: float = 10.0):
    """The oracle as it stands, single-threaded, on whole steps of the same workload."""
    times, lines, linked = [], None, None
    t_start = time.perf_counter()
    while not times or (time.perf_counter() - t_start < budget_s and len(times) < 5):
        dt, lines, linked = run_oracle_step(w, mb)
        times.append(dt)
    v = OPS_PER_STEP * len(times) / sum(times) / 1e6
    return {"value": round(v, 3), "unit": "Mops/s", "cores": 1, "kind": "oracle", "host": host_cpu(),
            "sample": f"{len(times)} whole step(s) of the workload ({OPS_PER_STEP} ops each), "
                      f"plain C oracle, one thread"}, (lines, linked), times


# ---------------------------------------------------------------- clocks
class ClockSampler:
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap,utilization.gpu")

    def __init__(self, index: int):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.p = None
        return self

    def __exit__(self, *a):
        self.rows = []
        if self.p is None:
            return
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                self.rows.append(f)

    def summary(self):
        if not getattr(self, "rows", None):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[0]) for r in self.rows if num(r[0]) is not None]
        busy = [num(r[0]) for r in self.rows if num(r[8]) and num(r[8]) > 0 and num(r[0]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[4 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(busy or sm) if sm else None,
                "sm_max_mhz": num(self.rows[0][1]), "reasons": reasons, "samples": len(self.rows),
                "power_w_max": max((num(r[2]) or 0) for r in self.rows)}


# ---------------------------------------------------------------- GPU arm
def slowest_rank_ms(local_ms: float, world: int) -> float:
    """The job's time: the largest of the ranks' timed totals (replicas run the same
    workload each, so the slowest one decides when all of them are done)."""
    if world <= 1:
        return float(local_ms)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    x = torch.tensor([float(local_ms)], dtype=torch.float64, device=dev)
    dist.all_reduce(x, op=dist.ReduceOp.MAX)
    return float(x.item())


def job_value(ms_per_step: float, world: int) -> float:
    """Whole-job Mops/s: every rank runs OPS_PER_STEP per step (weak scaling)."""
    return OPS_PER_STEP * world / (ms_per_step * 1e3)


def gpu_arm(args, rank, world, device):
    import torch

    from paper_1710_11246_gb300 import slabhash as sh

    sh.load_library()
    w, mb = make_step_inputs(args.seed)
    dev = sh.as_device_u32
    t = sh.SlabHash(w.num_buckets, w.hash_a, w.hash_b, POOL_SLABS)
    if args.variant == "direct":
        t.configure(variant=sh.SLAB_VARIANT_DIRECT)
    if args.threads_per_block:
        t.configure(threads_per_block=args.threads_per_block)
    if args.blocks_per_sm is not None:
        t.configure(blocks_per_sm=args.blocks_per_sm)
    stream = torch.cuda.Stream()
    h = t.handle

    # device-resident inputs and outputs
    k_build, v_build = dev(w.keys), dev(w.values)
    k_search = dev(w.search.keys)
    k_del = dev(w.delete_keys)
    m_ops = torch.from_numpy(mb.ops).to(device)
    m_keys, m_vals = dev(mb.keys), dev(mb.values)
    o_search = torch.empty(N_SEARCH, dtype=torch.int32, device=device)
    f_search = torch.empty(N_SEARCH, dtype=torch.uint8, device=device)
    f_del = torch.empty(N_DELETE, dtype=torch.uint8, device=device)
    o_mixed = torch.empty(N_MIXED, dtype=torch.int32, device=device)
    f_mixed = torch.empty(N_MIXED, dtype=torch.uint8, device=device)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    torch.cuda.synchronize()

    def step(evs, at=None):
        """One step. evs is None (no events), a list of 6 events around every
        phase, or (with `at` a phase index) 4 events: step start, before and after
        phase `at` (not recorded when `at` is -1), step end."""
        calls = (lambda: sh.slab_reset(h, stream),
                 lambda: sh.slab_insert_batch(h, k_build, v_build, None, stream=stream),
                 lambda: sh.slab_search_batch(h, k_search, o_search, f_search, stream=stream),
                 lambda: sh.slab_delete_batch(h, k_del, f_del, stream=stream),
                 lambda: sh.slab_mixed_batch(h, m_ops, m_keys, m_vals, o_mixed, f_mixed, stream=stream))
        if evs is not None and at is None:
            for i, c in enumerate(calls):
                evs[i].record(stream)
                c()
            evs[5].record(stream)
            return
        if evs is not None:
            evs[0].record(stream)
        for i, c in enumerate(calls):
            if evs is not None and i == at:
                evs[1].record(stream)
            c()
            if evs is not None and i == at:
                evs[2].record(stream)
        if evs is not None:
            evs[3].record(stream)

    def new_events(k=6):
        return [torch.cuda.Event(enable_timing=True) for _ in range(k)]

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.zero_()
            step(new_events())
    torch.cuda.synchronize()
    rc, flags = t.status(stream)
    if rc != sh.SLAB_OK:
        raise RuntimeError(f"device status after warm-up: rc={rc} flags={flags}")

    # instrumented pass: events between every phase give the per-op breakdown (the
    # events keep consecutive batch kernels from overlapping, so this pass is a
    # few per cent slower than the timed one)
    all_evs = []
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            flush.zero_()
            evs = new_events()
            step(evs)
            all_evs.append(evs)
    torch.cuda.synchronize()
    per_phase = {p: [] for p in PHASES}
    for evs in all_evs:
        for i, p in enumerate(PHASES):
            per_phase[p].append(evs[i].elapsed_time(evs[i + 1]))
    dom = max(PHASES[1:], key=lambda p: statistics.fmean(per_phase[p]))
    at = PHASES.index(dom)

    # timed pass: K steps, events at the step bounds and, in every tenth step (and
    # the last), around the dominant kernel (its launch durations feed the
    # roofline). An event between two batch kernels keeps the second from being
    # launched as the first one's blocks exit, so the other steps carry none.
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    timed = []
    with ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ
                      else int(os.environ.get("LOCAL_RANK", 0))) as clk:
        time.sleep(0.25)
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for i in range(args.steps):
                flush.zero_()
                evs = new_events(4)
                probe = i % 10 == 9 or i == args.steps - 1
                step(evs, at if probe else -1)
                timed.append((evs, probe))
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        time.sleep(0.25)
    if world > 1:
        torch.distributed.barrier()
    rc, flags = t.status(stream)
    if rc != sh.SLAB_OK:
        raise RuntimeError(f"device status after timed steps: rc={rc} flags={flags}")
    step_ms = [evs[0].elapsed_time(evs[3]) for evs, _ in timed]
    dom_ms = [evs[1].elapsed_time(evs[2]) for evs, probe in timed if probe]
    total_ms = slowest_rank_ms(sum(step_ms), world)

    # end to end through the C ABI from pinned host buffers
    # every replica runs it, so the ranks stay in step; the job's time is the slowest
    e2e = e2e_arm(args, t, w, mb, device, stream)
    e2e_ms = slowest_rank_ms(e2e["ms_per_step"], world)
    e2e["value"] = round(job_value(e2e_ms, world), 1)
    e2e["ms_per_step"] = round(e2e_ms, 4)
    res = dict(per_phase=per_phase, step_ms=step_ms, total_ms=total_ms, wall=wall, clocks=clk.summary(),
               e2e=e2e, table=t, w=w, mb=mb, dom=dom, dom_ms=dom_ms)
    return res


def e2e_arm(args, t, w, mb, device, stream):
    """End to end through the C ABI's host-memory batch call (slab_batch_host): every
    step passes page-locked host arrays of all its inputs and gets all its results
    back in host arrays. The library copies each chunk in and its results out on
    its own copy streams, overlapping the kernels of the neighbouring chunks; each
    call records a completion event instead of making the kernel stream wait for
    its copies, so a step's copies also overlap the next step's batches."""
    import torch

    from paper_1710_11246_gb300 import slabhash as sh
    h = t.handle
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32 if a.dtype == np.uint32 else a.dtype)).pin_memory()  # noqa: E731
    hin = dict(k=pin(w.keys), v=pin(w.values), s=pin(w.search.keys), dl=pin(w.delete_keys), ops=pin(mb.ops),
               mk=pin(mb.keys), mv=pin(mb.values))
    out_shapes = [(N_SEARCH, torch.int32), (N_SEARCH, torch.uint8), (N_DELETE, torch.uint8), (N_MIXED, torch.int32),
                  (N_MIXED, torch.uint8)]
    hout = [torch.empty(n, dtype=dt).pin_memory() for n, dt in out_shapes]
    h2d = sum(x.numel() * x.element_size() for x in hin.values())
    d2h = sum(x.numel() * x.element_size() for x in hout)
    ks = stream

    def one(last_event=None):
        sh.slab_reset(h, ks)
        sh.slab_batch_host(h, sh.SLAB_BATCH_INSERT, hin["k"], values=hin["v"], stream=ks, done_event=torch.cuda.Event())
        sh.slab_batch_host(h, sh.SLAB_BATCH_SEARCH, hin["s"], results=hout[0], found=hout[1], stream=ks,
                           done_event=torch.cuda.Event())
        sh.slab_batch_host(h, sh.SLAB_BATCH_DELETE, hin["dl"], found=hout[2], stream=ks, done_event=torch.cuda.Event())
        sh.slab_batch_host(h, sh.SLAB_BATCH_MIXED, hin["mk"], ops=hin["ops"], values=hin["mv"], results=hout[3],
                           found=hout[4], stream=ks, done_event=last_event or torch.cuda.Event())

    steps = max(3, min(args.steps, 20))
    for _ in range(args.warmup):
        one()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(ks)
    for i in range(steps):
        one(e1 if i == steps - 1 else None)
    e1.synchronize()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    # the last step's results on the host: every present key found, every delete hit
    if int(hout[1].sum()) != int(w.search.present.sum()) or not bool((hout[2] == 1).all()):
        raise RuntimeError("end-to-end results on the host disagree with the workload")
    return {"value": round(OPS_PER_STEP / (ms * 1e3), 1), "unit": "Mops/s", "ms_per_step": round(ms, 4),
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": steps,
            "api": "slab_batch_host (host arrays in, host arrays out, default chunks of 2^22 ops)",
            "overlap": "each chunk's copies overlap the neighbouring chunks' kernels; completion events let a "
                       "step's copies overlap the next step's batches"}


def random_line_probe(device, footprint_bytes: int, n_reads: int = 1 << 24, line_bytes: int = 128,
                      quick: bool = False):
    """Best random 128-byte-line read rate (lines/s) at a footprint, over three access
    forms (32 lanes x 4 B per line; 8 lanes x 16 B into registers; 8 lanes x 16 B
    cp.async into a shared-memory stage, as the staged kernels move slabs), lines in
    flight and block size."""
    import torch

    from paper_1710_11246_gb300 import slabhash as sh
    lines = footprint_bytes // line_bytes
    buf = torch.zeros(lines * (line_bytes // 4), dtype=torch.int32, device=device)
    sink = torch.zeros(1, dtype=torch.int32, device=device)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    lanes = line_bytes // 16  # lanes per line in the 16-byte-per-lane forms
    forms = []
    if line_bytes == 128 and not quick:
        forms += [("32x4B", lif, lambda rep, lif, tpb: sh.slab_probe_random_lines(buf, lines, n_reads, rep + 1, lif,
                                                                                 tpb, sink)) for lif in (4, 8, 16)]
    forms += [(f"{lanes}x16B_ld", lif, lambda rep, lif, tpb: sh.slab_probe_random_lines_v4(
        buf, lines, n_reads, rep + 1, 0, lif, tpb, sink, line_bytes=line_bytes))
        for lif in ((8, 16) if quick else (8, 16, 32))]
    forms += [(f"{lanes}x16B_cp.async", lif, lambda rep, lif, tpb: sh.slab_probe_random_lines_v4(
        buf, lines, n_reads, rep + 1, 1, lif, tpb, sink, line_bytes=line_bytes))
        for lif in ((64,) if quick else (32, 64))]
    best = (0.0, None)
    per_form = {}
    for name, lif, fn in forms:
        for tpb in (256, 512):
            ts = []
            for rep in range(3 if quick else 4):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                fn(rep, lif, tpb)
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            rate = n_reads / (min(ts[1:]) * 1e-3)
            per_form[name] = max(per_form.get(name, 0.0), rate)
            if rate > best[0]:
                best = (rate, {"form": name, "lines_in_flight": lif, "threads_per_block": tpb})
    del buf
    best[1]["glines_per_s_by_form"] = {k: round(v / 1e9, 3) for k, v in per_form.items()}
    return best


def random_cas_probe(device, footprint_bytes: int, n_ops: int = 1 << 22, quick: bool = False):
    """Best random 64-bit atomicCAS rate (ops/s) on pair slots of lines at a footprint,
    the buffer zeroed before each timing so most CASes claim an empty slot."""
    import torch

    from paper_1710_11246_gb300 import slabhash as sh
    lines = footprint_bytes // 128
    buf = torch.zeros(lines * 16, dtype=torch.int64, device=device)
    best = (0.0, None)
    for oif in ((8,) if quick else (2, 4, 8)):
        for tpb in (256, 512):
            ts = []
            for rep in range(3 if quick else 4):
                buf.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                sh.slab_probe_random_cas(buf, lines, n_ops, rep + 1, oif, tpb)
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            rate = n_ops / (min(ts[1:]) * 1e-3)
            if rate > best[0]:
                best = (rate, {"ops_in_flight": oif, "threads_per_block": tpb})
    del buf
    return best


# ---------------------------------------------------------------- sweep
def _time_ms(fn, stream, flush):
    """Device time of fn() on `stream`, after an L2 flush queued on the same stream."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        flush.zero_()
        e0.record(stream)
        fn()
        e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def sweep(args, device):
    """Extra JSON lines: the bulk benchmark over beta and hit rate (Sec. 6.1), the
    SlabAlloc microbenchmark (Sec. 5) and full-size concurrent batches (Sec. 6.3)."""
    import torch

    from paper_1710_11246_gb300 import slabhash as sh
    sh.load_library()
    dev = sh.as_device_u32
    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    reps = 5

    def best(fn):
        return min(_time_ms(fn, stream, flush) for _ in range(reps))

    def want(name):
        return args.sweep in ("all", name)

    # bulk: build, search at 0/50/100 % hit, delete, for every beta
    for beta in (W.CONFIG2_BETAS if want("bulk") else ()):
        print(json.dumps({"sweep": "bulk", **bulk_point(args, device, stream, flush, beta, reps)[0]}), flush=True)

    if want("slaballoc"):
        slaballoc_sweep(device, stream, flush, reps)
    if want("learned"):
        learned_sweep(args, device, stream, flush)
    if want("group"):
        group_sweep(args, device, stream, flush)
    if want("serving"):
        serving_sweep(args, device, stream, flush)
    if want("flush"):
        flush_sweep(args, device, stream, flush)
    if want("sizes"):
        sizes_sweep(args, device, stream, flush)
    if want("incremental"):
        incremental_sweep(args, device, stream, flush)
    if not want("mixed"):
        return
    # concurrent batches at full size: preload 2^22 (beta = 0.6), 64 batches of 2^20
    for ratios in W.CONFIG3_RATIOS:
        print(json.dumps({"sweep": "mixed", **mixed_series(args, device, stream, flush, ratios)[0]}), flush=True)


def bulk_point(args, device, stream, flush, beta, reps=5, slab_bytes=128):
    """The bulk benchmark (Sec. 6.1) at one beta: build 2^22 pairs (incl. the reset),
    search 2^22 keys at 0 / 50 / 100 % hit, delete 2^20 keys, each timed alone after
    an L2 flush, best of `reps`. Returns (rates, host inputs for the oracle)."""
    import torch

    from paper_1710_11246_gb300 import slabhash as sh
    dev = sh.as_device_u32
    per = (slab_bytes // 4 - 2) // 2
    w = W.config2(beta, 0.5, args.seed, per_slab=per)
    stream_k = W.KeyStream(args.seed)
    stream_k.take(N_KEYS + N_SEARCH)
    rng = np.random.default_rng([args.seed, 0x5EA])
    absent = stream_k.take(N_SEARCH)
    hit100 = w.keys[rng.permutation(N_KEYS)]
    queries = {0.0: absent, 0.5: w.search.keys, 1.0: hit100}
    t = sh.SlabHash(w.num_buckets, w.hash_a, w.hash_b, 1 << 21, slab_bytes=slab_bytes)
    h = t.handle
    kb, vb, kd = dev(w.keys), dev(w.values), dev(w.delete_keys)
    out = torch.empty(N_SEARCH, dtype=torch.int32, device=device)
    fnd = torch.empty(N_SEARCH, dtype=torch.uint8, device=device)

    def best(fn):
        return min(_time_ms(fn, stream, flush) for _ in range(reps))

    def build():
        sh.slab_reset(h, stream)
        sh.slab_insert_batch(h, kb, vb, None, stream=stream)
    ms_build = best(build)  # includes the reset fill
    with torch.cuda.stream(stream):
        sh.slab_reset(h, stream)
        sh.slab_insert_batch(h, kb, vb, None, stream=stream)
    torch.cuda.synchronize()
    tot = t.stats()
    util = 8.0 * tot["live"] / (float(slab_bytes) * tot["slabs"])
    rates = {}
    for hr, q in queries.items():
        dq = dev(q)
        ms = best(lambda: sh.slab_search_batch(h, dq, out, fnd, stream=stream))
        rates[f"search_{int(hr * 100)}"] = round(N_SEARCH / (ms * 1e3), 1)
    ms_del = []
    for _ in range(reps):
        with torch.cuda.stream(stream):
            sh.slab_reset(h, stream)
            sh.slab_insert_batch(h, kb, vb, None, stream=stream)
        ms_del.append(_time_ms(lambda: sh.slab_delete_batch(h, kd, None, stream=stream), stream, flush))
    rc, flags = t.status(stream)
    t.close()
    line = {"beta": beta, "num_buckets": w.num_buckets, "unit": "Mops/s",
            "build_incl_reset": round(N_KEYS / (ms_build * 1e3), 1), **rates,
            "delete": round(N_DELETE / (min(ms_del) * 1e3), 1), "utilization": round(util, 4),
            "slabs_per_bucket": round(tot["slabs"] / w.num_buckets, 4), "status": rc}
    return line, (w, queries)


def bulk_oracle_lines(w, queries, slab_bytes=128):
    """The oracle's slab reads per op for bulk_point's batches."""
    from oracle import OracleTable
    o = OracleTable(w.num_buckets, w.hash_a, w.hash_b, slab_bytes=slab_bytes)
    o.insert(w.keys, w.values)
    out = {"build_incl_reset": o.lines / N_KEYS}
    for hr, q in queries.items():
        o.lines = 0
        o.search(q)
        out[f"search_{int(hr * 100)}"] = o.lines / N_SEARCH
    o.lines = 0
    o.delete(w.delete_keys)
    out["delete"] = o.lines / N_DELETE
    o.close()
    return out


def mixed_series(args, device, stream, flush, ratios, batches=64):
    """The concurrent benchmark (Sec. 6.3) at one ratio: preload 2^22 pairs (beta
    0.6), then `batches` batches of 2^20 mixed ops, each timed alone after an L2
    flush; tombstones accumulate (no flush of the table). Returns (rates, host
    inputs for the oracle)."""
    import torch

    from paper_1710_11246_gb300 import slabhash as sh
    dev = sh.as_device_u32
    w = W.config2(BETA, HIT, args.seed)
    ks = W.KeyStream(args.seed)
    ks.take(N_KEYS + N_SEARCH)
    rng = np.random.default_rng([args.seed, 0xC0C0])
    live = w.keys
    host_batches, dev_batches = [], []
    for _ in range(batches):
        mb, live = W.mixed_batch(ks, live, N_MIXED, ratios, rng)
        host_batches.append(mb)
        dev_batches.append((torch.from_numpy(mb.ops).to(device), dev(mb.keys), dev(mb.values)))
    t = sh.SlabHash(w.num_buckets, w.hash_a, w.hash_b, 1 << 22)
    h = t.handle
    res = torch.empty(N_MIXED, dtype=torch.int32, device=device)
    with torch.cuda.stream(stream):
        sh.slab_insert_batch(h, dev(w.keys), dev(w.values), None, stream=stream)
    torch.cuda.synchronize()
    ms = []
    for ops, keys, vals in dev_batches:
        ms.append(_time_ms(lambda: sh.slab_mixed_batch(h, ops, keys, vals, res, None, stream=stream),
                           stream, flush))
    rc, flags = t.status(stream)
    tot = t.stats()
    t.close()
    line = {"ratios": ratios, "batches": batches, "batch_ops": N_MIXED, "unit": "Mops/s",
            "mean": round(batches * N_MIXED / (sum(ms) * 1e3), 1),
            "first_batch": round(N_MIXED / (ms[0] * 1e3), 1),
            "last_batch": round(N_MIXED / (ms[-1] * 1e3), 1),
            "final_slabs_per_bucket": round(tot["slabs"] / w.num_buckets, 4), "status": rc}
    return line, (w, host_batches, ms)


def mixed_oracle_lines(w, host_batches):
    """The oracle's slab reads per op, batch by batch, for mixed_series' batches."""
    from oracle import OracleTable
    o = OracleTable(w.num_buckets, w.hash_a, w.hash_b)
    o.insert(w.keys, w.values)
    per = []
    for mb in host_batches:
        o.lines = 0
        o.mixed(mb.ops, mb.keys, mb.values)
        per.append(o.lines / len(mb.keys))
    o.close()
    return per


def slaballoc_sweep(device, stream, flush, reps):
    """SlabAlloc microbenchmark (Sec. 5), printed as a sweep line."""
    print(json.dumps({"sweep": "slaballoc", **slaballoc_point(device, stream, flush, reps)}), flush=True)


def slaballoc_point(device, stream, flush, reps):
    """SlabAlloc microbenchmark (Sec. 5): 2^24 single-slab allocations (one per lane,
    batched and one at a time), 2^24 frees, against a random 32-bit atomicOr probe
    on a bitmap region of the same size."""
    import torch

    from paper_1710_11246_gb300 import slabhash as sh
    dev = sh.as_device_u32

    # SlabAlloc: 2^24 single-slab allocations (one per lane), then 2^24 frees
    n = 1 << 24
    t = sh.SlabHash(8, 3, 4, 1 << 25)
    addrs = torch.empty(n, dtype=torch.int32, device=device)
    a_ms, f_ms, a1_ms = [], [], []
    for _ in range(reps):
        with torch.cuda.stream(stream):
            sh.slab_reset(t.handle, stream)
        a_ms.append(_time_ms(lambda: sh.slab_alloc_batch(t.handle, addrs, stream=stream), stream, flush))
        f_ms.append(_time_ms(lambda: sh.slab_free_batch(t.handle, addrs, stream=stream), stream, flush))
    # the paper's warp serves its requests one at a time (direct variant)
    t.configure(variant=sh.SLAB_VARIANT_DIRECT)
    for _ in range(reps):
        with torch.cuda.stream(stream):
            sh.slab_reset(t.handle, stream)
        a1_ms.append(_time_ms(lambda: sh.slab_alloc_batch(t.handle, addrs, stream=stream), stream, flush))
        sh.slab_free_batch(t.handle, addrs, stream=stream)
    t.configure(variant=sh.SLAB_VARIANT_STAGED)
    rc, flags = t.status(stream)
    bm_zero = bool((t.bitmaps() == 0).all().item())
    # allocator ceiling: random 32-bit atomicOr on a bitmap region of the same size
    words = (1 << 25) // 32
    bm = torch.zeros(words, dtype=torch.int32, device=device)
    or_rate = 0.0
    for oif in (2, 4, 8):
        ms = []
        for rep in range(3):
            bm.zero_()
            ms.append(_time_ms(lambda: sh.slab_probe_random_or(bm, words, n, rep + 1, oif, 512, stream=stream),
                               stream, flush))
        or_rate = max(or_rate, n / (min(ms) * 1e-3))
    del bm
    t.close()
    del addrs
    return {"allocations": n, "pool_slabs": 1 << 25, "unit": "Mops/s",
            "alloc": round(n / (min(a_ms) * 1e3), 1), "free": round(n / (min(f_ms) * 1e3), 1),
            "alloc_one_at_a_time": round(n / (min(a1_ms) * 1e3), 1),
            "random_atomic_or_bitmap": round(or_rate / 1e6, 1),
            "alloc_frac_of_atomic_rate": round(n / (min(a_ms) * 1e-3) / or_rate, 4),
            "status": rc, "bitmaps_clear_after_free": bm_zero}



def learned_sweep(args, device, stream, flush):
    """Learned bucket function vs the universal hash on clustered keys."""
    import torch

    from paper_1710_11246_gb300 import slabhash as sh
    dev = sh.as_device_u32

    # learned bucket function vs universal hash on clustered keys (2^22, beta = 0.6)
    w = W.config4(seed=args.seed)
    kb, vb, kq = dev(w.keys), dev(w.values), dev(w.search.keys)
    out = torch.empty(N_SEARCH, dtype=torch.int32, device=device)
    fnd = torch.empty(N_SEARCH, dtype=torch.uint8, device=device)
    line = {"sweep": "learned", "keys": len(w.keys), "clusters": 64, "num_buckets": w.num_buckets,
            "sample_stride": 100, "unit": "Mops/s"}
    for label, policy in (("universal", sh.SLAB_LEARN_MEASURE), ("learned", sh.SLAB_LEARN_ALWAYS)):
        t = sh.SlabHash(w.num_buckets, w.hash_a, w.hash_b, 1 << 21)
        h = t.handle
        fit_ms = _time_ms(lambda: sh.slab_learn_buckets(h, kb, 100, policy, stream=stream), stream, flush)
        rep = sh.slab_learn_buckets(h, kb, 100, policy, stream=stream)
        with torch.cuda.stream(stream):
            sh.slab_insert_batch(h, kb, vb, None, stream=stream)
        torch.cuda.synchronize()
        _, slabs, tot = t.stats(per_bucket=True)
        hist = np.bincount(np.minimum(sh.to_host_u32(slabs), 16)).tolist()
        ms = min(_time_ms(lambda: sh.slab_search_batch(h, kq, out, fnd, stream=stream), stream, flush)
                 for _ in range(5))
        rc, _ = t.status(stream)
        line[label] = {"search_50": round(N_SEARCH / (ms * 1e3), 1), "fit_ms": round(fit_ms, 3),
                       "mean_slabs": round(tot["slabs"] / w.num_buckets, 4), "max_slabs": int(max(
                           np.flatnonzero(np.bincount(sh.to_host_u32(slabs))))),
                       "slabs_histogram_1_to_16plus": hist[1:], "status": rc}
        line["report"] = rep
        t.close()
    print(json.dumps(line), flush=True)



def group_sweep(args, device, stream, flush):
    """Groups of tables: per-table launches, one group launch, CUDA graph, autotuned."""
    import torch

    from paper_1710_11246_gb300 import slabhash as sh
    dev = sh.as_device_u32

    # 512 independent tables, sizes log-uniform in [2^8, 2^18]: per-table launches vs
    # one group launch per batch vs the group step replayed from a CUDA graph, and the
    # autotuned group configuration
    from paper_1710_11246_gb300 import autotune as AT
    gw = W.group_workload(512, 1 << 8, 1 << 18, seed=args.seed)
    ops = 2 * int(gw.sizes.sum())
    arrays = AT._arrays(gw, device)
    gout = torch.empty(len(gw.search_keys), dtype=torch.int32, device=device)
    gfnd = torch.empty(len(gw.search_keys), dtype=torch.uint8, device=device)
    g = AT.create_group(gw, BETA)
    line = {"sweep": "group", "tables": 512, "keys": int(gw.sizes.sum()), "ops_per_step": ops,
            "sizes": "log-uniform [2^8, 2^18]", "unit": "Mops/s"}
    ms = AT.time_group(g, arrays, gout, gfnd, stream)
    line["group_launch"] = round(ops / (ms * 1e3), 1)
    # the same step as 2 x 512 single-table launches through the tables' own handles
    views = [sh.slab_group_table(g, i) for i in range(512)]
    st, ks, vs, qs, q = arrays
    o, so = gw.op_start.tolist(), gw.search_start.tolist()

    def per_table():
        sh.slab_group_reset(g, stream)
        for i, t in enumerate(views):
            if o[i + 1] > o[i]:
                sh.slab_insert_batch(t, ks[o[i]:o[i + 1]], vs[o[i]:o[i + 1]], None, stream=stream)
        for i, t in enumerate(views):
            if so[i + 1] > so[i]:
                sh.slab_search_batch(t, q[so[i]:so[i + 1]], gout[so[i]:so[i + 1]], gfnd[so[i]:so[i + 1]],
                                     stream=stream)
    per_table()
    torch.cuda.synchronize()
    ms_pt = min(_time_ms(per_table, stream, flush) for _ in range(3))
    line["per_table_launches"] = round(ops / (ms_pt * 1e3), 1)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        AT.group_step(g, arrays, gout, gfnd, stream)
    graph.replay()
    torch.cuda.synchronize()
    ms_gr = min(_time_ms(graph.replay, stream, flush) for _ in range(5))
    line["group_cuda_graph"] = round(ops / (ms_gr * 1e3), 1)
    rc, _ = sh.slab_group_status(g, stream)
    line["status"] = rc
    sh.slab_group_destroy(g)
    g64 = AT.create_group(gw, BETA, 64)
    line["group_launch_64B_slabs"] = round(ops / (AT.time_group(g64, arrays, gout, gfnd, stream) * 1e3), 1)
    sh.slab_group_destroy(g64)
    best, cands = AT.tune_group(gw, device=device)
    line["autotuned"] = {"slab_bytes": best.slab_bytes, "beta": best.beta,
                         "threads_per_block": best.threads_per_block,
                         "blocks_per_sm": best.blocks_per_sm, "mops": round(best.mops, 1),
                         "candidates": len(cands),
                         "best_per_width": {w: round(max(c.mops for c in cands if c.slab_bytes == w), 1)
                                            for w in sorted({c.slab_bytes for c in cands})},
                         "worst_mops": round(min(c.mops for c in cands), 1)}
    print(json.dumps(line), flush=True)



def serving_sweep(args, device, stream, flush):
    """Serving loop on one resident 2^26-pair table (beta = 0.6, universal hash):
    requests of log-uniform size 1..2^16 with ops (0.1, 0.1, 0.8), admitted by free
    SlabAlloc memory, overlapped on the server's slot streams. Lines: throughput at
    saturation (every request queued at time 0) per slot count, p50 / p99 latency
    under Poisson arrivals at fractions of the 8-slot saturation rate, and the plain
    slab hash on the same ops as one mixed batch."""
    import torch

    from paper_1710_11246_gb300 import slabhash as sh
    dev = sh.as_device_u32
    R = SERVING_REQUESTS
    tr = W.serving_trace(SERVING_KEYS, R, None, seed=args.seed)
    total = int(tr.op_start[-1])
    t = sh.SlabHash(tr.num_buckets, tr.hash_a, tr.hash_b, SERVING_POOL)
    kb, vb = dev(tr.preload), dev(W.values_for(tr.preload))

    def load():
        with torch.cuda.stream(stream):
            sh.slab_reset(t.handle, stream)
            sh.slab_insert_batch(t.handle, kb, vb, None, stream=stream)
        torch.cuda.synchronize()

    h_ops, h_keys, h_vals = (sh.pinned_copy(a) for a in (tr.ops, tr.keys, tr.values))

    def serve(slots, arrival, flags):
        load()
        sv = sh.slab_server_create(t.handle, slots, SERVING_SLOT_OPS, flags=flags)
        try:
            out = sh.slab_server_run(sv, arrival, tr.op_start, h_ops, h_keys, h_vals, pinned_outputs=True)
            st = sh.slab_server_get_stats(sv)
        finally:
            sh.slab_server_destroy(sv)
        rc, _ = t.status()
        return out, st, rc

    line = {"sweep": "serving", "table_pairs": SERVING_KEYS, "num_buckets": tr.num_buckets,
            "slot_ops": SERVING_SLOT_OPS,
            "pool_slabs": t.info.pool_slabs, "requests": R, "ops": total, "ratios": [0.1, 0.1, 0.8],
            "sizes": "log-uniform [1, 2^16]", "unit": "Mops/s"}
    # the plain slab hash: the trace's ops as one mixed batch, inputs resident
    ops_d, keys_d, vals_d = torch.from_numpy(tr.ops).to(device), dev(tr.keys), dev(tr.values)
    res = torch.empty(total, dtype=torch.int32, device=device)
    plain = []
    for _ in range(3):
        load()
        plain.append(_time_ms(lambda: sh.slab_mixed_batch(t.handle, ops_d, keys_d, vals_d, res, None,
                                                          stream=stream), stream, flush))
    line["plain_one_batch"] = round(total / (min(plain) * 1e3), 1)
    del ops_d, keys_d, vals_d, res
    zero = np.zeros(R, np.uint64)
    modes = {"copy": 0, "zero_copy": sh.SLAB_SERVER_ZERO_COPY}
    sat = {}
    for mode, flags in modes.items():
        serve(8, zero, flags)  # warm-up
        for slots in (1, 2, 4, 8, 16):
            out, st, rc = serve(slots, zero, flags)
            sat[(mode, slots)] = (out["makespan_ns"], rc, st["batches"])
    line["saturated"] = {m: {str(k): round(total / v[0] * 1e3, 1) for (mm, k), v in sat.items() if mm == m}
                         for m in modes}
    line["saturated_batches"] = {m: {str(k): v[2] for (mm, k), v in sat.items() if mm == m} for m in modes}
    mode = max(modes, key=lambda m: total / sat[(m, 8)][0])
    rate8 = R / (sat[(mode, 8)][0] * 1e-9)
    line["poisson_mode"] = mode
    line["saturated_requests_per_s_8_slots"] = round(rate8)
    rng = np.random.default_rng([args.seed, 0x9015])
    gaps = rng.exponential(1.0, R)
    line["poisson_8_slots"] = []
    for frac in (0.01, 0.1, 0.5, 0.8):
        rate = frac * rate8
        arrival = np.floor(np.cumsum(gaps) * (1e9 / rate)).astype(np.uint64)
        out, st, rc = serve(8, arrival, modes[mode])
        lat, wait = out["latency_ns"] / 1e3, out["wait_ns"] / 1e3
        line["poisson_8_slots"].append({
            "load": frac, "offered_requests_per_s": round(rate), "mops": round(total / out["makespan_ns"] * 1e3, 1),
            "p50_us": round(float(np.percentile(lat, 50)), 1), "p99_us": round(float(np.percentile(lat, 99)), 1),
            "wait_p50_us": round(float(np.percentile(wait, 50)), 1),
            "wait_p99_us": round(float(np.percentile(wait, 99)), 1),
            "requests_per_batch": round(R / st["batches"], 2),
            "deferred_slot": st["deferred_slot"], "deferred_memory": st["deferred_memory"],
            "status": rc, "all_served": bool((out["status"] == 0).all())})
    line["status"] = max(v[1] for v in sat.values())
    print(json.dumps(line), flush=True)
    t.close()


def flush_sweep(args, device, stream, flush):
    """FLUSH (Sec. 4.3.4) after tombstones pile up: preload 2^22 pairs (beta 0.6),
    churn with 32 mixed batches of 2^20 ops at (0.5, 0.5, 0) (every delete leaves a
    tombstone, every insert takes a new slot), then time search (2^22 at 50 % hit)
    and one more churn batch before and after one flush of the whole table."""
    import torch

    from paper_1710_11246_gb300 import slabhash as sh
    dev = sh.as_device_u32
    w = W.config2(BETA, HIT, args.seed)
    ks = W.KeyStream(args.seed)
    ks.take(N_KEYS + N_SEARCH)
    rng = np.random.default_rng([args.seed, 0xF1])
    t = sh.SlabHash(w.num_buckets, w.hash_a, w.hash_b, 1 << 22)
    h = t.handle
    with torch.cuda.stream(stream):
        sh.slab_insert_batch(h, dev(w.keys), dev(w.values), None, stream=stream)
    live = w.keys
    res = torch.empty(N_MIXED, dtype=torch.int32, device=device)
    churn_ms = []
    for _ in range(33):
        mb, live = W.mixed_batch(ks, live, N_MIXED, (0.5, 0.5, 0.0), rng)
        o, k, v = torch.from_numpy(mb.ops).to(device), dev(mb.keys), dev(mb.values)
        churn_ms.append(_time_ms(lambda: sh.slab_mixed_batch(h, o, k, v, res, None, stream=stream), stream, flush))
    # search keys: half live, half absent
    q = np.concatenate([live[rng.permutation(len(live))[: N_SEARCH // 2]], ks.take(N_SEARCH // 2)])
    dq = dev(q[rng.permutation(N_SEARCH)])
    out = torch.empty(N_SEARCH, dtype=torch.int32, device=device)
    search_before = min(_time_ms(lambda: sh.slab_search_batch(h, dq, out, None, stream=stream), stream, flush)
                        for _ in range(3))
    before = t.stats()
    flush_ms = _time_ms(lambda: sh.slab_flush(h, stream, wait=False), stream, flush)
    after = t.stats()
    search_after = min(_time_ms(lambda: sh.slab_search_batch(h, dq, out, None, stream=stream), stream, flush)
                       for _ in range(3))
    mb, live = W.mixed_batch(ks, live, N_MIXED, (0.5, 0.5, 0.0), rng)
    o, k, v = torch.from_numpy(mb.ops).to(device), dev(mb.keys), dev(mb.values)
    churn_after = _time_ms(lambda: sh.slab_mixed_batch(h, o, k, v, res, None, stream=stream), stream, flush)
    rc, _ = t.status(stream)
    line = {"sweep": "flush", "keys": N_KEYS, "num_buckets": w.num_buckets, "churn_batches": 32,
            "churn_ops": N_MIXED, "unit": "Mops/s",
            "slabs_per_bucket_before": round(before["slabs"] / w.num_buckets, 3),
            "slabs_per_bucket_after": round(after["slabs"] / w.num_buckets, 3),
            "slabs_released": before["slabs"] - after["slabs"], "live": after["live"],
            "flush_ms": round(flush_ms, 3), "flush_buckets_per_s": round(w.num_buckets / (flush_ms * 1e-3)),
            "search_50_before": round(N_SEARCH / (search_before * 1e3), 1),
            "search_50_after": round(N_SEARCH / (search_after * 1e3), 1),
            "churn_first_batch": round(N_MIXED / (churn_ms[0] * 1e3), 1),
            "churn_batch_before_flush": round(N_MIXED / (churn_ms[-1] * 1e3), 1),
            "churn_batch_after_flush": round(N_MIXED / (churn_after * 1e3), 1), "status": rc}
    print(json.dumps(line), flush=True)
    t.close()


def sizes_sweep(args, device, stream, flush):
    """Rates against table size at a fixed mean of 0.6 slabs per bucket (about 55 %
    memory utilization, the paper's bulk benchmark over table sizes, Sec. 6.1):
    build, search at 0 % and 100 % hit, n = 2^16 .. 2^24."""
    import torch

    from paper_1710_11246_gb300 import slabhash as sh
    dev = sh.as_device_u32
    rows = []
    for lg in (16, 18, 20, 22, 24):
        n = 1 << lg
        ks = W.KeyStream(args.seed + lg)
        keys = ks.take(n)
        absent = ks.take(n)
        rng = np.random.default_rng([args.seed, lg])
        B = W.buckets_for(n, BETA)
        a, b = W.hash_params(args.seed + lg)
        t = sh.SlabHash(B, a, b, max(1024, n // 8))
        h = t.handle
        kb, vb, kq, ka = dev(keys), dev(W.values_for(keys)), dev(keys[rng.permutation(n)]), dev(absent)
        out = torch.empty(n, dtype=torch.int32, device=device)

        def build():
            sh.slab_reset(h, stream)
            sh.slab_insert_batch(h, kb, vb, None, stream=stream)
        ms_b = min(_time_ms(build, stream, flush) for _ in range(3))
        with torch.cuda.stream(stream):
            build()
        ms_hit = min(_time_ms(lambda: sh.slab_search_batch(h, kq, out, None, stream=stream), stream, flush)
                     for _ in range(3))
        ms_miss = min(_time_ms(lambda: sh.slab_search_batch(h, ka, out, None, stream=stream), stream, flush)
                      for _ in range(3))
        rc, _ = t.status(stream)
        tot = t.stats()
        rows.append({"n": n, "num_buckets": B, "build_incl_reset": round(n / (ms_b * 1e3), 1),
                     "search_100": round(n / (ms_hit * 1e3), 1), "search_0": round(n / (ms_miss * 1e3), 1),
                     "utilization": round(8.0 * tot["live"] / (128.0 * tot["slabs"]), 4), "status": rc})
        t.close()
    print(json.dumps({"sweep": "sizes", "beta": BETA, "unit": "Mops/s", "rows": rows}), flush=True)


def incremental_sweep(args, device, stream, flush):
    """Incremental insertion (the slab hash's half of the paper's Sec. 6.2
    experiment): 2^21 elements inserted in batches of 2^15, 2^16 or 2^17 into a table
    sized for the final count (beta 0.6); mean insert rate over the batches."""
    import torch

    from paper_1710_11246_gb300 import slabhash as sh
    dev = sh.as_device_u32
    total = 1 << 21
    keys = W.KeyStream(args.seed + 99).take(total)
    B = W.buckets_for(total, BETA)
    a, b = W.hash_params(args.seed + 99)
    kb, vb = dev(keys), dev(W.values_for(keys))
    t = sh.SlabHash(B, a, b, 1 << 18)
    h = t.handle
    line = {"sweep": "incremental", "elements": total, "num_buckets": B, "unit": "Mops/s",
            "launch": "the batches replayed from one CUDA graph (host launch cost excluded)"}
    with torch.cuda.stream(stream):  # warm-up: the launch path caches its occupancy query
        sh.slab_insert_batch(h, kb[:32], vb[:32], None, n=32, stream=stream)
    torch.cuda.synchronize()
    for lg in (15, 16, 17):
        bs = 1 << lg
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            for i in range(0, total, bs):
                sh.slab_insert_batch(h, kb[i:i + bs], vb[i:i + bs], None, n=bs, stream=stream)
        with torch.cuda.stream(stream):
            sh.slab_reset(h, stream)
            flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            graph.replay()
            e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        rc, _ = t.status(stream)
        line[f"batch_{bs}"] = {"batches": total // bs, "mops": round(total / (ms * 1e3), 1), "status": rc}
    tot = t.stats()
    line["live"] = tot["live"]
    print(json.dumps(line), flush=True)
    t.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--variant", default="staged", choices=["staged", "direct"])
    ap.add_argument("--threads-per-block", type=int, default=0)
    ap.add_argument("--blocks-per-sm", type=int, default=None)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-probe", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="leave out the config-2 / config-3 / 64-byte keys of the step line")
    ap.add_argument("--sweep", nargs="?", const="all", default=None,
                    choices=["all", "bulk", "slaballoc", "learned", "group", "serving", "flush", "sizes", "incremental",
                             "mixed"],
                    help="print the sweep lines (all, or one section) instead of the step line")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        return reference_arm(args, rank, world)

    import torch
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if args.sweep:
        return sweep(args, device)
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=device)

    r = gpu_arm(args, rank, world, device)
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    ms_step = r["total_ms"] / args.steps
    value = job_value(ms_step, world)  # Mops/s over all ranks
    mean = {p: statistics.fmean(v) for p, v in r["per_phase"].items()}
    ops = {"build": N_KEYS, "search": N_SEARCH, "delete": N_DELETE, "mixed": N_MIXED}
    per_op = {p: round(ops[p] / (mean[p] * 1e3), 1) for p in ops}

    cpu = None
    lines = linked = None
    if world == 1 and not args.no_cpu_baseline:
        cpu, (lines, linked), _ = cpu_baseline(r["w"], r["mb"])

    # Algorithmic bytes per batch: 128 B per slab the ops must read (the oracle's line
    # count of this workload), the 8 B pair CAS of every insert, 4 B bitmap claim and
    # 4 B link CAS per slab linked, the 4 B tombstone store of every delete hit, and
    # each op's own input / output bytes.
    n_ins_mixed = int((r["mb"].ops == W.OP_INSERT).sum())
    n_del_mixed = int((r["mb"].ops == W.OP_DELETE).sum())
    io = {"build": 8, "search": 4 + 4 + 1, "delete": 4 + 1, "mixed": 1 + 4 + 4 + 4 + 1}
    cas_ops = {"build": N_KEYS, "search": 0, "delete": 0, "mixed": n_ins_mixed}
    stores = {"build": 0, "search": 0, "delete": N_DELETE, "mixed": n_del_mixed}
    dom = r["dom"]  # dominant kernel, timed live in the timed pass
    dom_mean = statistics.fmean(r["dom_ms"])
    roof = None
    rl = None
    if lines is not None:
        alg = {p: 128 * lines[p] + 8 * cas_ops[p] + 8 * linked[p] + 4 * stores[p] + io[p] * ops[p] for p in ops}
        peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"] \
            if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0
        achieved = alg[dom] / (dom_mean * 1e-3) / 1e9
        traffic = ncu_traffic(dom) if args.variant == "staged" else None
        hbm_view = {"achieved": round(achieved, 1), "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                    "note": "the table is L2-resident: most of these bytes come from L2, not HBM"}
        roof = {"bound": "hbm", "kernel": f"{dom} ({args.variant}_kernel)", "achieved": round(achieved, 1),
                "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": traffic,
                "algorithmic_bytes": alg[dom], "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                "lines_per_op": {p: round(lines[p] / ops[p], 4) for p in ops}}
        if not args.no_probe:
            fp = r["table"].info.num_buckets * 128
            rate, cfg = random_line_probe(device, fp)
            rate_big, cfg_big = random_line_probe(device, 4 << 30)
            cas_rate, cas_cfg = random_cas_probe(device, fp)
            # CAS per op the method must issue: one pair claim per insert; deletes
            # store a tombstone and searches only read
            cas_per_op = {p: cas_ops[p] / ops[p] for p in ops}
            bound = {p: min(rate / (lines[p] / ops[p]),
                            cas_rate / cas_per_op[p] if cas_per_op[p] else float("inf")) for p in ops}
            frac_lc = {p: ops[p] / (mean[p] * 1e-3) / bound[p] for p in ops}
            rl = {"footprint_bytes": fp, "glines_per_s": round(rate / 1e9, 3), "probe": cfg,
                  "glines_per_s_4GiB": round(rate_big / 1e9, 3), "probe_4GiB": cfg_big,
                  "gcas_per_s": round(cas_rate / 1e9, 3), "cas_probe": cas_cfg, "cas_per_op": cas_per_op,
                  "per_phase_frac": {p: round(lines[p] / (mean[p] * 1e-3) / rate, 4) for p in ops},
                  "per_phase_bound_gops": {p: round(bound[p] / 1e9, 2) for p in ops},
                  "per_phase_frac_line_cas": {p: round(frac_lc[p], 4) for p in ops}}
            # The ceiling the dominant kernel runs against is the random-line / CAS
            # rate at the table's footprint (the table lives in L2), expressed in the
            # kernel's algorithmic bytes: peak = bound ops/s x bytes per op.
            bpo = alg[dom] / ops[dom]
            lc_peak = bound[dom] * bpo / 1e9
            lc_achieved = ops[dom] / (dom_mean * 1e-3) * bpo / 1e9
            roof = {"bound": "random-line/CAS", "kernel": f"{dom} ({args.variant}_kernel)",
                    "achieved": round(lc_achieved, 1), "peak": round(lc_peak, 1), "unit": "GB/s",
                    "frac": round(lc_achieved / lc_peak, 4), "traffic": traffic, "algorithmic_bytes": alg[dom],
                    "peak_source": "min(random 128 B line rate / lines per op, random 64-bit CAS rate / CAS per op),"
                                   " both probed live at the table's footprint (of measured)",
                    "lines_per_op": {p: round(lines[p] / ops[p], 4) for p in ops},
                    "hbm_view": hbm_view}
    sweeps = None
    if world == 1 and rl is not None and not args.no_extras:
        sweeps = extras(args, device, (rl["glines_per_s"] * 1e9, rl["gcas_per_s"] * 1e9))
    out = {
        "metric": METRIC, "value": round(value, 1), "unit": "Mops/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": config_dict({"variant": args.variant}),
        "per_op_mops": per_op, "phase_ms": {p: round(mean[p], 4) for p in PHASES},
        "per_op_source": "instrumented pass: CUDA events between every phase, K steps after the timed ones",
        "dominant_kernel_ms_timed": round(dom_mean, 4),
        "roofline": roof, "random_line_roofline": rl, "cpu_baseline": cpu,
        "e2e": r["e2e"], "gpu_launches": 5 * args.steps, "clocks": r["clocks"], "sweeps": sweeps,
    }
    print(json.dumps(out))
    r["table"].close()
    if world > 1:
        torch.distributed.destroy_process_group()


def width_step(args, device, slab_bytes):
    """The benchmark step (reset, build, search, delete, mixed) on a table of
    `slab_bytes` slabs at the same beta (B = ceil(n / (M beta)) with M pairs per
    slab), L2 flushed before every step, CUDA events between phases, K steps after
    W warm-up steps. Returns (per-phase results, host inputs for the oracle)."""
    import torch

    from paper_1710_11246_gb300 import slabhash as sh
    per = (slab_bytes // 4 - 2) // 2
    w, mb = make_step_inputs(args.seed, per_slab=per)
    dev = sh.as_device_u32
    t = sh.SlabHash(w.num_buckets, w.hash_a, w.hash_b, POOL_SLABS, slab_bytes=slab_bytes)
    h = t.handle
    stream = torch.cuda.Stream()
    k_build, v_build, k_search, k_del = dev(w.keys), dev(w.values), dev(w.search.keys), dev(w.delete_keys)
    m_ops, m_keys, m_vals = torch.from_numpy(mb.ops).to(device), dev(mb.keys), dev(mb.values)
    o_search = torch.empty(N_SEARCH, dtype=torch.int32, device=device)
    f_search = torch.empty(N_SEARCH, dtype=torch.uint8, device=device)
    f_del = torch.empty(N_DELETE, dtype=torch.uint8, device=device)
    o_mixed = torch.empty(N_MIXED, dtype=torch.int32, device=device)
    f_mixed = torch.empty(N_MIXED, dtype=torch.uint8, device=device)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    calls = (lambda: sh.slab_reset(h, stream),
             lambda: sh.slab_insert_batch(h, k_build, v_build, None, stream=stream),
             lambda: sh.slab_search_batch(h, k_search, o_search, f_search, stream=stream),
             lambda: sh.slab_delete_batch(h, k_del, f_del, stream=stream),
             lambda: sh.slab_mixed_batch(h, m_ops, m_keys, m_vals, o_mixed, f_mixed, stream=stream))
    all_evs = []
    with torch.cuda.stream(stream):
        for i in range(args.warmup + args.steps):
            flush.zero_()
            evs = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
            for j, c in enumerate(calls):
                evs[j].record(stream)
                c()
            evs[5].record(stream)
            if i >= args.warmup:
                all_evs.append(evs)
    torch.cuda.synchronize()
    rc, flags = t.status(stream)
    if rc != sh.SLAB_OK:
        raise RuntimeError(f"{slab_bytes}-byte step: device status rc={rc} flags={flags}")
    ok = int(f_search.sum().item()) == int(w.search.present.sum()) and bool((f_del == 1).all().item())
    t.close()
    mean = {p: statistics.fmean(e[i].elapsed_time(e[i + 1]) for e in all_evs) for i, p in enumerate(PHASES)}
    ops = {"build": N_KEYS, "search": N_SEARCH, "delete": N_DELETE, "mixed": N_MIXED}
    res = {"slab_bytes": slab_bytes, "pairs_per_slab": per, "num_buckets": w.num_buckets, "beta": BETA,
           "steps": args.steps, "per_op_mops": {p: round(ops[p] / (mean[p] * 1e3), 1) for p in ops},
           "phase_ms": {p: round(mean[p], 4) for p in PHASES}, "results_checked": ok}
    return res, (w, mb)


def line_cas_fracs(rates_mops, lines_per_op, cas_per_op, line_rate, cas_rate):
    """Each phase's rate as a fraction of min(line rate / lines per op, CAS rate / CAS per op)."""
    out = {}
    for p, r in rates_mops.items():
        if p not in lines_per_op:
            continue
        bound = min(line_rate / lines_per_op[p], cas_rate / cas_per_op[p] if cas_per_op.get(p) else float("inf"))
        out[p] = round(r * 1e6 / bound, 4)
    return out


def extras(args, device, main_rates):
    """Configs 2 and 3 and the 64-byte slab width as keys of the step's line: the
    bulk benchmark over beta at 0 / 50 / 100 % hit (Sec. 6.1), the SlabAlloc
    microbenchmark (Sec. 5), 64 concurrent batches at each ratio (Sec. 6.3) and the
    step on 64-byte slabs, each figure with its fraction of the random-line / CAS
    bound at its table's footprint. The oracle's line counts run in threads beside
    the GPU work (the C oracle releases the interpreter lock)."""
    import torch
    from concurrent.futures import ThreadPoolExecutor
    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    ex = ThreadPoolExecutor(max_workers=max(2, min(8, (os.cpu_count() or 4) - 1)))
    t0 = time.perf_counter()

    bulk = []
    for beta in W.CONFIG2_BETAS:
        line, (w, queries) = bulk_point(args, device, stream, flush, beta, reps=3)
        fut = ex.submit(bulk_oracle_lines, w, queries)
        fp = w.num_buckets * 128
        lr, _ = random_line_probe(device, fp, quick=True)
        cr, _ = random_cas_probe(device, fp, quick=True)
        bulk.append((line, fut, lr, cr))
    slaballoc = slaballoc_point(device, stream, flush, 3)
    series = []
    for ratios in W.CONFIG3_RATIOS:
        line, (w, hb, ms) = mixed_series(args, device, stream, flush, ratios)
        ins = [float((mb.ops == W.OP_INSERT).mean()) for mb in hb]
        series.append((line, ex.submit(mixed_oracle_lines, w, hb), ins, ms))
    s64, (w64, mb64) = width_step(args, device, 64)
    fut64 = ex.submit(run_oracle_step, w64, mb64, 64)
    lr64, cfg64 = random_line_probe(device, w64.num_buckets * 64, line_bytes=64, quick=True)
    cr64, _ = random_cas_probe(device, w64.num_buckets * 64, quick=True)

    out = {"config2_beta_sweep": [], "slaballoc_2e24": slaballoc, "config3_concurrent": []}
    for line, fut, lr, cr in bulk:
        lines = fut.result()
        rates = {k: line[k] for k in lines}
        line["lines_per_op"] = {k: round(v, 4) for k, v in lines.items()}
        line["glines_per_s"], line["gcas_per_s"] = round(lr / 1e9, 2), round(cr / 1e9, 2)
        line["frac_line_cas"] = line_cas_fracs(rates, lines, {"build_incl_reset": 1.0}, lr, cr)
        out["config2_beta_sweep"].append(line)
    lr3, cr3 = main_rates
    for line, fut, ins, ms in series:
        per = fut.result()
        fr = []
        for lpo, fi, m in zip(per, ins, ms):
            bound = min(lr3 / lpo, cr3 / fi if fi else float("inf"))
            fr.append(N_MIXED / (m * 1e-3) / bound)
        line["lines_per_op_first_last"] = [round(per[0], 4), round(per[-1], 4)]
        line["frac_line_cas"] = {"mean": round(statistics.fmean(fr), 4), "first_batch": round(fr[0], 4),
                                 "last_batch": round(fr[-1], 4)}
        out["config3_concurrent"].append(line)
    _, lines64, _ = fut64.result()
    ops = {"build": N_KEYS, "search": N_SEARCH, "delete": N_DELETE, "mixed": N_MIXED}
    lpo64 = {p: lines64[p] / ops[p] for p in ops}
    cas64 = {"build": 1.0, "mixed": float((mb64.ops == W.OP_INSERT).mean())}
    s64["lines_per_op"] = {p: round(v, 4) for p, v in lpo64.items()}
    s64["random_64B_line_roofline"] = {"footprint_bytes": w64.num_buckets * 64, "glines_per_s": round(lr64 / 1e9, 2),
                                       "probe": cfg64, "gcas_per_s": round(cr64 / 1e9, 2)}
    s64["frac_line_cas"] = line_cas_fracs(s64["per_op_mops"], lpo64, cas64, lr64, cr64)
    out["slab64_step"] = s64
    out["seconds"] = round(time.perf_counter() - t0, 1)
    ex.shutdown()
    return out


def reference_arm(args, rank, world):
    """The oracle as it stands on the host cores, whole steps of the same workload."""
    if rank != 0:
        return
    w, mb = make_step_inputs(args.seed)
    for _ in range(args.warmup):
        run_oracle_step(w, mb)
    times = []
    for _ in range(args.steps):
        dt, _, _ = run_oracle_step(w, mb)
        times.append(dt)
    total = sum(times)
    value = OPS_PER_STEP * args.steps / total / 1e6
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "Mops/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total / args.steps * 1e3, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
           "config": config_dict(),
           "cpu_baseline": {"kind": "oracle", "cores": 1, "host": host_cpu(), "value": round(value, 3), "unit": "Mops/s",
                            "sample": f"whole steps ({OPS_PER_STEP} ops each), plain C oracle, one thread"},
           "e2e": {"value": round(value, 3), "unit": "Mops/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
