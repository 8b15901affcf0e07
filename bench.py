#!/usr/bin/env python
"""Benchmark: OTLM problems solved per second to a 1e-5 marginal tolerance at n = 4096 on GB300.

One step = one solve of a whole batch (every problem run from the cold start until its
source-marginal violation e <= tol, Algorithm 1 with one MM step per iteration) through the C ABI.

  python bench.py [--gpus N --steps K --warmup W] [--impl ours|reference] [--workload NAME]

Prints one JSON line (rank 0).  `value` = problems solved per second over all ranks (replicas:
every rank solves its own batch, no collective on the data path).  `e2e` = the same metric through
otlm_solve_host with pinned host buffers (host<->device copies inside the timed region).
`roofline` = the dominant kernel (the kernel apply) against the exponent-unit peak; its launch
durations are measured live with CUDA events on the solver's stream.  `cpu_baseline` = the FP64
oracle (numpy, one thread) on a bounded sample of the same workload.
`--impl reference` times that oracle alone (the CPU reference arm).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import spectra  # noqa: E402

METRIC = "OTLM problems solved/s to 1e-5 marginal tol (n=4096) vs plain FP32 on 1 GB300; % roofline"
# the metric of each secondary workload, by name prefix (the same for the GPU arm and the reference arm)
WORKLOAD_METRICS = {
    "batch1024_n1024": "OTLM problems solved/s to 1e-5 marginal tol (n=1024 batch) vs plain FP32 on 1 GB300",
    "ragged": "OTLM problems solved/s to 1e-5 marginal tol, uneven batch (n ~ U{256..4096}) in one persistent launch",
    "warmstart": "OTLM problems solved/s to 1e-5 marginal tol, learned warm start vs cold start (n=2048)",
    "single": "OTLM single-target FP64 solve time (n=m=200, k=10, 500 iterations)",
    "hbm": "single-target OTLM solves/s to 1e-5 marginal tol at n=16384 (stored kernel streamed from HBM)",
    "banded": "OTLM problems/s to 1e-5 marginal tol, banded cost + sparse dictionary at n=100000 "
              "(the paper's scalability test)",
}


def workload_metric(workload: str) -> str:
    for prefix, metric in WORKLOAD_METRICS.items():
        if workload.startswith(prefix):
            return metric
    return METRIC
SMS = 152
MAX_SM_MHZ = 2070.0
# exponent-unit (MUFU.EX2) results per SM per clock on GB300; a throughput probe measured 30.3
EX2_PER_SM_CLK = 32


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ------------------------------------------------------------------------------------------------
# replicas: each rank solves its own shard of the workload's problem stream; the only cross-rank
# steps are the timing barrier and the max of the timings (no collective on the data path)
# ------------------------------------------------------------------------------------------------

def shard_first(rank: int, per_rank: int) -> int:
    """Index of rank `rank`'s first problem: ranks solve disjoint, consecutive shards."""
    return rank * per_rank


def max_over_ranks(values, world: int, device="cpu"):
    """Element-wise max of per-rank timings (the slowest rank sets the whole-job time)."""
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def whole_job_rate(per_rank: int, world: int, steps: int, seconds: float) -> float:
    """Problems per second of the whole job: every rank's problems over the slowest rank's time."""
    return per_rank * world * steps / seconds


# ------------------------------------------------------------------------------------------------
# CPU legs: the FP64 oracle in a pool of single-threaded worker processes (started with spawn, so
# they never inherit the CUDA context), and the parallel generation of large input sets into shared
# memory.  The workers regenerate every problem from its seed (spectra), so nothing large is pickled.
# ------------------------------------------------------------------------------------------------

_THREAD_ENV = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def _noop(_):
    return 0


class CpuPool:
    """`procs` spawned worker processes, each limited to one BLAS thread; started (imports done)
    before any timing."""

    def __init__(self, procs: int):
        import multiprocessing as mp
        saved = {k: os.environ.get(k) for k in _THREAD_ENV}
        for k in _THREAD_ENV:
            os.environ[k] = "1"
        try:
            self.pool = mp.get_context("spawn").Pool(procs)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        self.procs = procs
        self.pool.map(_noop, range(procs), chunksize=1)

    def map(self, fn, jobs):
        return self.pool.map(fn, jobs, chunksize=1)

    def close(self):
        self.pool.close()
        self.pool.join()


def _problem(workload: str, p: int):
    """Problem p of a workload as the GPU gets it (FP32-rounded inputs), as float64 arrays."""
    c = spectra.WORKLOADS[workload]
    if workload.startswith("ragged"):
        q = spectra.ragged(c["id"], 1, first=p)[0]
        x, D, y, eps = q["x"], q["D"], q["y"], q["eps"]
    else:
        d = spectra.batch(c["id"], 1, c["n"], c["k"], c["nnz"], dtype=c.get("dtype", np.float32), first=p)
        x, D, y, eps = d["x"], d["D"], d["y"][0], c["eps"]
    return np.asarray(x, np.float64), np.asarray(D, np.float64), np.asarray(y, np.float64), eps


def _oracle_job(job):
    """One FP64 oracle solve in a worker: job = (workload, problem, iterations, g0, w0, keep_state
    [, tol]); returns (solve seconds, iterations, (w, t) or None).  Exactly `iterations` iterations
    (the GPU's count for trajectory parity, or a bounded sample of a solve), or up to them until the
    violation is <= tol when tol is given."""
    import oracle
    wl, p, n_iter, g0, w0, keep = job[:6]
    tol = job[6] if len(job) > 6 else 0.0
    c = spectra.WORKLOADS[wl]
    x, D, y, eps = _problem(wl, p)
    C = spectra.squared_cost(x)
    if w0 is None:
        w0 = spectra.initial_weights(y, D)
    t0 = time.perf_counter()
    r = oracle.solve_log(C, D, y, eps, c["lam"], c["alpha"], c["datafit"], c["penalty"], w0, n_iter, g0=g0, tol=tol)
    secs = time.perf_counter() - t0
    return secs, int(r["iters"]), ((r["w"], r["t"]) if keep else None)


def _oracle_banded_job(job):
    """The oracle's banded solve (scalability test form) of target p for `iterations` iterations."""
    import oracle
    from scipy.sparse import csc_matrix
    wl, p, n_iter = job
    c = spectra.WORKLOADS[wl]
    d = spectra.scaling_batch(c["id"], 1, c["n"], first=p)
    X = csc_matrix((d["val"].astype(np.float64), d["row_idx"], d["col_ptr"]), shape=(d["n"], d["k"]))
    y = d["y"][0].astype(np.float64)
    w0 = y.sum() / (d["k"] * d["x_col"])
    t0 = time.perf_counter()
    r = oracle.solve_log_banded(d["Cd"].astype(np.float64), d["h"], X, y, c["eps"], c["lam"], c["alpha"],
                                c["datafit"], c["penalty"], w0, n_iter)
    return time.perf_counter() - t0, int(r["iters"]), None


def cpu_baseline(workload: str, problems, sample_iters: int, gpu_iters, banded=False, pool=None, one_core=None,
                 all_cores=True):
    """The FP64 oracle on `problems` of the workload, each run `sample_iters` iterations, timed on
    every core of this host (os.cpu_count()) and, on the first `one_core` of them (all by default),
    on one core; each problem's time is scaled to its whole solve, (2 T + 1) / (2 S + 1) kernel
    applies for T = its GPU iteration count (gpu_iters, per problem or one number) and
    S = sample_iters.  Returns the cpu_baseline object (problems/s on all cores, with the one-core
    figure beside it)."""
    problems = list(problems)
    cores = os.cpu_count() or 1
    T = np.broadcast_to(np.asarray(gpu_iters, np.float64), (len(problems),))
    factor = (2 * T + 1) / (2 * sample_iters + 1)
    jobs = [(workload, int(p), sample_iters) if banded else (workload, int(p), sample_iters, None, None, False)
            for p in problems]
    fn = _oracle_banded_job if banded else _oracle_job
    m1 = len(jobs) if one_core is None else min(one_core, len(jobs))
    one = CpuPool(1)
    r1 = one.map(fn, jobs[:m1])
    one.close()
    solve_1 = float(np.sum([r[0] * f for r, f in zip(r1, factor[:m1])]))  # one core: whole solves, back to back
    if not all_cores:
        return {"value": m1 / solve_1, "unit": "problems/s", "cores": 1, "kind": "oracle",
                "sample": f"FP64 numpy oracle on {m1} problem(s) of {workload}, {sample_iters} iteration(s) each "
                          f"({2 * sample_iters + 1} kernel applies), scaled to its GPU iteration count "
                          f"({T.mean():.1f}); one core ({sum(r[0] for r in r1):.1f} s of solves)"}
    own = pool is None
    pool = pool or CpuPool(cores)
    t0 = time.perf_counter()
    rN = pool.map(fn, jobs)
    wall = time.perf_counter() - t0
    if own:
        pool.close()
    busy_N = float(np.sum([r[0] for r in rN]))
    scaled_N = float(np.sum([r[0] * f for r, f in zip(rN, factor)]))
    wall_full = wall * scaled_N / max(busy_N, 1e-30)  # the pool's wall time, scaled the same way
    n = len(problems)
    return {"value": n / wall_full, "unit": "problems/s", "cores": cores, "kind": "oracle",
            "single_core": {"value": m1 / solve_1, "unit": "problems/s", "cores": 1, "problems": m1},
            "sample": f"FP64 numpy oracle on {n} problems of {workload} ({m1} of them also on one core), "
                      f"{sample_iters} iteration(s) each ({2 * sample_iters + 1} kernel applies), each scaled "
                      f"to its GPU iteration count (mean {T.mean():.1f}); one core: "
                      f"{sum(r[0] for r in r1):.1f} s of solves; {cores} cores: {wall:.1f} s wall"}


def oracle_errors(pool, workload: str, problems, iters, w_gpu, t_gpu, g0=None, w0=None):
    """Per-problem relative L1 error of the GPU's w and t against the FP64 oracle run from the same
    start for the GPU's own iteration count (trajectory parity), computed on the CPU pool."""
    jobs = [(workload, int(p), int(iters[i]), None if g0 is None else np.asarray(g0[i], np.float64),
             None if w0 is None else np.asarray(w0[i], np.float64), True) for i, p in enumerate(problems)]
    res = pool.map(_oracle_job, jobs)
    ew, et = [], []
    for i, (_, _, (wo, to)) in enumerate(res):
        ew.append(float(np.abs(np.asarray(w_gpu[i], np.float64) - wo).sum() / np.abs(wo).sum()))
        et.append(float(np.abs(np.asarray(t_gpu[i], np.float64) - to).sum() / np.abs(to).sum()))
    return {"n": len(problems), "w_rel_l1": {"max": max(ew), "median": float(np.median(ew))},
            "t_rel_l1": {"max": max(et), "median": float(np.median(et))},
            "problems": [int(p) for p in problems], "w_per_problem": ew, "t_per_problem": et,
            "method": "FP64 oracle from the same start for each problem's GPU iteration count"}


def _gen_targets_job(job):
    """Fill rows [a, b) of a shared float32 [B][n] array with targets first + a .. first + b - 1."""
    from multiprocessing import shared_memory
    name, B, n, k, nnz, wid, first, a, b = job
    shm = shared_memory.SharedMemory(name=name)
    Y = np.ndarray((B, n), np.float32, buffer=shm.buf)
    Y[a:b] = spectra.batch(wid, b - a, n, k, nnz, first=first + a)["y"]
    del Y
    shm.close()
    return b - a


def gen_targets(pool, wid: int, B: int, n: int, k: int, nnz: int, first: int, device):
    """spectra.batch(wid, B, n, k, nnz, first) generated by the pool's workers straight into shared
    memory, returned as (x, D, y) device tensors (the same values as the serial generator)."""
    import torch
    from multiprocessing import shared_memory
    shm = shared_memory.SharedMemory(create=True, size=4 * B * n)
    try:
        step = max(1, -(-B // (4 * pool.procs)))
        pool.map(_gen_targets_job, [(shm.name, B, n, k, nnz, wid, first, a, min(B, a + step))
                                    for a in range(0, B, step)])
        Y = np.ndarray((B, n), np.float32, buffer=shm.buf)
        y = torch.from_numpy(Y).to(device, copy=True)  # the shared memory is released below
        del Y
    finally:
        shm.close()
        shm.unlink()
    d = spectra.batch(wid, 1, n, k, nnz, first=first)
    return torch.tensor(d["x"], device=device), torch.tensor(d["D"], device=device), y


def _gen_ragged_job(job):
    """Problems first + a .. first + b - 1 of an uneven batch into shared x / D / y arrays at their
    packed offsets."""
    from multiprocessing import shared_memory
    names, tot, wid, first, a, b, off_n, off_D, off_k = job
    bufs = [shared_memory.SharedMemory(name=nm) for nm in names]
    x = np.ndarray((tot[0],), np.float32, buffer=bufs[0].buf)
    D = np.ndarray((tot[1],), np.float32, buffer=bufs[1].buf)
    y = np.ndarray((tot[0],), np.float32, buffer=bufs[2].buf)
    w0 = np.ndarray((tot[2],), np.float32, buffer=bufs[3].buf)
    for i, q in enumerate(spectra.ragged(wid, b - a, first=first + a)):
        on, oD, ok = off_n[i], off_D[i], off_k[i]
        x[on:on + q["n"]] = q["x"]
        D[oD:oD + q["n"] * q["k"]] = q["D"].ravel()
        y[on:on + q["n"]] = q["y"]
        w0[ok:ok + q["k"]] = spectra.initial_weights(q["y"], q["D"])
    del x, D, y, w0
    for bf in bufs:
        bf.close()
    return b - a


def gen_ragged(pool, wid: int, count: int, first: int, device):
    """spectra.ragged(wid, count, first) packed as otlm.RaggedBatch device tensors, generated by
    the pool's workers into shared memory (the same values as the serial generator), with the
    cold-start weights w0 [sum k] (spectra.initial_weights per problem) and the sizes n, k."""
    import torch
    from multiprocessing import shared_memory

    from paper_2504_04609_gb300 import otlm as api
    n, k, eps = spectra.ragged_sizes(wid, count, first=first)
    off_n = np.concatenate([[0], np.cumsum(n)[:-1]]).astype(np.int64)
    off_D = np.concatenate([[0], np.cumsum(n * k)[:-1]]).astype(np.int64)
    off_k = np.concatenate([[0], np.cumsum(k)[:-1]]).astype(np.int64)
    tot = (int(n.sum()), int((n * k).sum()), int(k.sum()))
    sizes = (tot[0], tot[1], tot[0], tot[2])
    shms = [shared_memory.SharedMemory(create=True, size=4 * sz) for sz in sizes]
    try:
        step = max(1, -(-count // (4 * pool.procs)))
        pool.map(_gen_ragged_job, [([m.name for m in shms], tot, wid, first, a, min(count, a + step),
                                    off_n[a:a + step], off_D[a:a + step], off_k[a:a + step])
                                   for a in range(0, count, step)])
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device, copy=True)  # noqa: E731
        arrs = [np.ndarray((sz,), np.float32, buffer=m.buf) for sz, m in zip(sizes, shms)]
        rb = api.RaggedBatch(count, t(n.astype(np.int32)), t(k.astype(np.int32)), t(eps.astype(np.float32)),
                             t(off_n), t(off_D), t(off_k), *(t(a) for a in arrs[:3]))
        w0 = t(arrs[3])
        del arrs
    finally:
        for m in shms:
            m.close()
            m.unlink()
    return rb, w0, n, k


# ------------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.gpu = gpu_index

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------------

# DRAM bytes per launch of the tensor-core apply (gemm3_pair_kernel<KIND_BF16>) at n = 4096, 4096
# problems, averaged over the applies of one solve under the precision schedule, from a one-pass
# ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of the kernel as it stands.
TC_APPLY_TRAFFIC_WORKLOAD = "batch4096_n4096_l2_l2sq"
TC_APPLY_TRAFFIC = 189.7e6
TC_APPLY_TRAFFIC_NOTE = ("mean DRAM bytes per apply over the 40 applies of one solve under the schedule at 3e-5 "
                         "(25 single-product on 256 x 256 pair tiles: 119 MB, 14 hi/lo: 329 MB, against 134 / 201 MB "
                         "algorithmic), one-pass ncu capture: profiles/gemm3_pair_apply_n4096_b4096.md")

# Precision schedule of the tensor-core applies (otlm_config.bf16_single_until) by workload: used
# where the tests show the 1e-5 bar holds with it (the squared-error datafit, up to three times the
# tolerance); 0 = hi/lo throughout.
SINGLE_UNTIL = {"batch4096_n4096_l2_l2sq": 3e-5}


def tc_apply_roofline(workload, n, iters, apply_timing, peaks, iters_hilo=None, apply_timing_hilo=None):
    """Roofline of the tensor-core apply (gemm3_pair_kernel<KIND_BF16>) from one timed solve.

    Algorithmic work is 2 n^2 flops per problem per apply (one multiply-add per kernel entry); a
    problem stopping after T iterations sees T + 1 source and T target applies.  apply_timing =
    (ms, launches) of the solve's applies (CUDA events).  Under the precision schedule the first
    applies issue one tensor product per algorithmic one and the rest three (the hi/lo split); the
    solve with the split throughout (iters_hilo, apply_timing_hilo) gives the issued rate of the
    three-product launches.  DRAM traffic is reported for the workload it was captured on only."""
    it = np.asarray(iters, dtype=np.float64)
    flops = 2.0 * n * n * float(np.sum(2 * it + 1))
    g_ms, g_cnt = apply_timing
    achieved = flops / (g_ms / 1e3) / 1e12
    peak = float(peaks.get("bf16_tflops_sustained", 1700.0))
    captured = workload == TC_APPLY_TRAFFIC_WORKLOAD
    r = {"bound": "tensor",
         "kernel": "gemm3_pair_kernel<KIND_BF16> (two-SM tcgen05 K V^T, BF16 hi/lo, FP32 accumulate)",
         "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
         "traffic": TC_APPLY_TRAFFIC if captured else None, "launch_ms_avg": g_ms / max(g_cnt, 1),
         "peak_basis": "MEASURED_PEAKS.json bf16_tflops_sustained (kernel timed inside a long step)"
         if "bf16_tflops_sustained" in peaks else "fallback 1.7 PFLOP/s sustained",
         "traffic_note": TC_APPLY_TRAFFIC_NOTE if captured else "no DRAM capture of this workload"}
    if iters_hilo is not None:
        it3 = np.asarray(iters_hilo, dtype=np.float64)
        issued = 3 * 2.0 * n * n * float(np.sum(2 * it3 + 1)) / (apply_timing_hilo[0] / 1e3) / 1e12
    else:
        issued = 3 * achieved
    r["issued_tensor_tflops_hilo"] = issued
    r["issued_frac_hilo"] = issued / peak
    return r


def run_ours(args, rank, world, local_rank, pool=None):
    import torch
    import torch.distributed as dist

    from paper_2504_04609_gb300 import otlm as api

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    c = spectra.WORKLOADS[args.workload]
    B, n, k = c["B"], c["n"], c["k"]
    d = spectra.batch(c["id"], B, n, k, c["nnz"], first=shard_first(rank, B))
    x = torch.tensor(d["x"], device=dev)
    D = torch.tensor(d["D"], device=dev)
    y = torch.tensor(d["y"], device=dev)
    w0_np = spectra.initial_weights(d["y"], d["D"]).astype(np.float32)
    w0 = torch.tensor(w0_np, device=dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            dist.barrier()

    def measure(precision, steps, warmup, single_until=0.0):
        """Device-resident inputs; returns timing of `steps` whole-batch solves."""
        w = torch.empty_like(w0)
        t = torch.empty_like(y)
        iters = torch.empty(B, dtype=torch.int32, device=dev)
        err = torch.empty(B, dtype=torch.float32, device=dev)
        status = torch.empty(B, dtype=torch.int32, device=dev)
        h = api.Handle(n, k, B, precision, c["datafit"], c["penalty"], c["iters"], c["tol"], poll_every=4,
                       stream=stream.cuda_stream, bf16_single_until=single_until)

        def step():
            w.copy_(w0)
            h.solve(x, D, y, c["eps"], c["lam"], c["alpha"], w, None, t, iters, err, status)

        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        l0 = h.launches
        with ClockSampler(local_rank) as clk:
            barrier()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                step()
            e1.record(stream)
            torch.cuda.synchronize()
            barrier()
        launches = h.launches - l0
        # per-kernel times from one more solve with a CUDA-event pair around every launch (kept out
        # of the timed steps: recording the events costs host time per launch)
        h.set_timing(True)
        h.get_timing()
        step()
        torch.cuda.synchronize()
        timing = h.get_timing()
        h.set_timing(False)
        return dict(ms=e0.elapsed_time(e1), launches=launches, timing=timing, iters=iters.cpu().numpy(),
                    status=status.cpu().numpy(), clocks=clk.summary(), handle=h, w=w, t=t)

    sched = SINGLE_UNTIL.get(args.workload, 0.0)
    tc = measure("bf16tc", args.steps, args.warmup, sched)
    tc3 = measure("bf16tc", max(1, min(args.steps, 3)), max(3, min(args.warmup, 3))) if sched > 0 else None
    if tc3 is not None:
        tc3["handle"].close()
    fp = measure("fp32", max(1, min(args.steps, 3)), max(1, min(args.warmup, 3)))
    fp["handle"].close()

    # end to end through the host-buffer entry point (pinned host memory), tensor-core path
    h = tc["handle"]
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
    hx, hD, hy, hw0 = pin(d["x"]), pin(d["D"]), pin(d["y"]), pin(w0_np)
    hw = torch.empty_like(hw0).pin_memory()
    ht = torch.empty_like(hy).pin_memory()
    hit = torch.empty(B, dtype=torch.int32).pin_memory()
    herr = torch.empty(B, dtype=torch.float32).pin_memory()
    hst = torch.empty(B, dtype=torch.int32).pin_memory()

    def step_host():
        hw.copy_(hw0)
        h.solve_host(hx, hD, hy, c["eps"], c["lam"], c["alpha"], hw, None, ht, hit, herr, hst)

    step_host()
    e2e_steps = max(1, args.steps)
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        step_host()
    barrier()
    e2e_s = time.perf_counter() - t0
    h.close()
    h2d = hx.numel() * 4 + hD.numel() * 4 + hy.numel() * 4 + hw.numel() * 4
    d2h = hw.numel() * 4 + ht.numel() * 4 + B * 4 * 3

    tc_ms, fp_ms, e2e_s, tc3_ms = max_over_ranks([tc["ms"], fp["ms"], e2e_s, tc3["ms"] if tc3 else 0.0], world, dev)
    if rank != 0:
        return None

    fp_steps = max(1, min(args.steps, 3))
    value = whole_job_rate(B, world, args.steps, tc_ms / 1e3)
    fp_value = whole_job_rate(B, world, fp_steps, fp_ms / 1e3)
    peaks = _peaks()

    it_tc = tc["iters"].astype(np.float64)
    roofline = tc_apply_roofline(args.workload, n, tc["iters"], tc["timing"]["apply"], peaks,
                                 tc3["iters"] if tc3 is not None else None,
                                 tc3["timing"]["apply"] if tc3 is not None else None)

    # plain FP32 path: the log-sum-exp apply against the exponent unit
    it_fp = fp["iters"].astype(np.float64)
    exps_step = float(n) * n * float(np.sum(2 * it_fp + 1))
    a_ms, a_cnt = fp["timing"]["apply"]
    ach = exps_step / (a_ms / 1e3) / 1e9
    peak_ex = SMS * EX2_PER_SM_CLK * MAX_SM_MHZ * 1e6 / 1e9
    plain = {"value": fp_value, "unit": "problems/s", "ms_per_step": fp_ms / fp_steps, "steps": fp_steps,
             "mean_iters": float(it_fp.mean()), "converged": int(np.sum(fp["status"] == 0)),
             "kernel_ms_per_step": {kk: v[0] for kk, v in fp["timing"].items()},
             "roofline": {"bound": "alu", "kernel": "apply_kernel (FP32 log-sum-exp)", "achieved": ach,
                          "peak": peak_ex, "unit": "Gexp2/s", "frac": ach / peak_ex, "traffic": None,
                          "launch_ms_avg": a_ms / max(a_cnt, 1),
                          "peak_basis": f"{SMS} SMs x {EX2_PER_SM_CLK} ex2/clk x {MAX_SM_MHZ:.0f} MHz (derived; "
                                        "probe measured 30.3 ex2/clk/SM)"},
             "clocks": fp["clocks"]}
    out = {
        "metric": workload_metric(args.workload),
        "value": value,
        "unit": "problems/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": tc_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "bf16x3 tensor (hi/lo split) + f32" + (", bf16x1 until a violation <= %g" % sched if sched else ""),
        "data": "synthetic (seeded Gaussian-peak spectra, no dataset)",
        "config": {"workload": args.workload, "B_per_gpu": B, "n": n, "k": k, "eps": c["eps"],
                   "datafit": c["datafit"], "lam": c["lam"], "penalty": c["penalty"], "alpha": c["alpha"],
                   "tol": c["tol"], "path": "tensor-core applies (tcgen05, BF16 hi/lo, FP32 accumulate)",
                   "bf16_single_until": sched,
                   "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (4096 x 4096 FP32 state arrays, 64 MiB each, several per step)",
                   "mean_iters": float(it_tc.mean()), "max_iters": int(it_tc.max()),
                   "converged": int(np.sum(tc["status"] == 0))},
        "iters_per_s": float(it_tc.sum()) * world * args.steps / (tc_ms / 1e3),
        "speedup_vs_plain_fp32": value / fp_value,
        "plain_fp32": plain,
        "tensor_hilo_throughout": ({"value": whole_job_rate(B, world, max(1, min(args.steps, 3)), tc3_ms / 1e3),
                                    "unit": "problems/s", "kernel_ms_per_step": {kk: v[0] for kk, v in
                                                                                 tc3["timing"].items()},
                                    "mean_iters": float(tc3["iters"].mean())} if tc3 else None),
        "roofline": roofline,
        "kernel_ms_per_step": {kk: v[0] for kk, v in tc["timing"].items()},
        "e2e": {"value": whole_job_rate(B, world, e2e_steps, e2e_s), "unit": "problems/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": tc["launches"],
        "clocks": tc["clocks"],
    }
    # the FP64 duality gap of every returned state, computed on the GPU (check_every = 10): its cost
    # beside the plain solve, and the gaps it reports
    gh = api.Handle(n, k, B, "bf16tc", c["datafit"], c["penalty"], c["iters"], c["tol"], poll_every=4,
                    stream=stream.cuda_stream, check_every=10)
    wg = w0.clone()
    P = torch.empty(B, dtype=torch.float64, device=dev)
    Dv = torch.empty(B, dtype=torch.float64, device=dev)
    gh.solve(x, D, y, c["eps"], c["lam"], c["alpha"], wg)  # warm-up
    torch.cuda.synchronize()
    wg.copy_(w0)
    g0_ = torch.cuda.Event(enable_timing=True)
    g1_ = torch.cuda.Event(enable_timing=True)
    g0_.record(stream)
    gh.solve(x, D, y, c["eps"], c["lam"], c["alpha"], wg)
    g1_.record(stream)
    gh.solve_stats(B, None, P, Dv)
    torch.cuda.synchronize()
    gh.close()
    rel_gap = ((P - Dv) / P.abs()).cpu().numpy()
    out["fp64_gap"] = {"check_every": 10, "ms_per_step": g0_.elapsed_time(g1_),
                       "overhead_vs_plain": g0_.elapsed_time(g1_) / (tc_ms / args.steps) - 1.0,
                       "rel_gap_of_returned_states": {"median": float(np.median(rel_gap)), "max": float(rel_gap.max()),
                                                      "min": float(rel_gap.min())},
                       "note": "primal and Fenchel dual of each returned state reduced in FP64 on the GPU (one "
                               "extra tensor-core apply per check); the stop here is the 1e-5 violation alone"}
    if world == 1 and not args.no_cpu_baseline:
        own_pool = pool is None
        pool = pool or CpuPool(os.cpu_count() or 1)
        pick = np.unique(np.linspace(0, B - 1, 16).astype(np.int64))
        out["err_vs_fp64"] = oracle_errors(pool, args.workload, pick, it_tc[pick], tc["w"][pick].cpu().numpy(),
                                           tc["t"][pick].cpu().numpy())
        out["err_vs_fp64"]["path"] = "tensor-core (BF16 hi/lo applies, TF32 hi/lo contractions)"
        nb = min(B, 64)
        out["cpu_baseline"] = cpu_baseline(args.workload, range(nb), 1, it_tc[:nb], pool=pool,
                                           one_core=16 if n >= 4096 else nb)
        if own_pool:
            pool.close()
    return out


def run_ragged(args, rank, world, local_rank, pool=None):
    """Uneven batch: 10,000 problems with their own n, k, eps, grid and dictionary, solved to tol
    in one persistent, graph-captured launch (CTA size from the library's tuner)."""
    import torch
    import torch.distributed as dist

    from paper_2504_04609_gb300 import otlm as api

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    c = spectra.WORKLOADS[args.workload]
    B = c["count"]
    own_pool = pool is None
    pool = pool or CpuPool(os.cpu_count() or 1)
    rb, w0, n_np, _ = gen_ragged(pool, c["id"], B, shard_first(rank, B), dev)
    stream = torch.cuda.current_stream(dev)
    h = api.Handle(4096, 128, B, "fp32", c["datafit"], c["penalty"], c["iters"], c["tol"],
                   stream=stream.cuda_stream)
    cta, rows_tab = h.tune_ragged(rb, c["lam"], c["alpha"], w0, sample_every=40, iters=6, with_rows=True)
    w = torch.empty_like(w0)
    t = torch.empty_like(rb.y)
    iters = torch.empty(B, dtype=torch.int32, device=dev)
    err = torch.empty(B, device=dev)
    status = torch.empty(B, dtype=torch.int32, device=dev)

    def step():
        w.copy_(w0)
        h.solve_ragged(rb, c["lam"], c["alpha"], w, None, t, iters, err, status)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    l0 = h.launches
    with ClockSampler(local_rank) as clk:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    ms = e0.elapsed_time(e1)
    launches = h.launches - l0
    # the persistent launch's device time from one more solve with a CUDA-event pair around it
    h.set_timing(True)
    h.get_timing()
    step()
    torch.cuda.synchronize()
    timing = h.get_timing()
    h.set_timing(False)
    it_np = iters.cpu().numpy().astype(np.float64)
    st_np = status.cpu().numpy()

    # end to end: pinned host inputs copied in and results copied out inside the timed region
    pin = lambda a: a.cpu().pin_memory()  # noqa: E731
    hx, hD, hy, hw0 = pin(rb.x), pin(rb.D), pin(rb.y), pin(w0)
    hw = torch.empty_like(hw0).pin_memory()
    ht = torch.empty_like(hy).pin_memory()
    hit = torch.empty(B, dtype=torch.int32).pin_memory()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(max(1, args.steps)):
        rb.x.copy_(hx, non_blocking=True)
        rb.D.copy_(hD, non_blocking=True)
        rb.y.copy_(hy, non_blocking=True)
        w.copy_(hw0, non_blocking=True)
        h.solve_ragged(rb, c["lam"], c["alpha"], w, None, t, iters, err, status)
        hw.copy_(w, non_blocking=True)
        ht.copy_(t, non_blocking=True)
        hit.copy_(iters, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    h.close()
    ms, e2e_s = max_over_ranks([ms, e2e_s], world, dev)
    if rank != 0:
        if own_pool:
            pool.close()
        return None
    exps_step = float(np.sum(n_np.astype(np.float64) ** 2 * (2 * it_np + 1)))
    k_ms = timing["apply"][0]  # one step
    ach = exps_step / (k_ms / 1e3) / 1e9
    peak_ex = SMS * EX2_PER_SM_CLK * MAX_SM_MHZ * 1e6 / 1e9
    h2d = (hx.numel() + hD.numel() + hy.numel() + hw0.numel()) * 4
    d2h = (hw.numel() + ht.numel() + hit.numel()) * 4
    out = {
        "metric": workload_metric(args.workload),
        "value": whole_job_rate(B, world, args.steps, ms / 1e3), "unit": "problems/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded Gaussian-peak spectra, no dataset)",
        "config": {"workload": args.workload, "problems_per_gpu": B, "n": "U{256..4096}", "k": "U{8..128}",
                   "eps": "logU[2e-3, 5e-2]", "datafit": c["datafit"], "penalty": c["penalty"], "lam": c["lam"],
                   "alpha": c["alpha"], "tol": c["tol"], "cta_threads_tuned": cta,
                   "rows_per_thread_log2_by_bucket": rows_tab,
                   "l2": "inputs larger than L2 (dictionaries 6 GB)",
                   "converged": int(np.sum(st_np == 0)), "iters_p50": float(np.percentile(it_np, 50)),
                   "iters_p99": float(np.percentile(it_np, 99)), "iters_mean": float(it_np.mean())},
        "iters_per_s": float(it_np.sum()) * world * args.steps / (ms / 1e3),
        "roofline": {"bound": "alu", "kernel": "ragged_kernel (persistent, whole solve)", "achieved": ach,
                     "peak": peak_ex, "unit": "Gexp2/s", "frac": ach / peak_ex, "traffic": None,
                     "launch_ms_avg": timing["apply"][0] / max(timing["apply"][1], 1),
                     "note": "algorithmic exp2 = sum_p n_p^2 (2 iters_p + 1); the kernel also runs the MM and "
                             "source steps, so the fraction is a lower bound for the apply itself"},
        "e2e": {"value": whole_job_rate(B, world, max(1, args.steps), e2e_s), "unit": "problems/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.workload, range(64), 1, it_np[:64], pool=pool)
    if own_pool:
        pool.close()
    return out


def run_single_fp64(args, rank, local_rank):
    """Single target, FP64 throughout (n = m = 200, k = 10, 500 iterations): time only."""
    import torch

    from paper_2504_04609_gb300 import otlm as api
    if rank != 0:
        return None
    torch.cuda.set_device(local_rank)
    c = spectra.WORKLOADS[args.workload]
    d = spectra.batch(c["id"], 1, c["n"], c["k"], c["nnz"], dtype=np.float64)
    dev = torch.device("cuda", local_rank)
    x, D, y = (torch.tensor(d[q], device=dev) for q in ("x", "D", "y"))
    w0 = torch.tensor(spectra.initial_weights(d["y"], d["D"]), device=dev)
    w = torch.empty_like(w0)
    stream = torch.cuda.current_stream(dev)
    h = api.Handle(c["n"], c["k"], 1, "fp64", c["datafit"], c["penalty"], c["iters"], 0.0, poll_every=64,
                   stream=stream.cuda_stream)
    for _ in range(args.warmup):
        w.copy_(w0)
        h.solve(x, D, y, c["eps"], c["lam"], c["alpha"], w)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        w.copy_(w0)
        h.solve(x, D, y, c["eps"], c["lam"], c["alpha"], w)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    h.close()
    return {"metric": workload_metric(args.workload), "value": ms,
            "unit": "ms", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded Gaussian-peak spectra, no dataset)",
            "config": {"workload": args.workload, "n": c["n"], "k": c["k"], "eps": c["eps"], "iters": c["iters"]}}


WS_TEST_FIRST = 10_000_000  # held-out problems of the warm-start workload start at this index


def run_warmstart(args, rank, local_rank, pool=None):
    """Learned warm start at n = 2048, k = 64 (KL datafit, squared-l2 penalty, eps = 5e-3): train on
    problems labelled by the solver, then solve held-out problems cold and warm, FP32 and tensor-core
    paths, to the same 1e-5 tolerance.  Sizes: --ws-train (default 200,000), --ws-test (20,000)."""
    import torch

    from paper_2504_04609_gb300 import otlm as api
    from paper_2504_04609_gb300 import warmstart as ws
    if rank != 0:
        return None
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    c = dict(spectra.WORKLOADS[args.workload])
    n, k = c["n"], c["k"]
    own_pool = pool is None
    pool = pool or CpuPool(os.cpu_count() or 1)
    t0 = time.perf_counter()
    x, D, ytr = gen_targets(pool, c["id"], args.ws_train, n, k, c["nnz"], 0, dev)
    _, _, yte = gen_targets(pool, c["id"], args.ws_test, n, k, c["nnz"], WS_TEST_FIRST, dev)
    gen_s = time.perf_counter() - t0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    net = api.WarmStart(n, k, 512, 512, seed=2504_04609)
    targets = ws.make_labels(net, x, D, ytr, c)
    torch.cuda.synchronize()
    label_s = time.perf_counter() - t0
    ws.normalization(net, targets)
    t0 = time.perf_counter()
    losses = ws.train(net, ytr, targets, epochs=args.ws_epochs, batch=512, lr=1e-3, weight_decay=1e-5, log_every=100)
    train_s = time.perf_counter() - t0
    out = {"metric": workload_metric(args.workload),
           "unit": "problems/s", "n_gpus": 1, "steps": 1, "warmup": 0, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32 solve, bf16-weight MLP", "data": "synthetic (seeded Gaussian-peak spectra)",
           "config": {"workload": args.workload, "n": n, "k": k, "eps": c["eps"], "datafit": c["datafit"],
                      "penalty": c["penalty"], "alpha": c["alpha"], "tol": c["tol"], "train_problems": args.ws_train,
                      "test_problems": args.ws_test, "mlp": "4 layers, width 512, GELU, BF16 weights, FP32 accumulate",
                      "epochs": args.ws_epochs, "batch": 512},
           "timings_s": {"generate_host": gen_s, "label_solves": label_s, "train": train_s},
           "train_loss_first_last": [losses[0], losses[-1]], "forms": {}}
    for prec in ("fp32", "bf16tc"):  # warm-up of both arms
        for _ in range(3):
            ws.evaluate(net, x, D, yte[:min(512, args.ws_test)], c, precision=prec)
    clk = ClockSampler(local_rank)
    clk.__enter__()
    for prec in ("fp32", "bf16tc"):
        r = ws.evaluate(net, x, D, yte, c, precision=prec)
        ok_c = r["cold_status"] == 0
        ok_w = r["warm_status"] == 0
        out["forms"][prec] = {
            "cold": {"problems_per_s": args.ws_test / r["cold_s"], "iters_mean": float(r["cold_iters"].mean()),
                     "iters_p50": float(np.percentile(r["cold_iters"], 50)),
                     "iters_p99": float(np.percentile(r["cold_iters"], 99)), "converged": int(ok_c.sum())},
            "warm": {"problems_per_s": args.ws_test / r["warm_s"], "iters_mean": float(r["warm_iters"].mean()),
                     "iters_p50": float(np.percentile(r["warm_iters"], 50)),
                     "iters_p99": float(np.percentile(r["warm_iters"], 99)), "converged": int(ok_w.sum()),
                     "predict_s": r["predict_s"]},
            "warm_vs_cold_rel_l1": {"w_median": float(np.median(r["w_rel_diff"])),
                                    "t_median": float(np.median(r["t_rel_diff"])),
                                    "t_p99": float(np.percentile(r["t_rel_diff"], 99))}}
    clk.__exit__(None, None, None)
    out["clocks"] = clk.summary()
    base = out["forms"]["fp32"]["cold"]["problems_per_s"]
    best = max(v["warm"]["problems_per_s"] for v in out["forms"].values())
    out["value"] = out["forms"]["bf16tc"]["warm"]["problems_per_s"]
    out["speedup_warm_bf16_vs_plain_fp32_cold"] = out["value"] / base
    out["target_5x_met"] = bool(out["speedup_warm_bf16_vs_plain_fp32_cold"] >= 5.0)
    out["best_form_problems_per_s"] = best

    # the warm tensor-core solve once more with per-kernel device timing: its dominant kernel, the
    # tcgen05 apply (2 n^2 FLOP per problem per apply, 2 T + 1 applies for T iterations)
    B = args.ws_test
    g0, w0 = ws.predict(net, yte, D, c["eps"])
    stream = torch.cuda.current_stream(dev)
    h = api.Handle(n, k, B, "bf16tc", c["datafit"], c["penalty"], c["iters"], c["tol"], poll_every=4,
                   stream=stream.cuda_stream)
    w, g, t = w0.clone(), g0.clone(), torch.empty_like(yte)
    it = torch.empty(B, dtype=torch.int32, device=dev)
    err = torch.empty(B, device=dev)
    st = torch.empty(B, dtype=torch.int32, device=dev)
    h.set_timing(True)
    h.get_timing()
    h.solve(x, D, yte, c["eps"], c["lam"], c["alpha"], w, g, t, it, err, st)
    torch.cuda.synchronize()
    timing = h.get_timing()
    h.close()
    it_np = it.cpu().numpy()
    flops = 2.0 * n * n * float(np.sum(2 * it_np.astype(np.float64) + 1))
    a_ms, a_cnt = timing["apply"]
    peak = float(_peaks().get("bf16_tflops_sustained", 1700.0))
    ach = flops / (a_ms / 1e3) / 1e12
    out["roofline"] = {"bound": "tensor", "kernel": "gemm3_pair_kernel<KIND_BF16> (warm tensor-core solve)",
                       "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
                       "launch_ms_avg": a_ms / max(a_cnt, 1), "kernel_ms_per_solve": {kk: v[0] for kk, v in timing.items()},
                       "peak_basis": "MEASURED_PEAKS.json bf16_tflops_sustained"}
    # error of the warm BF16 results against the FP64 oracle started from the same predicted state
    pick = np.arange(min(8, B))
    out["err_vs_fp64"] = oracle_errors(pool, args.workload, WS_TEST_FIRST + pick, it_np[pick], w[pick].cpu().numpy(),
                                       t[pick].cpu().numpy(), g0=g0[pick].cpu().numpy(), w0=w0[pick].cpu().numpy())
    out["err_vs_fp64"]["path"] = "warm start (predicted g0, w0) + tensor-core solve"
    if not args.no_cpu_baseline:
        cold_iters = out["forms"]["fp32"]["cold"]["iters_mean"]
        out["cpu_baseline"] = cpu_baseline(args.workload, WS_TEST_FIRST + np.arange(64), 1, cold_iters, pool=pool)
        out["cpu_baseline"]["sample"] += " (the oracle's cold start: the plain method)"
    if own_pool:
        pool.close()
    net.close()
    return out


# Single target at n = 16384: the FP64 oracle takes several seconds per iteration there, so its
# samples run HBM_ORACLE_ITERS iterations and are scaled to HBM_ITERS_TO_TOL, the iterations this
# problem takes to reach the 1e-5 tolerance (the tensor-core solve reports 22).
HBM_ORACLE_ITERS = 2
HBM_ITERS_TO_TOL = 22


def run_single_hbm(args, rank, world, local_rank):
    """One target at n = 16384 on the tensor-core path: the stored kernel (BF16 hi/lo, 4 n^2 bytes =
    1 GiB) is streamed from HBM by each of the two applies per iteration, so the apply is bound by
    HBM bandwidth.  Each rank solves its own target (replicas)."""
    import torch
    import torch.distributed as dist

    from paper_2504_04609_gb300 import otlm as api

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    c = spectra.WORKLOADS[args.workload]
    B, n, k = c["B"], c["n"], c["k"]
    d = spectra.batch(c["id"], B, n, k, c["nnz"], first=shard_first(rank, B))
    x, D, y = (torch.tensor(d[key], device=dev) for key in ("x", "D", "y"))
    w0_np = spectra.initial_weights(d["y"], d["D"]).astype(np.float32)
    w0 = torch.tensor(w0_np, device=dev)
    stream = torch.cuda.current_stream(dev)
    w = torch.empty_like(w0)
    t = torch.empty_like(y)
    iters = torch.empty(B, dtype=torch.int32, device=dev)
    err = torch.empty(B, dtype=torch.float32, device=dev)
    status = torch.empty(B, dtype=torch.int32, device=dev)
    h = api.Handle(n, k, B, "bf16tc", c["datafit"], c["penalty"], c["iters"], c["tol"], poll_every=8,
                   stream=stream.cuda_stream)

    def step():
        w.copy_(w0)
        h.solve(x, D, y, c["eps"], c["lam"], c["alpha"], w, None, t, iters, err, status)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    l0 = h.launches
    with ClockSampler(local_rank) as clk:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    ms = e0.elapsed_time(e1)
    launches = h.launches - l0
    # per-kernel times from one more solve with CUDA-event pairs (outside the timed steps)
    h.set_timing(True)
    h.get_timing()
    step()
    torch.cuda.synchronize()
    timing = h.get_timing()
    h.set_timing(False)
    it = int(iters.cpu().numpy()[0])
    st = int(status.cpu().numpy()[0])

    # end to end through the host-buffer entry point
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
    hx, hD, hy, hw0 = pin(d["x"]), pin(d["D"]), pin(d["y"]), pin(w0_np)
    hw, ht = torch.empty_like(hw0).pin_memory(), torch.empty_like(hy).pin_memory()
    hit, herr, hst = (torch.empty(B, dtype=dt).pin_memory() for dt in (torch.int32, torch.float32, torch.int32))

    def step_host():
        hw.copy_(hw0)
        h.solve_host(hx, hD, hy, c["eps"], c["lam"], c["alpha"], hw, None, ht, hit, herr, hst)

    step_host()
    t0 = time.perf_counter()
    for _ in range(max(1, args.steps)):
        step_host()
    e2e_s = time.perf_counter() - t0
    h.close()
    ms, e2e_s = max_over_ranks([ms, e2e_s], world, dev)
    if rank != 0:
        return None

    # the apply streams the stored kernel once: 4 n^2 bytes (BF16 hi + lo) per launch; the operand
    # (4 n bytes) and the sums (4 n bytes) are negligible beside it
    a_ms, a_cnt = timing["apply"]
    launch_ms = a_ms / max(a_cnt, 1)
    achieved = 4.0 * n * n / (launch_ms / 1e3) / 1e9
    peak = float(_peaks().get("hbm_gbs", 6800.0))
    out = {
        "metric": workload_metric(args.workload),
        "value": whole_job_rate(B, world, args.steps, ms / 1e3), "unit": "problems/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "iters_per_s": whole_job_rate(B, world, args.steps, ms / 1e3) * it,
        "vs_baseline": None, "dtype": "bf16x3 tensor (hi/lo split) + f32",
        "data": "synthetic (seeded Gaussian-peak spectra, no dataset)",
        "config": {"workload": args.workload, "B_per_gpu": B, "n": n, "k": k, "eps": c["eps"], "datafit": c["datafit"],
                   "penalty": c["penalty"], "tol": c["tol"], "iters": it, "status": st,
                   "path": "tensor-core applies with the reduction split over 16 ranges (small batch)",
                   "l2": "the stored kernel (1 GiB) is larger than L2", "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "kernel": "gemm3_kernel<KIND_BF16> + tc_split_reduce_kernel (one apply)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": 1081.2e6, "traffic_note": "GEMM 1079.4 MB read + 0.9 MB written, split reduce "
                                                          "0.9 MB read (ncu, profiles/hbm_single_n16384.md)",
                     "launch_ms_avg": launch_ms, "bytes_per_launch": 4.0 * n * n,
                     "peak_basis": "MEASURED_PEAKS.json hbm_gbs" if "hbm_gbs" in _peaks() else "fallback 6.8 TB/s"},
        "kernel_ms_per_step": {kk: v[0] for kk, v in timing.items()},
        "e2e": {"value": whole_job_rate(B, world, max(1, args.steps), e2e_s), "unit": "problems/s",
                "h2d_bytes_per_step": (hx.numel() + hD.numel() + hy.numel() + hw.numel()) * 4,
                "d2h_bytes_per_step": (hw.numel() + ht.numel() + 3 * B) * 4},
        "gpu_launches": launches, "clocks": clk.summary()}
    if world == 1 and not args.no_cpu_baseline:
        # one target: the oracle's solve of it does not spread over cores, so one core is the figure
        out["cpu_baseline"] = cpu_baseline(args.workload, [0], HBM_ORACLE_ITERS, it, all_cores=False)
    return out


BANDED_ORACLE_ITERS = 10
BANDED_ITERS_TO_TOL = 731  # the FP64 oracle's own count to 1e-5 on target 0 of the workload (131 s on one core)


def run_banded(args, rank, world, local_rank):
    """The paper's scalability test at n = 100000 (k = 10000 truncated Gaussians, cost rho |i - j|
    below 10 samples): 32 targets per GPU through otlm_solve_banded, solved to 1e-5.  Each rank
    solves its own 32 targets (replicas)."""
    import torch
    import torch.distributed as dist

    from paper_2504_04609_gb300 import otlm as api

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    c = spectra.WORKLOADS[args.workload]
    B, n = c["B"], c["n"]
    d = spectra.scaling_batch(c["id"], B, n, first=shard_first(rank, B))
    k, hw = d["k"], d["h"]
    Cd = torch.tensor(d["Cd"], device=dev)
    col_ptr = torch.tensor(d["col_ptr"], dtype=torch.int32, device=dev)
    row_idx = torch.tensor(d["row_idx"], dtype=torch.int32, device=dev)
    val = torch.tensor(d["val"], device=dev)
    y = torch.tensor(d["y"], device=dev)
    w0_np = (d["y"].astype(np.float64).sum(axis=1)[:, None] / (k * d["x_col"])[None, :]).astype(np.float32)
    w0 = torch.tensor(w0_np, device=dev)
    stream = torch.cuda.current_stream(dev)
    w = torch.empty_like(w0)
    t = torch.empty_like(y)
    iters = torch.empty(B, dtype=torch.int32, device=dev)
    err = torch.empty(B, dtype=torch.float32, device=dev)
    status = torch.empty(B, dtype=torch.int32, device=dev)
    h = api.Handle(64, 8, B, "fp32", c["datafit"], c["penalty"], c["iters"], c["tol"], poll_every=16,
                   stream=stream.cuda_stream)

    def step():
        w.copy_(w0)
        h.solve_banded(Cd, hw, col_ptr, row_idx, val, y, c["eps"], c["lam"], c["alpha"], w, None, t, iters, err,
                       status)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    l0 = h.launches
    with ClockSampler(local_rank) as clk:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    ms = e0.elapsed_time(e1)
    launches = h.launches - l0
    h.set_timing(True)
    h.get_timing()
    step()
    torch.cuda.synchronize()
    timing = h.get_timing()
    h.set_timing(False)
    its = iters.cpu().numpy()
    st = status.cpu().numpy()

    # end to end: targets and initial weights from pinned host memory, weights and marginals back
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
    hy, hw0 = pin(d["y"]), pin(w0_np)
    h_w, h_t = torch.empty_like(hw0).pin_memory(), torch.empty_like(hy).pin_memory()

    def step_host():
        y.copy_(hy, non_blocking=True)
        w.copy_(hw0, non_blocking=True)
        h.solve_banded(Cd, hw, col_ptr, row_idx, val, y, c["eps"], c["lam"], c["alpha"], w, None, t, iters, err,
                       status)
        h_w.copy_(w, non_blocking=True)
        h_t.copy_(t, non_blocking=True)
        torch.cuda.current_stream(dev).synchronize()

    step_host()
    t0 = time.perf_counter()
    for _ in range(max(1, args.steps)):
        step_host()
    e2e_s = time.perf_counter() - t0
    h.close()
    ms, e2e_s = max_over_ranks([ms, e2e_s], world, dev)
    if rank != 0:
        return None

    # both applies evaluate one exp2 per finite band entry and problem: the roofline is the exponent
    # unit (MUFU ex2), as for the FP32 log-domain apply
    Cd_np = d["Cd"].astype(np.float64)
    rows = np.arange(n)
    finite = sum(int(np.sum(np.isfinite(Cd_np[dd]) & (rows + dd - hw >= 0) & (rows + dd - hw < n)))
                 for dd in range(2 * hw + 1))
    a_ms, a_cnt = timing["apply"]
    launch_ms = a_ms / max(a_cnt, 1)
    ex2_per_launch = float(finite) * B
    achieved = ex2_per_launch / (launch_ms / 1e3) / 1e9
    peak = 152 * 32 * 2.07
    out = {
        "metric": workload_metric(args.workload),
        "value": whole_job_rate(B, world, args.steps, ms / 1e3), "unit": "problems/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "iters_per_s": float(its.sum()) * world * args.steps / (ms / 1e3),
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (log domain)",
        "data": "synthetic (the scalability appendix's recipe: skew-normal mixtures, truncated Gaussian basis)",
        "config": {"workload": args.workload, "B_per_gpu": B, "n": n, "k": k, "hw": hw, "nnz": int(d["val"].size),
                   "eps": c["eps"], "datafit": c["datafit"], "penalty": c["penalty"], "alpha": c["alpha"],
                   "tol": c["tol"], "mean_iters": float(its.mean()), "max_iters": int(its.max()),
                   "converged": int(np.sum(st == 0)), "parallelism": f"replicas x{world}",
                   "l2": "working set (about 6 arrays of 12.8 MB) stays in L2 across iterations; no flush"},
        "roofline": {"bound": "alu", "kernel": "band_source_kernel / band_target_kernel (log-sum-exp over the band)",
                     "achieved": achieved, "peak": peak, "unit": "Gexp2/s", "frac": achieved / peak,
                     "traffic": None, "launch_ms_avg": launch_ms, "ex2_per_launch": ex2_per_launch,
                     "peak_basis": "152 SMs x 32 ex2/clk x 2070 MHz (derived from unit counts and clock)"},
        "kernel_ms_per_step": {kk: v[0] for kk, v in timing.items()},
        "e2e": {"value": whole_job_rate(B, world, max(1, args.steps), e2e_s), "unit": "problems/s",
                "h2d_bytes_per_step": (hy.numel() + hw0.numel()) * 4,
                "d2h_bytes_per_step": (h_w.numel() + h_t.numel()) * 4},
        "gpu_launches": launches, "clocks": clk.summary()}
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.workload, range(B), 2, its, banded=True, one_core=8)
    return out


def run_reference(args, rank):
    """The CPU reference arm: the FP64 oracle (as it stands) on this host's cores.  Each step solves
    a bounded sample of the workload on every core at once (os.cpu_count() single-threaded worker
    processes, one problem each): to the workload's tolerance, or, where one solve takes minutes
    (n = 16384, n = 100000), a fixed number of iterations scaled to the iterations to tolerance."""
    if rank != 0:
        return None
    c = spectra.WORKLOADS[args.workload]
    cores = os.cpu_count() or 1
    pool = CpuPool(cores)
    banded = args.workload.startswith("banded")
    hbm = args.workload.startswith("hbm")
    single = args.workload.startswith("single")
    per_step = 1 if (hbm or single) else cores
    if banded:
        sample_iters, scale_to = BANDED_ORACLE_ITERS, BANDED_ITERS_TO_TOL
    elif hbm:
        sample_iters, scale_to = HBM_ORACLE_ITERS, HBM_ITERS_TO_TOL
    else:
        sample_iters, scale_to = None, None
    count = spectra.WORKLOADS[args.workload].get("B", c.get("count", 1)) or 1

    def jobs(step):
        ps = [(step * per_step + i) % max(count, 1) for i in range(per_step)]
        if banded:
            return _oracle_banded_job, [(args.workload, p, sample_iters) for p in ps]
        if args.workload.startswith("warmstart"):
            ps = [WS_TEST_FIRST + step * per_step + i for i in range(per_step)]
        n_iter = sample_iters if sample_iters else c["iters"]
        tol = 0.0 if (sample_iters or single) else c["tol"]
        return _oracle_job, [(args.workload, p, n_iter, None, None, False, tol) for p in ps]

    for s_ in range(args.warmup):  # warm-up steps: the same work, untimed
        fn, js = jobs(args.steps + s_)
        pool.map(fn, js)
    walls, iters = [], []
    for s_ in range(args.steps):
        fn, js = jobs(s_)
        t0 = time.perf_counter()
        res = pool.map(fn, js)
        walls.append(time.perf_counter() - t0)
        iters += [r[1] for r in res]
    pool.close()
    secs = float(np.sum(walls))
    solved = per_step * args.steps
    if sample_iters:
        secs *= (2 * scale_to + 1) / (2 * sample_iters + 1)
    if single:  # this workload's metric is a solve time
        v, unit, higher = secs * 1e3 / solved, "ms", False
    else:
        v, unit, higher = solved / secs, "problems/s", True
    sample = (f"{per_step} problem(s) per step on {per_step} core(s) at once, "
              + (f"{sample_iters} oracle iterations each, scaled to {scale_to} iterations to tolerance"
                 if sample_iters else ("its fixed iterations" if single else "each solved to the tolerance")))
    return {"impl": "reference", "metric": workload_metric(args.workload), "value": v, "unit": unit, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1e3 / args.steps,
            "higher_is_better": higher, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded spectra of the workload's recipe, no dataset)",
            "config": {"workload": args.workload, "n": c.get("n"), "k": c.get("k"), "eps": c.get("eps"),
                       "tol": c.get("tol"), "problems_per_step": per_step, "oracle_iters": iters},
            "cpu_baseline": {"value": v, "unit": unit, "cores": per_step, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# The other workloads of the measured configurations, reported inside the default line so that one
# run shows every target: name -> (workload, runner)
EXTRAS = {"batch1024": "batch1024_n1024_kl_l1", "hbm_single": "hbm_single_n16384_l2_l2sq",
          "ragged": "ragged10000_tv_l1", "warmstart": "warmstart_n2048_kl_l2sq"}
EXTRA_KEYS = ("metric", "value", "unit", "ms_per_step", "steps", "warmup", "iters_per_s", "dtype", "config", "roofline",
              "plain_fp32", "speedup_vs_plain_fp32", "kernel_ms_per_step", "e2e", "gpu_launches", "clocks",
              "err_vs_fp64", "cpu_baseline", "forms", "speedup_warm_bf16_vs_plain_fp32_cold", "target_5x_met",
              "timings_s", "best_form_problems_per_s", "fp64_gap")


def run_extras(args, local_rank, pool):
    """The batch of 1024 at n = 1024, the single target at n = 16384 (HBM), the uneven batch of
    10,000 and the learned warm start, each measured by its own runner (3 warm-up and 3 timed steps),
    compacted to the keys that carry its numbers."""
    out = {}
    for name, wl in EXTRAS.items():
        a = argparse.Namespace(**vars(args))
        a.workload, a.steps, a.warmup = wl, 3, 3
        t0 = time.perf_counter()
        if wl.startswith("ragged"):
            r = run_ragged(a, 0, 1, local_rank, pool=pool)
        elif wl.startswith("warmstart"):
            r = run_warmstart(a, 0, local_rank, pool=pool)
        elif wl.startswith("hbm"):
            r = run_single_hbm(a, 0, 1, local_rank)
        else:
            r = run_ours(a, 0, 1, local_rank, pool=pool)
        out[name] = {kk: r[kk] for kk in EXTRA_KEYS if kk in r}
        out[name]["workload"] = wl
        out[name]["wall_s"] = time.perf_counter() - t0
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batch4096_n4096_l2_l2sq")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload only: skip the other workloads' sub-objects")
    ap.add_argument("--ws-train", type=int, default=200_000, help="warm start: training problems")
    ap.add_argument("--ws-test", type=int, default=20_000, help="warm start: held-out problems")
    ap.add_argument("--ws-epochs", type=int, default=8, help="warm start: training epochs")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        out = run_reference(args, rank)
    else:
        if world > 1:
            import torch
            import torch.distributed as dist
            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
        if args.workload.startswith("ragged"):
            out = run_ragged(args, rank, world, local_rank)
        elif args.workload.startswith("warmstart"):
            out = run_warmstart(args, rank, local_rank)
        elif args.workload.startswith("single"):
            out = run_single_fp64(args, rank, local_rank)
        elif args.workload.startswith("hbm"):
            out = run_single_hbm(args, rank, world, local_rank)
        elif args.workload.startswith("banded"):
            out = run_banded(args, rank, world, local_rank)
        else:
            out = run_ours(args, rank, world, local_rank)
            if (out is not None and world == 1 and args.workload == "batch4096_n4096_l2_l2sq"
                    and not args.no_extras):
                pool = CpuPool(os.cpu_count() or 1)
                out["workloads"] = run_extras(args, local_rank, pool)
                pool.close()
                ws = out["workloads"].get("warmstart", {})
                out["targets"] = {
                    "warm_bf16_vs_plain_fp32_ge_5x": ws.get("target_5x_met"),
                    "memory_bound_apply_hbm_roofline_ge_0.7": (out["workloads"].get("hbm_single", {}).get("roofline", {})
                                                       .get("frac", 0.0) >= 0.7),
                    "note": "the HBM target applies to the memory-bound apply (single target, stored kernel); the "
                            "log-domain FP32 applies are exponent-unit bound (plain_fp32.roofline)"}
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
