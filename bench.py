"""SpAMM benchmark: one JSON line per run (rank 0).

A step is one pass of the hot path over the workload with inputs resident in
HBM: norm map of A, norm map of B, the pair test / work-queue plan at tau,
and the multiply that writes C.  The default workload is the largest
single-GPU configuration: N = 32768, a_ij = exp(-alpha |i-j|) * z_ij with
z ~ N(0,1) and alpha = 0.5 (A and B independent, seeded numpy draws on the
host), FP16 tensor-core block products with power-of-two block scaling and
FP32 accumulation (the paper's tensor-core precision), tau = 1e-6, the leaf
(64 or 128) and multiply schedule picked by the library's autotuner.  The
metric is dense-equivalent throughput 2 N^3 / t (TFLOP/s); ms_per_step gives
the time, and the line states the achieved error against the FP64 oracle on
sampled block rows.  Plain FP32 SpAMM and cuBLAS SGEMM (TF32 off) are timed on
the same GPU as baselines; the near-sparse N = 32768 product and the N = 8192
algebraic-decay product are summarised in the same line (extra_workloads).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload decay|c2|batch|sparse|table2]
                       [--precision fp32|bf16|...] [--tau T] [--alpha A]
With N > 1 (torchrun) every rank runs an independent replica (the path does
not shard); the value is the sum over ranks, timed by the slowest rank.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

# the oracle's BLAS calls run single-threaded (the all-core timing uses worker
# processes instead): pin BLAS before numpy loads
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("OMP_NUM_THREADS", "1")
os.environ.setdefault("MKL_NUM_THREADS", "1")

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))


def blas_threads() -> int:
    """Threads the oracle's BLAS calls may use: 1 under the pins above, or what the caller's
    environment set instead (the largest of the three); the oracle's own loops use one."""
    vals = [1]
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        try:
            vals.append(int(os.environ.get(k, "1")))
        except ValueError:
            pass
    return max(vals)

sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "SpAMM time & TFLOP/s at fixed rel. error vs plain FP32 SpAMM & cuBLAS; roofline %"

# DRAM bytes (read + write) per launch of a kernel, from one ncu capture of the
# kernel as it stands (the N = 32768 norm-map launch scaled from a capture at
# N = 16384 by the entries read); an entry is removed whenever the kernel
# changes, until it is captured again.
NCU_TRAFFIC = {("normmap_staged_kernel", 32768, 128): 8594854912.0}

# The synthetic workloads of a single product (one step = norm maps of A and B,
# plan, multiply).  decay: exp(-alpha |i-j|) N(0,1), N = 32768, A and B
# independent, the largest single-GPU configuration; c2: the algebraic-decay
# mixed-precision configuration at N = 8192.
WORKLOADS = {
    "decay": {"n": 32768, "leaves": (64, 128), "precision": "fp16", "tau": 1e-6, "config": 2},
    "c2": {"n": 8192, "leaves": (64,), "precision": "bf16_split", "tau": 1e-2, "config": 1},
}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return {"hbm_gbs": p["hbm_gbs"], "bf16_tflops": p["bf16_tflops"],
                "bf16_tflops_sustained": p.get("bf16_tflops_sustained"),
                "sm_max_mhz": p.get("sm_max_mhz", 2070.0), "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0, "source": "fallback"}


def workload(name: str, n: int, alpha: float = 0.5):
    """Host FP32 (A, B) of a single-product workload (seeded numpy PCG64, row-major draws)."""
    cfg = WORKLOADS[name]["config"]
    if name == "decay":
        return (synth.exp_decay_normal(n, alpha, synth.config_seed(cfg, operand="A")),
                synth.exp_decay_normal(n, alpha, synth.config_seed(cfg, operand="B")))
    return (synth.alg_decay_signed(n, 3.0, synth.config_seed(cfg, operand="A")),
            synth.alg_decay_signed(n, 3.0, synth.config_seed(cfg, operand="B")))


def workload_desc(name: str, n: int, alpha: float) -> str:
    if name == "decay":
        return f"exponential decay exp(-{alpha:g}|i-j|) * N(0,1), N={n}"
    return f"algebraic decay (|i-j|+1)^-3 * (+-1), N={n}"


# ---------------------------------------------------------------------------
# Replicas (one process per GPU, no data exchange): the job's time is the
# slowest rank's, its throughput the sum over ranks
# ---------------------------------------------------------------------------

def slowest_rank_ms(ms: float, world: int, device) -> float:
    """Max of the per-rank times over the process group (identity for one rank)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(per_rank_work: float, ms: float, world: int) -> float:
    """Units per second of the whole job: every rank does per_rank_work units in ms (max)."""
    return per_rank_work * world / (ms * 1e-3)


# ---------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
                self.lines = [ln for ln in out.splitlines() if ln.strip()]
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU baseline: the oracle as it stands on a bounded sample of the workload
# ---------------------------------------------------------------------------

def spread_rows(bd: int, count: int, offset: int = 0):
    """`count` output block-rows spread evenly over [0, bd) (edges and middle alike)."""
    count = max(1, min(bd, count))
    return sorted({(offset + (q * bd) // count) % bd for q in range(count)})


# Worker processes for the oracle's all-core timing.  They are forked before the
# first CUDA call of the process (a process forked after it can hang), inherit
# the host inputs copy-on-write through these globals and never touch the GPU;
# every worker runs the oracle single-threaded (BLAS pinned to one thread).
_ORACLE_A = None
_ORACLE_B = None


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OraclePool:
    def __init__(self, a, b, cores=None):
        import multiprocessing as mp
        global _ORACLE_A, _ORACLE_B
        _ORACLE_A, _ORACLE_B = a, b
        self.cores = cores or host_cores()
        self.pool = mp.get_context("fork").Pool(self.cores)

    def map(self, fn, items):
        return self.pool.map(fn, items, chunksize=1)

    def close(self):
        self.pool.terminate()
        self.pool.join()


def _w_norm_row(task):
    """One block row of A's (which == 'A') or B's norm map (oracle, Eq. 2)."""
    from oracle import spamm as OS
    which, leaf, i = task
    return OS.normmap_rows(_ORACLE_A if which == "A" else _ORACLE_B, leaf, [i])[0]


def _w_share(task):
    """The oracle's work for one output block row: that row of A's norm map, B's matching
    share of its norm pass, the row's pair tests and block products.  Returns its seconds."""
    from oracle import spamm as OS
    leaf, tau, i, nB = task
    t0 = time.perf_counter()
    nA_row = OS.normmap_rows(_ORACLE_A, leaf, [i])
    OS.normmap_rows(_ORACLE_B, leaf, [i])
    OS.spamm_rows(_ORACLE_A, _ORACLE_B, leaf, tau, [i], nA_row, nB)
    return time.perf_counter() - t0


def needed_normmap_b(pool, a, b, leaf, tau, rows):
    """B's norm map restricted to the block rows that can decide a triple of the sampled rows
    (oracle.spamm.needed_b_rows), computed on the pool (set-up, not timed)."""
    from oracle import spamm as OS
    bd = OS.num_blocks(a.shape[0], leaf)
    if pool is not None:
        nA_rows = np.array(pool.map(_w_norm_row, [("A", leaf, i) for i in rows]))
    else:
        nA_rows = OS.normmap_rows(a, leaf, rows)
    ks = OS.needed_b_rows(nA_rows, tau)
    if tau > 0.0 and ks.size < bd and not np.isfinite(b).all():
        ks = np.arange(bd)
    nB = np.zeros((bd, bd))
    if ks.size:
        if pool is not None:
            nB[ks] = np.array(pool.map(_w_norm_row, [("B", leaf, int(k)) for k in ks]))
        else:
            nB[ks] = OS.normmap_rows(b, leaf, ks)
    return nB


def cpu_baseline(a, b, leaf, tau, pool=None, single_rows=4, nB_full=None, gpu_c=None,
                 offset=0):
    """The oracle as it stands, timed on a bounded sample of the job: output block rows, each
    one share = that block row of A's norm map, B's matching share of its norm pass, the
    row's pair tests against B's blocks and its block products; the full job is bd such
    shares.  All cores: one row per worker process at a time (value, cores = workers);
    single thread: `single_rows` rows in this process.  B's norm map for the pair tests is
    set-up (its rows that can decide the sampled triples only), not timed.  Also the GPU's
    error on the single-thread rows against the oracle.  Returns (dict, nB_full)."""
    from oracle import spamm as OS
    n = a.shape[0]
    bd = OS.num_blocks(n, leaf)
    cores = pool.cores if pool is not None else 1
    rows_all = spread_rows(bd, max(cores, single_rows), offset)
    if nB_full is None:
        nB_full = needed_normmap_b(pool, a, b, leaf, tau, rows_all)
    res = {"unit": "TFLOP/s (dense-equivalent)", "kind": "oracle", "nproc": host_cores()}
    if pool is not None:
        t0 = time.perf_counter()
        secs = pool.map(_w_share, [(leaf, tau, i, nB_full) for i in rows_all])
        wall = time.perf_counter() - t0
        t_full = wall * bd / len(rows_all)
        res.update({"value": 2.0 * n ** 3 / t_full / 1e12, "cores": cores,
                    "sample": f"{len(rows_all)} of {bd} output block rows on {cores} worker "
                              f"processes (per row: its norm-map rows of A and B, pair tests "
                              f"and block products), {wall:.1f} s wall, extrapolated "
                              f"x{bd / len(rows_all):.1f}",
                    "seconds_full_extrapolated": t_full,
                    "row_seconds_median": statistics.median(secs)})
    rows = rows_all[:single_rows]
    t0 = time.perf_counter()
    nA_rows = OS.normmap_rows(a, leaf, rows)
    _ = OS.normmap_rows(b, leaf, rows)          # B's share of the norm pass
    out = OS.spamm_rows(a, b, leaf, tau, rows, nA_rows, nB_full)
    dt = time.perf_counter() - t0
    t1 = dt * bd / len(rows)
    single = {"value": 2.0 * n ** 3 / t1 / 1e12, "cores": 1,
              "sample": f"{len(rows)} of {bd} output block rows in one thread, {dt:.1f} s, "
                        f"extrapolated x{bd / len(rows):.0f}",
              "seconds_full_extrapolated": t1}
    if pool is None:
        res.update(single)
    else:
        res["single_thread"] = single
    if gpu_c is not None:
        errs, refs = 0.0, 0.0
        for i, (c, _) in out.items():
            g = gpu_c[i * leaf:min(n, (i + 1) * leaf)].astype(np.float64)
            errs += float(np.sum((g - c) ** 2))
            refs += float(np.sum(c ** 2))
        res["rel_err_vs_oracle_sampled_rows"] = (errs / refs) ** 0.5 if refs > 0 else 0.0
        res["abs_err_sampled_rows"] = errs ** 0.5
        res["sampled_rows"] = [int(i) for i in rows]
    return res, nB_full


# ---------------------------------------------------------------------------
# The GPU arm
# ---------------------------------------------------------------------------

def run_ours(args, rank, world):
    import torch
    import paper_2103_13042_gb300 as P

    local = int(os.environ.get("LOCAL_RANK", "0"))
    wl = WORKLOADS[args.workload]
    n = args.n or wl["n"]
    tau = wl["tau"] if args.tau is None else args.tau
    prec_name = args.precision or wl["precision"]
    prec = P.PRECISIONS[prec_name]
    t_gen = time.perf_counter()
    a_h, b_h = workload(args.workload, n, args.alpha)
    t_gen = time.perf_counter() - t_gen
    # the oracle's worker processes, forked before this process's first CUDA call
    pool = OraclePool(a_h, b_h) if (world == 1 and not args.no_cpu_baseline) else None
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    A = torch.from_numpy(a_h).to(dev)
    B = torch.from_numpy(b_h).to(dev)
    C = torch.empty_like(A)
    # leaf: given, or the project's autotuner on this instance (leaf x multiply schedule,
    # each candidate timed under graph replay); the single-product API then runs the
    # chosen leaf
    tune = None
    if args.leaf:
        leaf = args.leaf
    elif len(wl["leaves"]) == 1:
        leaf = wl["leaves"][0]
    else:
        best, allc = P.spamm_batch_autotune([A], [B], [C], [tau], prec, args.target, reps=3)
        tune = {"best": best, "candidates": allc}
        leaf = best["leaf"]
        torch.cuda.empty_cache()
    bd = P.num_blocks(n, leaf)
    nA = torch.empty((bd, bd), dtype=torch.float64, device=dev)
    nB = torch.empty_like(nA)
    plan = P.Plan(n, leaf, prec)
    schedule = tune["best"]["schedule"] if tune is not None else args.schedule
    plan.set_schedule(schedule)   # the autotuner's multiply schedule, or --schedule
    stream = torch.cuda.current_stream()

    def step(st=None):
        st = st if st is not None else torch.cuda.current_stream()
        P.spamm_normmap_pair(A, B, leaf, nA, nB, st)
        plan.plan_multiply(nA, nB, tau, A, B, C, args.target, st)

    # our kernels per step: one norm-map launch for both operands, 4 plan kernels,
    # zero-fill, multiply (tensor cores: + operand rounding)
    launches_per_step = 1 + 4 + 1 + (1 if prec == P.FP32 else 2)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    st = plan.stats()
    # peak rates of the modes no library routine gives (the library's microkernels)
    try:
        micro = P.spamm_peak_rates()
    except Exception as exc:   # reported, the line stands without them
        micro = {"error": f"{type(exc).__name__}: {exc}"}

    # per-call breakdown (events on the launching stream)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    parts = {"normmap_pair": [], "plan_multiply": [], "plan_alone": [], "multiply_alone": []}
    # a clean read of more than L2 before each breakdown iteration: the previous
    # iteration's dirty C lines are written back there, not inside the norm maps
    l2_flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev).fill_(1.0)
    for _ in range(max(3, args.steps // 2)):
        # the GPU first spins for ~1 ms while the host enqueues the calls below,
        # so no interval includes host launch latency
        torch.cuda._sleep(2_000_000)
        l2_flush.sum()
        ev[0].record(stream)
        P.spamm_normmap_pair(A, B, leaf, nA, nB, stream)
        ev[1].record(stream)
        plan.plan_multiply(nA, nB, tau, A, B, C, args.target, stream)
        ev[2].record(stream)
        plan.plan(nA, nB, tau, args.target, stream)     # the two halves, for the breakdown
        ev[3].record(stream)
        plan.multiply(A, B, C, stream)
        ev[4].record(stream)
        torch.cuda.synchronize()
        for k, name in enumerate(parts):
            parts[name].append(ev[k].elapsed_time(ev[k + 1]))
    part_ms = {k: statistics.median(v) for k, v in parts.items()}

    # eager per-step time (host enqueues every call)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    eager_ms = e0.elapsed_time(e1) / args.steps

    # the same API calls captured once into a CUDA graph (the library enqueues
    # no allocation or synchronisation after the first call), replayed K times
    graph = None
    if not args.eager:
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step()
        for _ in range(3):
            graph.replay()
        torch.cuda.synchronize()

    def timed_step():
        if graph is not None:
            graph.replay()
        else:
            step()

    # timed region: K steps
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        time.sleep(0.3)
        e0.record(stream)
        for _ in range(args.steps):
            timed_step()
        e1.record(stream)
        torch.cuda.synchronize()
        time.sleep(0.3)
    barrier()
    ms = slowest_rank_ms(e0.elapsed_time(e1) / args.steps, world, dev)

    # end to end through the public API with host buffers (pinned), as a serving
    # loop runs it: every step copies its inputs in from pinned host memory and
    # its result out; inputs and outputs are double-buffered on the device so
    # that step k+1's host-to-device copies run under step k's compute and its
    # device-to-host copy (the link is full duplex: ~0.21 TB/s each way here)
    a_pin = torch.from_numpy(a_h).pin_memory()
    b_pin = torch.from_numpy(b_h).pin_memory()
    c_pin = [torch.empty_like(a_pin).pin_memory() for _ in range(2)]
    e2e_steps = max(4, args.steps // 2)
    dA = [A, torch.empty_like(A)]
    dB = [B, torch.empty_like(B)]
    dC = [C, torch.empty_like(C)]
    dnA = [nA, torch.empty_like(nA)]
    dnB = [nB, torch.empty_like(nB)]
    plans = [plan, P.Plan(n, leaf, prec)]
    s_in, s_out = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    ev = lambda: torch.cuda.Event()
    ev_in = [ev(), ev()]          # inputs of buffer q are on the device
    ev_done = [ev(), ev()]        # compute of buffer q finished (inputs free, C ready)
    ev_out = [ev(), ev()]         # C of buffer q is back in host memory

    def e2e_run(steps):
        for k in range(steps):
            q = k & 1
            with torch.cuda.stream(s_in):
                if k >= 2:
                    s_in.wait_event(ev_done[q])            # buffer q's inputs no longer read
                dA[q].copy_(a_pin, non_blocking=True)
                dB[q].copy_(b_pin, non_blocking=True)
                ev_in[q].record(s_in)
            stream.wait_event(ev_in[q])
            if k >= 2:
                stream.wait_event(ev_out[q])               # buffer q's C has been copied out
            P.spamm_normmap_pair(dA[q], dB[q], leaf, dnA[q], dnB[q], stream)
            plans[q].plan_multiply(dnA[q], dnB[q], tau, dA[q], dB[q], dC[q], args.target, stream)
            ev_done[q].record(stream)
            with torch.cuda.stream(s_out):
                s_out.wait_event(ev_done[q])
                c_pin[q].copy_(dC[q], non_blocking=True)
                ev_out[q].record(s_out)
        stream.wait_stream(s_in)
        stream.wait_stream(s_out)

    e2e_run(2)
    torch.cuda.synchronize()
    barrier()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    s_in.wait_stream(stream)
    e2e_run(e2e_steps)
    f1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = slowest_rank_ms(f0.elapsed_time(f1) / e2e_steps, world, dev)
    last = (e2e_steps - 1) & 1
    assert torch.equal(c_pin[last], dC[last].cpu()), "e2e: the copied-out C differs from the device C"
    del dA[1], dB[1], dC[1], dnA[1], dnB[1], plans[1]

    # baselines on the same GPU: plain FP32 SpAMM (same tau) and cuBLAS SGEMM
    base = {}
    if not args.no_baselines:
        plan32 = P.Plan(n, leaf, P.FP32)
        C32 = torch.empty_like(A)

        def step32():
            P.spamm_normmap_pair(A, B, leaf, nA, nB, stream)
            plan32.plan_multiply(nA, nB, tau, A, B, C32, args.target, stream)

        def timed(fn, reps):
            for _ in range(3):
                fn()
            g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            g0.record(stream)
            for _ in range(reps):
                fn()
            g1.record(stream)
            torch.cuda.synchronize()
            return g0.elapsed_time(g1) / reps

        base["fp32_spamm_ms"] = timed(step32, max(3, args.steps // 2))
        base["fp32_spamm_leaf"] = leaf
        prev = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = False
        base["cublas_sgemm_ms"] = timed(lambda: torch.matmul(A, B, out=C32), 3)
        torch.backends.cuda.matmul.allow_tf32 = prev
        base["speedup_vs_fp32_spamm"] = base["fp32_spamm_ms"] / ms
        base["speedup_vs_cublas_sgemm"] = base["cublas_sgemm_ms"] / ms
        del plan32, C32

    # the error-targeted tau of the same product: the library's bisection on the measured
    # pruning error (spamm_tau_select, no network: its weights are for leaf 64) for a target
    # of half the relative-error budget (the FP16 rounding takes the rest), and the step's time
    # at that tau
    tau_eps = None
    if args.workload == "decay" and not args.no_baselines:
        sel = P.Plan(n, leaf, P.FP32)
        scratch = torch.empty_like(A)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        t_e, evals, err_e = sel.tau_select(nA, nB, A, B, 0.5 * args.target, None, scratch)
        t_sel = time.perf_counter() - t0
        del sel, scratch
        st_e = None

        def step_e():
            P.spamm_normmap_pair(A, B, leaf, nA, nB, stream)
            plan.plan_multiply(nA, nB, t_e, A, B, C, args.target, stream)

        for _ in range(3):
            step_e()
        torch.cuda.synchronize()
        st_e = plan.stats()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for _ in range(max(3, args.steps // 2)):
            step_e()
        g1.record(stream)
        torch.cuda.synchronize()
        tau_eps = {"target_pruning_rel_err": 0.5 * args.target, "tau": t_e, "evaluations": evals,
                   "pruning_rel_err": err_e, "select_s": t_sel,
                   "ms_per_step": g0.elapsed_time(g1) / max(3, args.steps // 2),
                   "survivors": st_e["survivors"],
                   "skipped_bound2_rel": st_e["skipped_bound2"] / (st_e["norm_a"] * st_e["norm_b"])}
        # back to the line's tau (C as the timed steps left it, for the oracle's check)
        step()
        torch.cuda.synchronize()

    if rank != 0:
        return None
    peaks = load_peaks()
    dense = 2.0 * n ** 3
    value = job_throughput(dense, ms, world) / 1e12
    # the multiply phase against its own mode's peak (useful flops over surviving triples
    # only; TF32x3 issues three MMAs per product): the microkernel rates for FP16, TF32 and
    # FP32 FFMA, MEASURED_PEAKS' cuBLAS figure for BF16
    useful = 2.0 * leaf ** 3 * st["survivors"]
    mode_peak = {P.FP32: micro.get("ffma_fp32"), P.FP16: micro.get("mma_fp16"),
                 P.FP16_SPLIT: micro.get("mma_fp16"), P.TF32X3: micro.get("mma_tf32"),
                 P.BF16: peaks["bf16_tflops"], P.BF16_SPLIT: peaks["bf16_tflops"]}.get(prec)
    issued = useful * (3.0 if prec == P.TF32X3 else 1.0)
    mul_frac = None
    if mode_peak and part_ms["multiply_alone"] > 0:
        mul_frac = issued / (part_ms["multiply_alone"] * 1e-3) / 1e12 / mode_peak
    # roofline of the dominant kernel: by the ncu launch list of this command the
    # norm map (one launch per step over both operands) has the largest share of device time
    norm_ms = part_ms["normmap_pair"]
    mul_ms = part_ms["multiply_alone"]
    if norm_ms > 0.0:
        bytes_ = 2.0 * (4.0 * n * n + 8.0 * bd * bd)
        ach = bytes_ / (norm_ms * 1e-3) / 1e9
        traffic = NCU_TRAFFIC.get(("normmap_staged_kernel", n, leaf))
        roof = {"kernel": "normmap_staged_kernel", "bound": "hbm", "achieved": ach,
                "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": ach / peaks["hbm_gbs"],
                "traffic": traffic, "per_launch_ms": norm_ms, "algorithmic_bytes": bytes_,
                "peak_source": peaks["source"] + " copy bandwidth (burst)",
                "timing": "CUDA events around one spamm_normmap_pair call on the launching stream, "
                          "queued behind a 1 ms spin and a clean 256 MB read (no host gap, "
                          "no dirty C lines left in L2 by the previous call)"}
    else:
        flops = 2.0 * leaf ** 3 * st["survivors"]
        if prec == P.FP32:
            peak = micro.get("ffma_fp32") or 152 * 128 * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12
            ach = flops / (mul_ms * 1e-3) / 1e12
            roof = {"kernel": "multiply_simt", "bound": "alu", "achieved": ach, "peak": peak,
                    "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
                    "per_launch_ms": mul_ms, "algorithmic_flops": flops,
                    "peak_source": "measured FFMA microkernel (spamm_peak_rates)"
                    if micro.get("ffma_fp32") else "derived: 152 SMs x 128 lanes x 2 x clock"}
        else:
            peak = peaks["bf16_tflops"]
            ach = flops / (mul_ms * 1e-3) / 1e12
            roof = {"kernel": "multiply_tc", "bound": "tensor", "achieved": ach, "peak": peak,
                    "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
                    "per_launch_ms": mul_ms, "algorithmic_flops": flops,
                    "peak_source": peaks["source"]}
    gb = 4.0 * n * n / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s (dense-equivalent, 2N^3/t)",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "tf32x3": "tf32", "bf16_split": "bf16", "bf16": "bf16",
                  "fp16_split": "f16", "fp16": "f16"}.get(prec_name, prec_name),
        "data": "synthetic (seeded numpy PCG64 draws on the host, copied to the GPU)",
        "config": {"workload": f"{workload_desc(args.workload, n, args.alpha)}, A and B "
                               f"independent, leaf {leaf}"
                               f"{' (autotuned)' if tune else ''}, tau={tau:g}, {prec_name}",
                   "name": args.workload, "n": n, "leaf": leaf, "tau": tau,
                   "precision": prec_name, "alpha": args.alpha if args.workload == "decay" else None,
                   "target_rel_err": args.target, "parallelism": f"replicas x{world}",
                   "launch": "eager" if graph is None else "cuda-graph replay of the API calls",
                   "ms_per_step_eager": eager_ms, "schedule": schedule, "autotune": tune,
                   "host_generation_s": t_gen,
                   "l2": f"inputs larger than L2 (A, B, C {gb:.2f} GB each vs 126 MB L2)",
                   "survivors": st["survivors"], "valid_ratio": st["valid_ratio"],
                   "nonempty_tiles": st["nonempty_tiles"],
                   "skipped_bound2_rel": st["skipped_bound2"] / (st["norm_a"] * st["norm_b"]),
                   "multiply_useful_tflops": useful / (part_ms["multiply_alone"] * 1e-3) / 1e12
                   if part_ms["multiply_alone"] > 0 else None,
                   "multiply_frac_of_mode_peak": mul_frac},
        "peaks_microkernel_tflops": micro,
        "breakdown_ms": part_ms,
        "baselines_same_gpu": base,
        "e2e": {"value": dense / (e2e_ms * 1e-3) / 1e12 * world,
                "unit": "TFLOP/s (dense-equivalent, 2N^3/t)", "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": 2 * 4 * n * n, "d2h_bytes_per_step": 4 * n * n},
        "gpu_launches": launches_per_step * args.steps,
        "roofline": roof,
        # the whole step against the HBM floor of reading A, B and writing C once
        "roofline_step": {"bound": "hbm", "algorithmic_bytes": 12.0 * n * n,
                          "achieved": 12.0 * n * n / (ms * 1e-3) / 1e9, "peak": peaks["hbm_gbs"],
                          "unit": "GB/s", "frac": 12.0 * n * n / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"]},
        "clocks": clk.summary(),
    }
    if tau_eps is not None:
        line["tau_for_target_error"] = tau_eps
    if not args.no_cpu_baseline:
        c_host = C.cpu().numpy()
        cb, _ = cpu_baseline(a_h, b_h, leaf, tau, pool, single_rows=args.cpu_rows, gpu_c=c_host)
        # the sampled rows' error relative to ||A||_F ||B||_F, scaled to the whole product
        # (rows alike by construction): the line's accuracy in the metric's normalisation
        if "abs_err_sampled_rows" in cb:
            ab = st["norm_a"] * st["norm_b"]
            cb["rel_err_ab_whole_product_est"] = (
                cb["abs_err_sampled_rows"] * math.sqrt(bd / len(cb["sampled_rows"])) / ab)
            line["config"]["rel_err_vs_oracle_ab_est"] = cb["rel_err_ab_whole_product_est"]
        line["cpu_baseline"] = cb
    if pool is not None:
        pool.close()
    return line


# ---------------------------------------------------------------------------
# Batched workload: 256 uneven decay instances in one pass of each kernel
# ---------------------------------------------------------------------------

BATCH_COUNT = 256


def _gen_instance(spec):
    return synth.spec_matrices(spec)


def batch_workload(count: int):
    """Seeded specs and matrices of the batched workload (generated on the host
    cores by a spawn pool, so no process is forked after CUDA starts)."""
    import multiprocessing as mp
    specs = synth.batch_specs(count, synth.config_seed(3))
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        mats = pool.map(_gen_instance, specs, chunksize=4)
    return specs, mats


def certified_taus(P, As, Bs, ns, leaf, eps, iters=40):
    """Per instance, the largest tau (bisection in log tau) whose skipped-product
    bound keeps ||C - AB||_F <= bound2 <= eps/2 * ||A||_F ||B||_F, measured with
    the library's own FP32 plan statistics (half the budget is left to rounding)."""
    import torch
    Cs = [torch.empty_like(A) for A in As]
    b = P.Batch(ns, leaf, P.FP32, graph=False)
    b.run(As, Bs, Cs, [0.0] * len(ns))
    st = b.stats()
    ab = np.array([s["norm_a"] * s["norm_b"] for s in st])
    lo = np.full(len(ns), -60.0)     # log2(tau / (|A||B|)): 2^-60 always meets the target
    hi = np.zeros(len(ns))
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        b.run(As, Bs, Cs, list(ab * np.exp2(mid)))
        st = b.stats()
        ok = np.array([s["skipped_bound2"] <= 0.5 * eps * s["norm_a"] * s["norm_b"] for s in st])
        lo = np.where(ok, mid, lo)
        hi = np.where(ok, hi, mid)
    b.close()
    del Cs
    return list(ab * np.exp2(lo))


def run_batch(args, rank, world):
    import torch
    import paper_2103_13042_gb300 as P

    specs, mats = batch_workload(args.count)
    dense_job = float(sum(2.0 * s["n"] ** 3 for s in specs))
    shard = args.partition == "instances" and world > 1
    if shard:   # this rank's instances (longest first to the least-loaded rank)
        from paper_2103_13042_gb300 import partition as PT
        mine = PT.instances_by_rank([s["n"] for s in specs], world)[rank]
        specs, mats = [specs[i] for i in mine], [mats[i] for i in mine]
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    args.precision = args.precision or "bf16_split"
    prec = P.PRECISIONS[args.precision]
    ns = [s["n"] for s in specs]
    As = [torch.from_numpy(a).to(dev) for a, _ in mats]
    Bs = [torch.from_numpy(b).to(dev) for _, b in mats]
    Cs = [torch.empty_like(A) for A in As]
    stream = torch.cuda.current_stream()
    sum_n2 = float(sum(n * n for n in ns))
    dense = float(sum(2.0 * n ** 3 for n in ns))

    t_tune = time.perf_counter()
    taus = certified_taus(P, As, Bs, ns, 64, args.target)
    t_tau = time.perf_counter() - t_tune

    # autotuner: leaf x multiply schedule, timed on this batch (--leaf fixes the leaf and
    # --schedule the schedule)
    if args.leaf:
        best, cands = {"leaf": args.leaf, "schedule": args.schedule, "ms": -1.0}, []
    else:
        best, cands = P.spamm_batch_autotune(As, Bs, Cs, taus, prec, args.target, reps=3)
    leaf = best["leaf"]
    batch = P.Batch(ns, leaf, prec, graph=True, dynamic=best["schedule"] == "dynamic",
                    groups=best["schedule"] == "groups")

    def step():
        batch.run(As, Bs, Cs, taus, args.target)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    st = batch.stats()
    assert P.spamm_last_device_status() == 0

    # phase breakdown (same configuration, events between phases, no graph)
    tb = P.Batch(ns, leaf, prec, graph=False, dynamic=best["schedule"] == "dynamic",
                    groups=best["schedule"] == "groups", timing=True)
    ph = {"normmap": [], "plan": [], "round": [], "multiply": []}
    for _ in range(max(3, args.steps // 4)):
        tb.run(As, Bs, Cs, taus, args.target)
        for k, v in tb.timings().items():
            ph[k].append(v)
    tb.close()
    part_ms = {k: statistics.median(v) for k, v in ph.items()}

    # timed region (inputs resident in HBM, ~2.8 GB per operand >> L2)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        time.sleep(0.3)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        time.sleep(0.3)
    ms = slowest_rank_ms(e0.elapsed_time(e1) / args.steps, world, dev)

    # accuracy on a sample of instances against an FP64 product on the GPU
    errs = []
    for i in range(0, len(ns), max(1, len(ns) // 8)):
        ref = torch.matmul(As[i].double(), Bs[i].double())
        e = torch.linalg.norm(Cs[i].double() - ref).item()
        errs.append(e / (st[i]["norm_a"] * st[i]["norm_b"]))
        del ref

    # end to end: inputs from pinned host memory, results back to pinned memory,
    # as a serving loop runs it (double-buffered on the device: step k+1's
    # host-to-device copies run under step k's compute and device-to-host copy)
    a_pin = [torch.from_numpy(a).pin_memory() for a, _ in mats]
    b_pin = [torch.from_numpy(b).pin_memory() for _, b in mats]
    c_pin = [[torch.empty(n, n, dtype=torch.float32).pin_memory() for n in ns] for _ in range(2)]
    dAs = [As, [torch.empty_like(x) for x in As]]
    dBs = [Bs, [torch.empty_like(x) for x in Bs]]
    dCs = [Cs, [torch.empty_like(x) for x in Cs]]
    batches = [batch, P.Batch(ns, leaf, prec, graph=True, dynamic=best["schedule"] == "dynamic",
                    groups=best["schedule"] == "groups")]
    s_in, s_out = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    ev_in = [torch.cuda.Event(), torch.cuda.Event()]
    ev_done = [torch.cuda.Event(), torch.cuda.Event()]
    ev_out = [torch.cuda.Event(), torch.cuda.Event()]

    def e2e_run(steps):
        for k in range(steps):
            q = k & 1
            with torch.cuda.stream(s_in):
                if k >= 2:
                    s_in.wait_event(ev_done[q])
                for i in range(len(ns)):
                    dAs[q][i].copy_(a_pin[i], non_blocking=True)
                    dBs[q][i].copy_(b_pin[i], non_blocking=True)
                ev_in[q].record(s_in)
            stream.wait_event(ev_in[q])
            if k >= 2:
                stream.wait_event(ev_out[q])
            batches[q].run(dAs[q], dBs[q], dCs[q], taus, args.target)
            ev_done[q].record(stream)
            with torch.cuda.stream(s_out):
                s_out.wait_event(ev_done[q])
                for i in range(len(ns)):
                    c_pin[q][i].copy_(dCs[q][i], non_blocking=True)
                ev_out[q].record(s_out)
        stream.wait_stream(s_in)
        stream.wait_stream(s_out)

    e2e_run(2)
    torch.cuda.synchronize()
    e2e_steps = max(4, args.steps // 4)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    s_in.wait_stream(stream)
    e2e_run(e2e_steps)
    f1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = slowest_rank_ms(f0.elapsed_time(f1) / e2e_steps, world, dev)
    last = (e2e_steps - 1) & 1
    assert all(torch.equal(c_pin[last][i], dCs[last][i].cpu()) for i in (0, len(ns) - 1))
    batches[1].close()
    del dAs[1], dBs[1], dCs[1], batches[1]
    del a_pin, b_pin, c_pin

    def timed(fn, reps):
        for _ in range(2):
            fn()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        g0.record(stream)
        for _ in range(reps):
            fn()
        g1.record(stream)
        torch.cuda.synchronize()
        return g0.elapsed_time(g1) / reps

    base = {}
    if not args.no_baselines:
        # the same instances one call sequence at a time (norm maps, plan, multiply each)
        plans = [P.Plan(n, leaf, prec) for n in ns]
        nAs = [torch.empty((P.num_blocks(n, leaf),) * 2, dtype=torch.float64, device=dev) for n in ns]
        nBs = [torch.empty_like(x) for x in nAs]

        def seq():
            for i in range(len(ns)):
                P.spamm_normmap(As[i], leaf, nAs[i], stream)
                P.spamm_normmap(Bs[i], leaf, nBs[i], stream)
                plans[i].plan(nAs[i], nBs[i], taus[i], args.target, stream)
                plans[i].multiply(As[i], Bs[i], Cs[i], stream)

        base["sequential_single_calls_ms"] = timed(seq, 3)
        del plans, nAs, nBs
        f32 = P.Batch(ns, 64, P.FP32, graph=True)
        base["fp32_spamm_batch_ms"] = timed(lambda: f32.run(As, Bs, Cs, taus), 5)
        f32.close()
        prev = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = False

        def sgemm():
            for i in range(len(ns)):
                torch.matmul(As[i], Bs[i], out=Cs[i])

        base["cublas_sgemm_ms"] = timed(sgemm, 2)
        torch.backends.cuda.matmul.allow_tf32 = prev
        for k in ("sequential_single_calls_ms", "fp32_spamm_batch_ms", "cublas_sgemm_ms"):
            base["speedup_vs_" + k[:-3]] = base[k] / ms

    if rank != 0:
        return None
    peaks = load_peaks()
    bd2 = float(sum(P.num_blocks(n, leaf) ** 2 for n in ns))
    norm_bytes = 2 * 4.0 * sum_n2 + 2 * 8.0 * bd2
    norm_ach = norm_bytes / (part_ms["normmap"] * 1e-3) / 1e9
    roof = {"kernel": "normmap (batched, both operands of all instances)", "bound": "hbm",
            "achieved": norm_ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": norm_ach / peaks["hbm_gbs"], "traffic": None,
            "per_launch_ms": part_ms["normmap"], "algorithmic_bytes": norm_bytes,
            "peak_source": peaks["source"]}
    survivors = sum(s["survivors"] for s in st)
    line = {
        "metric": METRIC,
        "value": (dense_job if shard else dense * world) / (ms * 1e-3) / 1e12,
        "unit": "TFLOP/s (dense-equivalent, sum of 2N^3 / t)",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "strong" if shard else "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "tf32x3": "tf32", "bf16_split": "bf16", "bf16": "bf16",
                  "fp16_split": "f16", "fp16": "f16"}.get(args.precision, args.precision),
        "data": "synthetic (seeded exponential / algebraic decay instances)",
        "config": {"workload": f"batch of {len(ns)} decay instances, N log-uniform "
                               f"[256, 4096] (sum N^2 = {sum_n2:.3g}), {args.precision}, "
                               f"per-instance certified tau for rel. error {args.target:g}",
                   "count": len(ns), "n_min": min(ns), "n_max": max(ns),
                   "precision": args.precision, "target_rel_err": args.target,
                   "leaf": leaf, "schedule": best["schedule"], "autotune": cands,
                   "tau_selection_s": t_tau, "launch": "cuda-graph replay (one run per step)",
                   "parallelism": (f"instances sharded over {world} ranks" if shard
                                   else f"replicas x{world}"),
                   "l2": f"inputs larger than L2 ({4 * sum_n2 / 1e9:.1f} GB per operand)",
                   "survivors": survivors,
                   "rel_err_sampled_max": max(errs), "rel_err_sampled_instances": len(errs)},
        "breakdown_ms": part_ms,
        "baselines_same_gpu": base,
        "e2e": {"value": (dense_job if shard else dense * world) / (e2e_ms * 1e-3) / 1e12,
                "unit": "TFLOP/s (dense-equivalent, sum of 2N^3 / t)", "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": int(2 * 4 * sum_n2), "d2h_bytes_per_step": int(4 * sum_n2)},
        # norm maps (one launch for the operands with 16-byte aligned rows, one for
        # the others), 4 plan kernels, zero-fill, rounding, multiply
        "gpu_launches": (len({int(m[0].shape[0]) % 4 == 0 for m in mats}) + 4 + 1 + 2) * args.steps,
        "roofline": roof,
        "clocks": clk.summary(),
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = batch_cpu_baseline(mats, taus, leaf, ns)
    batch.close()
    return line


def batch_cpu_baseline(mats, taus, leaf, ns, budget_s=15.0):
    """The oracle on whole instances (smallest first) until ~budget_s of work,
    extrapolated to the batch by sum of N^2 (norm passes and block products of
    these decay inputs both scale with N^2 at fixed leaf)."""
    from oracle import spamm as OS
    order = sorted(range(len(ns)), key=lambda i: ns[i])
    done, t_used, n2 = [], 0.0, 0.0
    for i in order[::max(1, len(order) // 32)]:
        a, b = mats[i]
        t0 = time.perf_counter()
        OS.spamm(a, b, leaf, taus[i])
        t_used += time.perf_counter() - t0
        done.append(ns[i])
        n2 += float(ns[i]) ** 2
        if t_used >= budget_s:
            break
    total_n2 = float(sum(float(n) ** 2 for n in ns))
    t_full = t_used * total_n2 / n2
    dense = float(sum(2.0 * n ** 3 for n in ns))
    return {"value": dense / t_full / 1e12, "unit": "TFLOP/s (dense-equivalent, sum of 2N^3 / t)",
            "cores": blas_threads(), "kind": "oracle",
            "sample": f"{len(done)} whole instances (N = {min(done)}..{max(done)}), "
                      f"{t_used:.1f} s, extrapolated by sum N^2 (x{total_n2 / n2:.1f})",
            "seconds_full_extrapolated": t_full}


# ---------------------------------------------------------------------------
# Near-sparse workload: tensor-core bound (most block products survive)
# ---------------------------------------------------------------------------

def run_sparse(args, rank, world):
    import torch
    import paper_2103_13042_gb300 as P

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = args.n or 32768
    prec = P.PRECISIONS[args.precision or "bf16"]
    prec_name = [k for k, v in P.PRECISIONS.items() if v == prec][0]
    A = synth.near_sparse_device(n, synth.config_seed(2, operand="A"), dev)
    B = synth.near_sparse_device(n, synth.config_seed(2, operand="B"), dev)
    C = torch.empty_like(A)
    stream = torch.cuda.current_stream()
    dense = 2.0 * n ** 3

    # tau by the paper's valid-ratio search (Section 3.5.2), per candidate leaf
    taus = {}
    for leaf in ((args.leaf,) if args.leaf else (64, 128)):
        nA, nB = P.spamm_normmap(A, leaf), P.spamm_normmap(B, leaf)
        pl = P.Plan(n, leaf, P.FP32)
        taus[leaf] = pl.tau_for_valid_ratio(nA, nB, args.ratio, 0.01, 30)
        del pl, nA, nB
    # autotuner on this instance: leaf x schedule (each leaf with its own tau); --leaf fixes
    # the leaf and --schedule the schedule
    cands = []
    if args.leaf:
        best = {"leaf": args.leaf, "schedule": args.schedule, "ms": -1.0}
    else:
        for leaf in (64, 128):
            best, allc = P.spamm_batch_autotune([A], [B], [C], [taus[leaf][0]], prec, args.target,
                                                reps=2)
            cands += [c for c in allc if c["leaf"] == leaf]
        best = min((c for c in cands if c["ms"] >= 0), key=lambda c: c["ms"])
    leaf = best["leaf"]
    tau, ratio, probes = taus[leaf]
    batch = P.Batch([n], leaf, prec, graph=True, dynamic=best["schedule"] == "dynamic",
                    groups=best["schedule"] == "groups")
    tb = P.Batch([n], leaf, prec, graph=False, dynamic=best["schedule"] == "dynamic",
                    groups=best["schedule"] == "groups", timing=True)

    def step():
        batch.run([A], [B], [C], [tau], args.target)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    st = batch.stats()[0]
    assert P.spamm_last_device_status() == 0
    ph = {"normmap": [], "plan": [], "round": [], "multiply": []}
    for _ in range(3):
        tb.run([A], [B], [C], [tau], args.target)
        for k, v in tb.timings().items():
            ph[k].append(v)
    tb.close()
    part_ms = {k: statistics.median(v) for k, v in ph.items()}

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        time.sleep(0.3)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        time.sleep(0.3)
    ms = slowest_rank_ms(e0.elapsed_time(e1) / args.steps, world, dev)

    # accuracy on sampled output tiles against FP64 products on the GPU
    g = np.random.default_rng(5)
    bd = P.num_blocks(n, leaf)
    errs, refs = 0.0, 0.0
    for _ in range(16):
        i, j = int(g.integers(0, bd)), int(g.integers(0, bd))
        r = slice(i * leaf, min(n, (i + 1) * leaf))
        c = slice(j * leaf, min(n, (j + 1) * leaf))
        ref = torch.matmul(A[r].double(), B[:, c].double())
        errs += float(((C[r, c].double() - ref) ** 2).sum())
        refs += float((ref ** 2).sum())
    rel_tiles = (errs / refs) ** 0.5

    base = {}
    if not args.no_baselines:
        def timed(fn, reps):
            fn()
            g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            g0.record(stream)
            for _ in range(reps):
                fn()
            g1.record(stream)
            torch.cuda.synchronize()
            return g0.elapsed_time(g1) / reps
        prev = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = False
        base["cublas_sgemm_ms"] = timed(lambda: torch.matmul(A, B, out=C), 1)
        torch.backends.cuda.matmul.allow_tf32 = prev
        Ab, Bb = A.to(torch.bfloat16), B.to(torch.bfloat16)
        Cb = torch.empty_like(Ab)
        base["cublas_bf16_gemm_ms"] = timed(lambda: torch.matmul(Ab, Bb, out=Cb), 3)
        del Ab, Bb, Cb
        f32 = P.Batch([n], leaf, P.FP32, graph=True)
        base["fp32_spamm_ms"] = timed(lambda: f32.run([A], [B], [C], [tau]), 1)
        f32.close()
        for k in ("cublas_sgemm_ms", "cublas_bf16_gemm_ms", "fp32_spamm_ms"):
            base["speedup_vs_" + k[:-3]] = base[k] / ms
    if rank != 0:
        return None
    peaks = load_peaks()
    useful = 2.0 * leaf ** 3 * st["survivors"]
    mul_ms = part_ms["multiply"]
    ach = useful / (mul_ms * 1e-3) / 1e12
    peak = peaks["bf16_tflops"]
    line = {
        "metric": METRIC,
        "value": dense / (ms * 1e-3) / 1e12 * world,
        "unit": "TFLOP/s (dense-equivalent, 2N^3/t)", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"bf16": "bf16", "fp16": "f16", "tf32x3": "tf32",
                                       "fp32": "f32"}.get(prec_name, prec_name),
        "data": "synthetic (seeded near-sparse ReLU(N(0,1)) with 70% of the rest zeroed, drawn on the GPU)",
        "config": {"workload": f"near-sparse N={n}, leaf {leaf}, {prec_name}, tau for valid ratio "
                               f"{args.ratio:g} (valid-ratio search)",
                   "n": n, "leaf": leaf, "tau": tau, "valid_ratio": st["valid_ratio"],
                   "search_probes": probes, "survivors": st["survivors"],
                   "schedule": best["schedule"], "autotune": cands,
                   "rel_err_sampled_tiles_vs_fp64": rel_tiles,
                   "useful_tflops": useful / (ms * 1e-3) / 1e12,
                   "l2": f"inputs larger than L2 ({4 * n * n / 1e9:.1f} GB each)",
                   "parallelism": f"replicas x{world}", "launch": "cuda-graph replay"},
        "breakdown_ms": part_ms,
        "baselines_same_gpu": base,
        # one norm-map launch (both operands alike), 4 plan kernels, zero-fill,
        # rounding, multiply
        "gpu_launches": 8 * args.steps,
        "roofline": {"kernel": "multiply phase (tcgen05 multiply; rounding excluded)",
                     "bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                     "frac": ach / peak, "traffic": None, "per_launch_ms": mul_ms,
                     "algorithmic_flops": useful,
                     "peak_source": peaks["source"] + " bf16 dense (burst)"},
        "clocks": clk.summary(),
    }
    batch.close()
    return line


# ---------------------------------------------------------------------------
# Table-2 analogue: the paper's Table 1 matrix, speedup over cuBLAS
# ---------------------------------------------------------------------------

# Section 4.2, Table 2: speedup of SpAMM over cuBLAS on one V100 (FP32 vs
# cublasSgemm / FP16 vs cublasHgemm), Table 1 matrix, rows = target valid ratio.
TABLE2_V100 = {
    "0.30": {1024: (5.7, 4.3), 2048: (3.1, 5.2), 4096: (1.0, 2.3), 8192: (0.9, 1.1)},
    "0.20": {1024: (7.6, 5.2), 2048: (4.3, 6.9), 4096: (1.5, 3.7), 8192: (1.4, 2.0)},
    "0.10": {1024: (10.8, 6.5), 2048: (7.6, 11.4), 4096: (2.6, 6.8), 8192: (2.6, 3.5)},
    "0.05": {1024: (13.4, 7.6), 2048: (11.7, 16.1), 4096: (5.0, 11.9), 8192: (5.2, 7.0)},
}


def run_table2(args, rank, world):
    """One pass of the hot path (norm map, plan, multiply) on the Table 1 matrix
    a_ij = 0.1 / (|i - j|^0.1 + 1) (A = B), tau from the valid-ratio search at each target
    ratio, timed against cuBLAS: FP32 SpAMM (SIMT, leaf 32 or 64) vs SGEMM, FP16 SpAMM
    (tensor cores, leaf 64 or 128) vs cuBLAS FP16 GEMM; the faster leaf is reported."""
    import torch
    import paper_2103_13042_gb300 as P

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    sizes = [int(x) for x in args.table2_sizes.split(",")]

    def timed(fn, reps):
        for _ in range(max(2, args.warmup)):
            fn()
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for _ in range(reps):
            fn()
        g1.record(stream)
        torch.cuda.synchronize()
        return g0.elapsed_time(g1) / reps

    cells = {}
    prev_tf32 = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False   # SGEMM in FP32
    with ClockSampler(local) as clk:
        for n in sizes:
            A = torch.from_numpy(synth.table1_matrix(n)).to(dev)
            C = torch.empty_like(A)
            Ah = A.half()
            sgemm = timed(lambda: torch.matmul(A, A, out=C), args.steps)
            hgemm = timed(lambda: torch.matmul(Ah, Ah), args.steps)
            for ratio in TABLE2_V100:
                row = {}
                # each precision at its leaf candidates (tau re-searched per leaf, as the
                # valid ratio is a per-leaf quantity); the faster one is reported
                for name, prec, leaves, gemm in (("fp32", P.FP32, (32, 64), sgemm),
                                                 ("fp16", P.FP16, (64, 128), hgemm)):
                    best = None
                    for leaf in leaves:
                        nA = P.spamm_normmap(A, leaf)
                        plan = P.Plan(n, leaf, prec)
                        tau, got, _ = plan.tau_for_valid_ratio(nA, nA, float(ratio), 0.01, 30)

                        def step():
                            P.spamm_normmap(A, leaf, nA, stream)
                            plan.plan_multiply(nA, nA, tau, A, A, C, args.target, stream)

                        ms = timed(step, args.steps)
                        if best is None or ms < best["spamm_ms"]:
                            best = {"leaf": leaf, "tau": tau, "valid_ratio": got, "spamm_ms": ms}
                        del plan, nA
                    best.update({"cublas_ms": gemm, "speedup": gemm / best["spamm_ms"],
                                 "paper_v100_speedup": TABLE2_V100[ratio][n][0 if name == "fp32" else 1]
                                 if n in TABLE2_V100[ratio] else None})
                    row[name] = best
                cells[f"{n}/{ratio}"] = row
            del A, C, Ah
            torch.cuda.empty_cache()
    torch.backends.cuda.matmul.allow_tf32 = prev_tf32
    assert P.spamm_last_device_status() == 0
    if rank != 0:
        return None
    head = cells[f"{sizes[-1]}/0.05"]["fp16"]
    paper = head["paper_v100_speedup"]
    return {
        "metric": "Table 2 analogue: speedup of SpAMM over cuBLAS (FP32 vs SGEMM, FP16 vs HGEMM)",
        "value": head["speedup"], "unit": f"x vs cuBLAS HGEMM (N={sizes[-1]}, valid ratio 5%, FP16)",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": head["spamm_ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": head["speedup"] / paper if paper else None, "dtype": "fp16",
        "data": "synthetic (the Table 1 matrix, computed)",
        "config": {"workload": "Table 1 matrix a_ij = 0.1/(|i-j|^0.1+1), A = B, tau by valid-ratio "
                               "search; one step = norm map (A = B) + plan + multiply",
                   "cells": cells, "parallelism": f"replicas x{world}"},
        "clocks": clk.summary(),
    }


# ---------------------------------------------------------------------------
# Reference arm: the oracle as it stands, on the host cores
# ---------------------------------------------------------------------------

def run_reference(args):
    """The oracle as it stands on the host cores, on the same workload, metric and unit as
    the GPU arm: every step times a bounded sample of the job (a different spread of output
    block rows each step, one row per worker process) and extrapolates it to the whole job."""
    wl = WORKLOADS[args.workload]
    n = args.n or wl["n"]
    tau = wl["tau"] if args.tau is None else args.tau
    prec_name = args.precision or wl["precision"]
    leaf = args.leaf or max(wl["leaves"])
    a_h, b_h = workload(args.workload, n, args.alpha)
    pool = OraclePool(a_h, b_h)
    bd = -(-n // leaf)
    rows_per_step = max(pool.cores, args.ref_rows)
    nB = None
    walls, vals = [], []
    cb = None
    try:
        for k in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            cb, nB_k = cpu_baseline(a_h, b_h, leaf, tau, pool, single_rows=1,
                                    offset=k * rows_per_step)
            if k >= args.warmup:
                walls.append(time.perf_counter() - t0)
                vals.append(cb["value"])
    finally:
        pool.close()
    value = statistics.median(vals)
    return {
        "impl": "reference", "metric": METRIC, "value": value,
        "unit": "TFLOP/s (dense-equivalent, 2N^3/t)", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": statistics.median(walls) * 1e3,
        "ms_per_step_full_job_extrapolated": cb["seconds_full_extrapolated"] * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded numpy PCG64 draws on the host)",
        "config": {"workload": f"{workload_desc(args.workload, n, args.alpha)}, A and B "
                               f"independent, leaf {leaf}, tau={tau:g}, {prec_name} (the GPU "
                               f"arm's configuration; the oracle computes in FP64)",
                   "name": args.workload, "n": n, "leaf": leaf, "tau": tau,
                   "precision": prec_name},
        "cpu_baseline": {"value": value, "unit": cb["unit"], "cores": cb["cores"],
                         "nproc": cb["nproc"], "kind": "oracle",
                         "sample": cb["sample"] + "; each step a different spread of rows",
                         "single_thread": cb.get("single_thread")},
        "e2e": {"value": value, "unit": "TFLOP/s (dense-equivalent, 2N^3/t)",
                "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_rowblocks(args, rank, world):
    """Algorithm 4's partition of one product: each rank computes its own output block rows
    (its rows of A as a row-major view, all of B and B's norm map on every rank), so the ranks
    exchange nothing; the job's time is the slowest rank's and the value the whole product's
    dense-equivalent rate (strong scaling: the product is fixed, the ranks share it)."""
    import torch
    import paper_2103_13042_gb300 as P
    from paper_2103_13042_gb300 import partition as PT

    local = int(os.environ.get("LOCAL_RANK", "0"))
    wl = WORKLOADS[args.workload]
    n = args.n or wl["n"]
    tau = wl["tau"] if args.tau is None else args.tau
    prec_name = args.precision or wl["precision"]
    prec = P.PRECISIONS[prec_name]
    leaf = args.leaf or max(wl["leaves"])
    a_h, b_h = workload(args.workload, n, args.alpha)
    r0, r1 = PT.row_blocks(n, leaf, world)[rank]
    m = r1 - r0
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    B = torch.from_numpy(b_h).to(dev)
    bd = P.num_blocks(n, leaf)
    nB = torch.empty((bd, bd), dtype=torch.float64, device=dev)
    step = None
    if m > 0:
        A = torch.from_numpy(np.ascontiguousarray(a_h[r0:r1])).to(dev)
        C = torch.empty((m, n), dtype=torch.float32, device=dev)
        nA = torch.empty((P.num_blocks(m, leaf), bd), dtype=torch.float64, device=dev)
        plan = P.GeneralPlan(m, n, n, leaf, prec)

        def step():
            P.spamm_normmap_rect(A, leaf, nA, stream)
            P.spamm_normmap(B, leaf, nB, stream)
            plan.plan_multiply(nA, nB, tau, A, B, C, args.target, stream=stream)

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step()
        graph.replay()
        torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            if step is not None:
                graph.replay()
        e1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = slowest_rank_ms(e0.elapsed_time(e1) / args.steps, world, dev)
    # end to end: this rank's rows of A and all of B in from pinned host memory, its rows of C
    # out, every step
    e2e_ms = 0.0
    h2d = d2h = 0
    if m > 0:
        a_pin = torch.from_numpy(np.ascontiguousarray(a_h[r0:r1])).pin_memory()
        b_pin = torch.from_numpy(b_h).pin_memory()
        c_pin = torch.empty((m, n), dtype=torch.float32).pin_memory()
        h2d, d2h = 4 * (m * n + n * n), 4 * m * n
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        f0.record(stream)
        for _ in range(max(2, args.steps // 4)):
            A.copy_(a_pin, non_blocking=True)
            B.copy_(b_pin, non_blocking=True)
            step()
            c_pin.copy_(C, non_blocking=True)
        f1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = f0.elapsed_time(f1) / max(2, args.steps // 4)
    e2e_ms = slowest_rank_ms(e2e_ms, world, dev)
    if rank != 0:
        return None
    dense = 2.0 * n ** 3
    return {
        "metric": METRIC, "value": dense / (ms * 1e-3) / 1e12,
        "unit": "TFLOP/s (dense-equivalent, 2N^3/t)", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None,
        "dtype": {"fp32": "f32", "tf32x3": "tf32", "bf16_split": "bf16", "bf16": "bf16",
                  "fp16_split": "f16", "fp16": "f16"}.get(prec_name, prec_name),
        "data": "synthetic (seeded numpy PCG64 draws on the host, copied to the GPU)",
        "config": {"workload": f"{workload_desc(args.workload, n, args.alpha)}, leaf {leaf}, "
                               f"tau={tau:g}, {prec_name}, output block rows split over "
                               f"{world} ranks (Algorithm 4)",
                   "name": args.workload, "n": n, "leaf": leaf, "tau": tau,
                   "parallelism": f"row blocks x{world}", "rank0_rows": [r0, r1],
                   "launch": "cuda-graph replay of the API calls",
                   "l2": "inputs larger than L2"},
        "e2e": {"value": dense / (e2e_ms * 1e-3) / 1e12 if e2e_ms > 0 else None,
                "unit": "TFLOP/s (dense-equivalent, 2N^3/t)", "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": 9 * args.steps if prec != P.FP32 else 8 * args.steps,
        "clocks": clk.summary(),
    }


def run_extras(args, rank, world):
    """Short summaries of two more configurations, timed in the same run after the main line:
    the near-sparse N = 32768 product at a 50% valid ratio (where the multiply is
    tensor-bound) and the N = 8192 algebraic-decay mixed-precision product.  Each is the
    full workload of its own --workload run, with fewer steps and no CPU baseline."""
    import copy
    import torch
    out = {}
    for name, overrides in (("near_sparse_n32768_ratio0.5", {"workload": "sparse"}),
                            ("c2_alg_decay_n8192", {"workload": "c2"})):
        a = copy.copy(args)
        a.n, a.tau, a.leaf, a.precision = None, None, None, None
        a.no_cpu_baseline = True
        a.steps = max(5, args.steps // 2)
        for k, v in overrides.items():
            setattr(a, k, v)
        torch.cuda.empty_cache()
        try:
            ln = (run_sparse if a.workload == "sparse" else run_ours)(a, rank, world)
        except Exception as exc:   # a summary that fails is reported, the main line stands
            out[name] = {"error": f"{type(exc).__name__}: {exc}"}
            continue
        roof = ln.get("roofline", {})
        out[name] = {"workload": ln["config"]["workload"], "ms_per_step": ln["ms_per_step"],
                     "value": ln["value"], "unit": ln["unit"], "steps": ln["steps"],
                     "breakdown_ms": ln.get("breakdown_ms"),
                     "baselines_same_gpu": ln.get("baselines_same_gpu"),
                     "roofline": {k: roof.get(k) for k in ("kernel", "bound", "achieved", "peak",
                                                           "unit", "frac")},
                     "clocks": ln.get("clocks")}
        for k in ("rel_err_sampled_tiles_vs_fp64", "survivors", "valid_ratio", "leaf", "tau",
                  "skipped_bound2_rel"):
            if k in ln["config"]:
                out[name][k] = ln["config"][k]
    torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="decay",
                    choices=["decay", "c2", "batch", "sparse", "table2"],
                    help="decay: exp(-alpha|i-j|) N(0,1) at N=32768 (default); c2: algebraic "
                         "decay N=8192 mixed precision; batch: 256 uneven instances; sparse: "
                         "near-sparse N=32768 at a target valid ratio; table2: the paper's "
                         "Table 2 analogue")
    ap.add_argument("--precision", default=None,
                    help="fp32|tf32x3|bf16|fp16|bf16_split|fp16_split (default per workload)")
    ap.add_argument("--tau", type=float, default=None, help="default per workload")
    ap.add_argument("--alpha", type=float, default=0.5, help="decay: rate alpha")
    ap.add_argument("--target", type=float, default=1e-5)
    ap.add_argument("--n", type=int, default=None, help="matrix size (default per workload)")
    ap.add_argument("--leaf", type=int, default=None, help="default: autotuned / per workload")
    ap.add_argument("--schedule", default="static", choices=["static", "dynamic", "groups"],
                    help="sparse / batch with --leaf: the multiply schedule (else autotuned)")
    ap.add_argument("--cpu-rows", type=int, default=4,
                    help="output block-rows of the oracle's single-thread sample (cpu_baseline)")
    ap.add_argument("--ref-rows", type=int, default=8,
                    help="output block-rows per step of --impl reference (at least the core count)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-baselines", action="store_true")
    ap.add_argument("--eager", action="store_true", help="time host-enqueued calls, no graph")
    ap.add_argument("--table2-sizes", default="1024,2048,4096,8192",
                    help="table2 workload: matrix sizes")
    ap.add_argument("--ratio", type=float, default=0.5, help="sparse: target valid ratio")
    ap.add_argument("--partition", default="replicas", choices=["replicas", "rows", "instances"],
                    help="N > 1: replicas (every rank the whole job), rows (decay/c2: the "
                         "product's block rows split over the ranks, Algorithm 4) or instances "
                         "(batch: the instances dealt to the ranks)")
    ap.add_argument("--no-extras", action="store_true",
                    help="decay: skip the near-sparse and N=8192 summaries added to the line")
    ap.add_argument("--count", type=int, default=BATCH_COUNT)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return
        if args.workload not in WORKLOADS:
            print(json.dumps({"impl": "reference", "unavailable":
                              "the reference arm covers the single-product workloads"}), flush=True)
            return
        print(json.dumps(run_reference(args)), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))   # before NCCL binds
        dist.init_process_group("nccl")
    runner = {"batch": run_batch, "sparse": run_sparse, "table2": run_table2}.get(args.workload, run_ours)
    if args.partition == "rows" and args.workload in WORKLOADS:
        runner = run_rowblocks
    line = runner(args, rank, world)
    if args.workload == "decay" and not args.no_extras and world == 1 and line is not None:
        line["extra_workloads"] = run_extras(args, rank, world)
    if line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
