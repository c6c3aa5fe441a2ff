#!/usr/bin/env python3
"""Benchmark: batched primal-dual iLQR MPC solves on one B300 (and N GPUs).

Workload (one step): 4096 single-rigid-body quadruped MPC problems with
horizons drawn from {25, 50, 75, 100} (n = m = 12, dt = 0.02 s, trot
contact schedule, friction-cone barrier), each solved by 10 SQP iterations
of the fused kernel (linearisation + LQ KKT solve by the parallel scan +
parallel line search + update) in one launch.  The metric counts KKT solves
(one per SQP iteration per instance) per second.

The JSON line also reports the single-instance latencies (one N = 50
problem, CUDA-graph replays: the MPC tick of the paper), the comparators
(sequential Riccati in the same fused kernel, and a plain sequential-Riccati
KKT kernel launched once per instance), the roofline of the fused kernel,
the end-to-end figure through the C ABI with host buffers, the FP64 oracle
timed on the host cores, and the SM clocks seen during the timed region.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
For N > 1 launch with torch.distributed.run (one rank per GPU); each rank
solves its own batch (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2506_07823_b300 import synth  # noqa: E402  (no GPU code)

METRIC = ("KKT solves/s and p99 solve latency at ≤1e-4 vs FP64 oracle, scan vs seq. "
          "Riccati, 1×B300")
UNIT = "KKT solves/s"
COUNT = 4096
HORIZONS = (25, 50, 75, 100)
ITERS = 10
SEED = 0
WORKLOAD = "srbd_batched_mpc"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "sqp_kernel_traffic.json")
KERNEL_SOURCES = ["dev_linalg.cuh", "kkt_scan.cuh", "srbd.cuh", "sqp.cuh", "sqp_rows.cuh"]

def flops_per_stage(n: int, solver: str) -> float:
    """Algorithmic flops of one LQ KKT solve per stage for n = m: about 50 n^3
    for the work-efficient scan (combines in both sweeps, element build,
    policy, trajectory) and about 13 n^3 for the sequential Riccati recursion
    (4 n^3 + 8 n^2 m + m^3 / 3)."""
    return (50.0 if solver == "scan" else 13.0) * n ** 3


def lq_flops_per_stage(n: int, m: int, solver: str) -> float:
    """Algorithmic flops of one LQ KKT solve per stage for general (n, m): the
    sequential recursion 4 n^3 + 8 n^2 m + m^3 / 3; the work-efficient scan
    the full combine (17 n^3), the value-function combine (8.7 n^3), the
    element build (m^3 / 3 + 4 m^2 n + 6 n^2 m), the policy (2 n^3 + 4 n^2 m +
    4 n m^2 + m^3 / 3) and the trajectory (2 n^3 + 2 n^2 m), about 50 n^3 at
    n = m."""
    if solver != "scan":
        return 4.0 * n ** 3 + 8.0 * n * n * m + m ** 3 / 3.0
    return (17.0 * n ** 3 + 8.7 * n ** 3 + (m ** 3 / 3.0 + 4.0 * m * m * n + 6.0 * n * n * m) +
            (2.0 * n ** 3 + 4.0 * n * n * m + 4.0 * n * m * m + m ** 3 / 3.0) +
            (2.0 * n ** 3 + 2.0 * n * n * m))


def roofline_rec(flops: float, ms: float, peak_tflops, ctas=None) -> dict:
    """Achieved algorithmic TFLOP/s of one timed call and its fraction of the
    measured FP32 FMA peak of the whole GPU (and, for a call that occupies
    `ctas` SMs of the 148, of those SMs' share of it)."""
    ach = flops / (ms / 1e3) / 1e12
    rec = {"algorithmic_flops": flops, "achieved_tflops": ach}
    if peak_tflops:
        rec["frac_of_ffma_peak"] = ach / peak_tflops
        if ctas:
            rec["frac_of_ffma_peak_of_its_sms"] = ach / (peak_tflops * ctas / 148.0)
    return rec


def _gj_flops(rows: int, cols: int) -> float:
    """Gauss-Jordan elimination of a rows x (rows + cols) augmented matrix as
    the kernels run it: every step updates the rows - 1 other rows over the
    columns right of the pivot (2 flop each), then the right-hand sides are
    divided by the pivots."""
    return sum(2.0 * (rows - 1) * (rows + cols - k - 1) for k in range(rows)) + rows * cols


def executed_flops(n: int, m: int, N: int, chunks: int) -> float:
    """Flops the LQ KKT solve of one instance executes in the fused kernel,
    counted from the operation sizes of the code: a Riccati step per stage
    (P'B, P'A, P'c, G, H, h, A^T P'A, A^T w, the SPD elimination of
    G^-1 [H | h], K^T H, K^T h, Abar, bbar), and for a scan with W > 2 chunks
    per stage of the middle chunks an element build (R^-1 [B^T | r], B X, b)
    and a full combine (C1 P2, P2 A1, the inversion of M = I + C1 P2, M^-1 A1,
    M^-1 C1, the five output blocks), per stage of every chunk but the last
    the chunk-map update (Psi Abar, Psi bbar), and per stage the rollout.
    The chunk partition is the kernels' (every chunk one stage, the rest in
    proportion 10 : 16 for the first/middle and the last chunk)."""
    ric = (2 * n * n * m + 2 * n ** 3 + 2 * n * n + 2 * m * m * n + 2 * m * n * n + 2 * m * n
           + 2 * n ** 3 + 2 * n * n + _gj_flops(m, n + 1) + 2 * n * n * m + 2 * n * m
           + 2 * n * n * m + 2 * n * m)
    build = _gj_flops(m, n + 1) + 2 * n * n * m + 2 * n * m
    comb = 16 * n ** 3 + 6 * n * n + _gj_flops(n, n)
    cmap = 2 * n ** 3 + 2 * n * n
    roll = 4 * n * n + 2 * n * m
    S = N + 1
    W = min(chunks, S)
    per = S * (ric + roll)
    if W > 1:
        units = (W - 1) * 10 + 16
        start = [w + ((S - W) * (w * 10)) // units for w in range(W)] + [S]
        for w in range(W - 1):
            size = start[w + 1] - start[w]
            per += size * cmap
            if w > 0:
                per += size * (build + comb)
    return per


def kernel_name(W: int, ipc: int = 2) -> str:
    """The fused SQP kernel that runs the batch with W horizon chunks (and,
    for the sequential solver, ipc instances per CTA: ipc / 2 warps)."""
    return f"sqp_rows_kernel<12,{max(ipc, 2) // 2}>" if W == 1 else f"sqp_scan_rows_kernel<12,{W}>"


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2506_07823_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# --------------------------------------------------------------- CPU oracle
def _oracle_worker(args):
    import oracle  # test infrastructure: only the CPU-baseline leg runs it
    prm, items, keep = args
    its, kept = 0, []
    for idx, pr in items:
        x, u, lam, info = oracle.srbd_sqp(prm, pr["x0hat"], pr["x"], pr["u"], pr["lam"],
                                          pr["xref"], pr["uref"], pr["contact"], max_iters=ITERS)
        its += info["iters"]
        if keep:
            al = np.zeros(ITERS)
            al[:min(ITERS, len(info["alpha"]))] = np.asarray(info["alpha"][:ITERS])
            kept.append((idx, x, u, lam, int(info["status"]), al))
    return its, kept


def oracle_pool(cores: int):
    return mp.get_context("spawn").Pool(cores)


def oracle_run(pool, cores: int, insts: list, keep: bool = False):
    """Solve ``insts`` with the FP64 oracle on ``cores`` processes; returns
    (KKT solves, wall seconds, per-instance results if ``keep``).  The oracle
    gets the FP32-rounded problem data, as the GPU does."""
    prm = synth.srbd_params()
    items = [(i, {**{k: np.asarray(pr[k], np.float32).astype(np.float64)
                     for k in ("x0hat", "x", "u", "lam", "xref", "uref")},
                  "contact": pr["contact"]}) for i, pr in enumerate(insts)]
    chunks = [items[i::cores] for i in range(cores)]
    t0 = time.perf_counter()
    res = pool.map(_oracle_worker, [(prm, c, keep) for c in chunks if c])
    secs = time.perf_counter() - t0
    its = sum(r[0] for r in res)
    kept = sorted((k for r in res for k in r[1]), key=lambda t: t[0])
    return its, secs, kept


# oracle status codes (0 ok, 1 no step accepted, 2 not SPD) as the C ABI's
ORACLE_STATUS = {0: 0, 1: 8, 2: 2}


def compare_with_oracle(kept, Nv, off, x, u, lam, status, alpha) -> dict:
    """Final iterates of the timed batch against the oracle's free-running
    solves of the same instances: status agreement, and per block
    |z_gpu - z_ref|_inf / |z_ref|_inf over the instances both end with status
    OK (all of them, and those whose step sizes agree at every iteration, where
    the two runs take the same path and must agree to 1e-4)."""
    agree = {}
    err_all = {"x": [], "u": [], "lam": []}
    err_same = {"x": [], "u": [], "lam": []}
    for idx, xr, ur, lr, st_o, al_o in kept:
        st_g = int(status[idx])
        st_o = ORACLE_STATUS.get(st_o, st_o)
        key = f"gpu{st_g}_oracle{st_o}"
        agree[key] = agree.get(key, 0) + 1
        if st_g != 0 or st_o != 0:
            continue
        N, o = int(Nv[idx]), int(off[idx])
        e = {"x": np.abs(x[o:o + N + 1] - xr).max() / max(np.abs(xr).max(), 1e-30),
             "u": np.abs(u[o:o + N] - ur[:N]).max() / max(np.abs(ur[:N]).max(), 1e-30),
             "lam": np.abs(lam[o:o + N + 1] - lr).max() / max(np.abs(lr).max(), 1e-30)}
        same = np.array_equal(alpha[idx].astype(np.float64), al_o)
        for k in e:
            err_all[k].append(e[k])
            if same:
                err_same[k].append(e[k])
    out = {"instances_compared": len(kept), "status_agreement": dict(sorted(agree.items())),
           "ok_pairs": len(err_all["x"]), "ok_pairs_same_steps": len(err_same["x"])}
    for name, errs in (("all_ok_pairs", err_all), ("same_steps", err_same)):
        if errs["x"]:
            out[name] = {
                "max_rel_err": {k: float(np.max(v)) for k, v in errs.items()},
                "p99_rel_err": {k: float(np.percentile(v, 99)) for k, v in errs.items()},
                "within_1e-4": int(sum(max(errs[k][i] for k in errs) <= 1e-4
                                       for i in range(len(errs["x"]))))}
    return out


def host_cores() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except Exception:
        return max(1, os.cpu_count() or 1)


def sample_size(cores: int) -> int:
    # about 10-30 s of oracle work (roughly 1.2k KKT solves/s per core)
    return int(min(COUNT, max(64, cores * 300)))


# ------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock samples (every 50 ms) during the timed region.

    ``start`` returns once nvidia-smi has printed its first sample (at most
    5 s), so that its start-up does not eat into the region; the summary keeps
    the samples taken inside the region, or, when the region was shorter than
    the interval, the last one before it (``samples_in_region`` says which)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self._t = None
        self._skip = 0

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
            t0 = time.perf_counter()
            while not self.lines and self.proc.poll() is None and time.perf_counter() - t0 < 5.0:
                time.sleep(0.01)
            self._skip = len(self.lines)
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self._t:
            self._t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        inside = self.lines[self._skip:]
        for ln in inside or self.lines[-1:]:
            parts = [p.strip() for p in ln.split(",")]
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
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "samples_in_region": len(inside), "reasons": sorted(reasons)}


# ------------------------------------------------------------- multi-rank
def rank_seed(rank: int, count: int) -> int:
    """Replicas: rank r solves its own batch of ``count`` instances drawn from
    the Philox streams seed + r * count .. seed + (r + 1) * count - 1."""
    return SEED + rank * count


def aggregate(ms_local: float, kkt_local: float, device) -> tuple[float, float]:
    """Whole-job step time (max over ranks) and KKT solves (sum over ranks).
    Works with any torch.distributed backend (gloo on CPU tensors, nccl on
    CUDA tensors); a single process returns its own numbers."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms_local, kkt_local
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    k = torch.tensor([kkt_local], dtype=torch.float64, device=device)
    dist.all_reduce(k, op=dist.ReduceOp.SUM)
    return float(t.item()), float(k.item())


# ---------------------------------------------------------------- GPU arm
def build_device_batch(torch, insts, packed, Nv, off, x0, dev):
    t = {}
    for k in ("x", "u", "lam", "xref", "uref"):
        t[k] = torch.tensor(np.asarray(packed[k], dtype=np.float32), device=dev)
    t["contact"] = torch.tensor(np.asarray(packed["contact"], dtype=np.uint8), device=dev)
    t["x0hat"] = torch.tensor(np.asarray(x0, dtype=np.float32), device=dev)
    return t


def event_times(torch, fn, reps, stream, before=None):
    """Per-call device times (ms) with CUDA events on ``stream``."""
    out = []
    for _ in range(reps):
        if before:
            before()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        out.append(e0.elapsed_time(e1))
    return out


def pct(v, q):
    return float(np.percentile(np.asarray(v), q))


def run_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_2506_07823_b300 import pdilqr

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    # CPU baseline pool: spawned before the first GPU kernel
    cores = host_cores()
    pool = oracle_pool(cores) if (rank == 0 and not args.no_cpu) else None

    insts, packed, Nv, off, x0 = synth.srbd_batch(args.count, seed=rank_seed(rank, args.count),
                                                  Ns_choices=HORIZONS)
    total_stages = int(Nv.sum() + len(Nv))
    prm = synth.srbd_params()
    md = pdilqr.srbd_model(prm)
    base = build_device_batch(torch, insts, packed, Nv, off, x0, dev)
    work = {k: v.clone() for k, v in base.items()}

    def reset():
        for k in ("x", "u", "lam"):
            work[k].copy_(base[k], non_blocking=True)

    flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def flush():
        flush_buf.zero_()

    # measured FP32 FMA peak of this GPU (the roofline's denominator)
    peak_ffma, _ = pdilqr.peak_probe(pdilqr.PEAK_FFMA, 3)

    # --- autotune the solver on this batch (paper_2506_07823_b300.autotune):
    # the sequential recursion (one chunk per instance) at 2, 4 or 8 instances
    # per CTA and the scan with 4, 8 or 16 chunks; two timed solves each
    from paper_2506_07823_b300 import autotune

    def solve_on(p):
        return p.solve(md, work["x0hat"], work["x"], work["u"], work["lam"], work["xref"],
                       work["uref"], work["contact"], max_iters=ITERS)
    cands = None
    if args.warps:
        cands = [(1, args.inst_per_cta or 2)] if args.warps == 1 else [(args.warps, 0)]
    plan, tune = autotune.autotune_sqp(torch, 12, 12, Nv, off, solve_on, reset=reset, flush=flush,
                                       reps=2, stream=stream, cands=cands)
    W, IPC = plan.warps, plan.inst_per_cta
    # one plan per chunk count for the comparators (the tuned one included)
    plans = {W: plan}
    for w in (1, 4, 8, 16):
        if w not in plans and (not args.warps or w == args.warps):
            try:
                plans[w] = pdilqr.Plan(12, 12, Nv, off, warps=w)
            except pdilqr.PdilqrError:
                pass
    solver = "sequential" if W == 1 else "scan"
    info = {"iters": torch.zeros(plan.count, device=dev, dtype=torch.int32),
            "status": torch.zeros(plan.count, device=dev, dtype=torch.int32),
            "alpha": torch.zeros(plan.count, ITERS, device=dev, dtype=torch.float32),
            "J": None, "theta": None}

    def solve_direct():
        plan.solve(md, work["x0hat"], work["x"], work["u"], work["lam"], work["xref"],
                   work["uref"], work["contact"], max_iters=ITERS, info=info)

    # the timed step replays the plan's captured CUDA graph of the batched
    # solve (pdilqr_solve_capture: the counter reset and one launch of the
    # fused kernel); the trajectory reset and the L2 flush stay outside it
    reset()
    solve_direct()
    torch.cuda.synchronize()
    plan.capture(md, work["x0hat"], work["x"], work["u"], work["lam"], work["xref"],
                 work["uref"], work["contact"], max_iters=ITERS, info=info)
    solve = plan.replay

    for _ in range(args.warmup):
        reset()
        solve()
    torch.cuda.synchronize()

    # --- timed region: K solves; reset and L2 flush between them, outside the events
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    times = event_times(torch, solve, args.steps, stream, before=lambda: (reset(), flush()))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    kkt_per_step = int(info["iters"].sum().item())
    st = info["status"].cpu().numpy()
    final = {k: work[k].double().cpu().numpy() for k in ("x", "u", "lam")}
    alpha_gpu = info["alpha"].cpu().numpy()
    ms, kkt_all = aggregate(float(np.mean(times)), float(kkt_per_step), dev)
    value = kkt_all / (ms / 1e3)

    result = None
    if rank == 0:
        n = 12
        its_inst = info["iters"].cpu().numpy()
        algo = flops_per_stage(n, solver) * float(np.sum((Nv + 1) * its_inst))
        executed = sum(executed_flops(n, n, int(Nv[i]), W) * int(its_inst[i]) for i in range(len(Nv)))
        achieved = algo / (ms / 1e3) / 1e12
        traffic = None
        try:
            tr = json.load(open(TRAFFIC_FILE)).get(kernel_name(W, IPC), {})
            if tr.get("source_hash") == kernel_source_hash():
                traffic = tr["bytes_per_launch_full"]
        except Exception:
            traffic = None
        extras = measure_extras(torch, pdilqr, md, prm, dev, stream, base, work, plan, plans, args)
        lqw = (measure_lq_workloads(torch, pdilqr, dev, stream, args, peak_ffma)
               if args.lq_workloads else None)
        serving = None
        if args.serve_seconds > 0:
            low = args.serve_rate_sustained
            serving = {
                "workload": "Poisson arrivals, one real-time SQP iteration per request, N = 50, "
                            "256 clients: one robot (n = 12) or two robots (n = 24)",
                "continuous_batching_scan": measure_serving(pdilqr, args, args.serve_seconds,
                                                            args.serve_rate, 1024, 8, 2),
                "one_request_per_launch_riccati": measure_serving(pdilqr, args, args.serve_seconds,
                                                                  args.serve_rate, 1, 1, 1),
                "equal_load_note": f"both servers at {low:g} requests/s, a rate the one-request-"
                                   "per-launch server sustains, so that its p99 is solve latency "
                                   "and not queue growth",
                "continuous_batching_scan_equal_load": measure_serving(
                    pdilqr, args, args.serve_seconds, low, 1024, 8, 2),
                "one_request_per_launch_riccati_equal_load": measure_serving(
                    pdilqr, args, args.serve_seconds, low, 1, 1, 1),
                "full_mix_workload": "Poisson arrivals, one real-time SQP iteration per request, "
                                     "N = 50, 1024 clients: 60 % one robot, 10 % each 2, 4, 8 "
                                     "and 16 robots (n = 12 R)",
                "continuous_batching_full_mix": measure_serving(pdilqr, args, args.mix_seconds,
                                                                args.serve_rate, 1024, 8,
                                                                args.mix_streams, mix="full",
                                                                large_cta_budget=args.mix_large_ctas)}
            if args.mix_split_seconds > 0:
                serving["full_mix_split_note"] = (
                    f"the same mix with the classes of {args.mix_split_robots}+ robots on the "
                    f"split scan (16 CTAs per instance, one split batch in flight, at most "
                    f"{args.mix_split_batch} instances per split batch)")
                serving["continuous_batching_full_mix_split"] = measure_serving(
                    pdilqr, args, args.mix_split_seconds, args.serve_rate, 1024, 8,
                    args.mix_streams, mix="full", large_cta_budget=args.mix_large_ctas,
                    split_min_robots=args.mix_split_robots, split_max_batch=args.mix_split_batch)
        e2e = measure_e2e(torch, pdilqr, md, dev, stream, base, plan, args)
        sweep = measure_sweep(torch, pdilqr, dev, stream, args.sweep_reps) if args.sweep_reps > 0 else None
        cpu = None
        vs_oracle = None
        if pool is not None:
            sample = insts[:sample_size(cores)]
            its, secs, kept = oracle_run(pool, cores, sample, keep=True)
            cpu = {"value": its / secs, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": f"{len(sample)} of the {args.count} instances, one 10-iteration "
                             f"SQP solve each, FP64 C oracle, {cores} processes, {secs:.1f} s"}
            vs_oracle = compare_with_oracle(kept, Nv, off, final["x"], final["u"], final["lam"],
                                            st, alpha_gpu)
            vs_oracle["replay"] = replay_check(torch, plan, md, work, base, kept, Nv, off)
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (FP64 line-search sums)", "data": "synthetic",
            "config": {"workload": WORKLOAD, "instances_per_gpu": args.count,
                       "horizons": list(HORIZONS), "n": 12, "m": 12, "sqp_iters": ITERS,
                       "stages_per_gpu": total_stages, "warps_per_instance": W,
                       "instances_per_cta": (IPC or 2) if W == 1 else 1,
                       "solver": ("sequential Riccati recursion (one chunk per instance)"
                                  if W == 1 else f"parallel scan ({W} horizon chunks)"),
                       "autotune_ms": {str(k): round(v, 3) for k, v in tune.items()},
                       "autotune": "paper_2506_07823_b300.autotune: seq/I = sequential recursion at "
                                   "I instances per CTA, scan/W = parallel scan over W chunks",
                       "l2": "flushed between timed steps (256 MiB write)",
                       "cuda_graph": "the timed step replays the plan's captured graph of the "
                                     "batched solve (pdilqr_solve_capture / pdilqr_plan_replay)",
                       "parallelism": f"replicas{world}"},
            "latency_ms": {"batch_p50": pct(times, 50), "batch_p99": pct(times, 99),
                           **extras["latency"]},
            "comparators": extras["comparators"],
            "serving": serving,
            "lq_workloads": lqw,
            "sweep": sweep,
            "status_counts": {str(int(s)): int((st == s).sum()) for s in np.unique(st)},
            "vs_oracle": vs_oracle,
            "kkt_solves_per_step": kkt_all,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_ffma,
                         "unit": "TFLOP/s", "frac": achieved / peak_ffma,
                         "traffic": traffic,
                         "kernel": kernel_name(W, IPC),
                         "algorithmic_flops_per_step": algo,
                         "algorithmic_flops_per_stage": flops_per_stage(n, solver),
                         "executed_kkt_flops_per_step": executed,
                         "executed_frac": executed / (ms / 1e3) / 1e12 / peak_ffma,
                         "peak_source": "measured in this run: FFMA probe (pdilqr_peak_probe), "
                                        "best of 3 launches of about 50 ms"},
            "e2e": e2e,
            "cpu_baseline": cpu,
            "clocks": clk,
            "gpu_launches": args.steps,
            "wall_s_timed_region": wall,
        }
    if pool is not None:
        pool.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return result


def replay_check(torch, plan, md, work, base, kept, Nv, off) -> dict:
    """The benchmarked solver once more on the same batch (untimed), each
    instance taking the oracle's step sizes (the replay mode of the parity
    tests), so that every instance follows the oracle's path: per block
    relative error of the final iterate over the instances the oracle solves
    with status OK, and how many are within 1e-4."""
    count = plan.count
    alpha = np.ones((count, ITERS), np.float32)
    for idx, _, _, _, _, al_o in kept:
        alpha[idx] = al_o
    dev = work["x"].device
    inf = {"iters": torch.zeros(count, device=dev, dtype=torch.int32),
           "status": torch.zeros(count, device=dev, dtype=torch.int32),
           "alpha": None, "J": None, "theta": None}
    for k in ("x", "u", "lam"):
        work[k].copy_(base[k])
    plan.solve(md, work["x0hat"], work["x"], work["u"], work["lam"], work["xref"], work["uref"],
               work["contact"], max_iters=ITERS, alpha_replay=torch.tensor(alpha, device=dev),
               info=inf)
    torch.cuda.synchronize()
    x, u, lam = (work[k].double().cpu().numpy() for k in ("x", "u", "lam"))
    st = inf["status"].cpu().numpy()
    errs, worst, status_match = [], {"x": 0.0, "u": 0.0, "lam": 0.0}, 0
    for idx, xr, ur, lr, st_o, al_o in kept:
        # an oracle run that stopped early (converged at its precision floor)
        # replays as a zero step, which the GPU reports as E_LINESEARCH with
        # the iterate left where the oracle stopped
        stopped = st_o == 0 and bool(np.any(al_o == 0.0)) and int(st[idx]) == 8
        status_match += int(int(st[idx]) == ORACLE_STATUS.get(st_o, st_o) or stopped)
        if st_o != 0 or (st[idx] != 0 and not stopped):
            continue
        N, o = int(Nv[idx]), int(off[idx])
        e = {"x": np.abs(x[o:o + N + 1] - xr).max() / max(np.abs(xr).max(), 1e-30),
             "u": np.abs(u[o:o + N] - ur[:N]).max() / max(np.abs(ur[:N]).max(), 1e-30),
             "lam": np.abs(lam[o:o + N + 1] - lr).max() / max(np.abs(lr).max(), 1e-30)}
        for k in e:
            worst[k] = max(worst[k], float(e[k]))
        errs.append(max(e.values()))
    return {"instances": len(errs), "status_match": status_match, "max_rel_err": worst,
            "within_1e-4": int(sum(v <= 1e-4 for v in errs))}


def measure_extras(torch, pdilqr, md, prm, dev, stream, base, work, plan, plans, args):
    """Single-instance latencies (MPC tick) and the comparators."""
    lat, comp = {}, {}
    # one N = 50 problem, the paper's SRBD MPC tick
    pr = synth.srbd_problem(50, seed=SEED)
    pk, Nv1, off1 = synth.pack([pr], synth.SRBD_KEYS)
    one = build_device_batch(torch, [pr], pk, Nv1, off1, pr["x0hat"][None], dev)
    w1 = {k: v.clone() for k, v in one.items()}
    reps = args.latency_reps
    for name, warps in (("scan_sqp_single", 16), ("riccati_sqp_single", 1)):
        p1 = pdilqr.Plan(12, 12, Nv1, off1, warps=warps)
        inf1 = {"iters": torch.zeros(1, device=dev, dtype=torch.int32),
                "status": torch.zeros(1, device=dev, dtype=torch.int32),
                "alpha": None, "J": None, "theta": None}

        def step(p1=p1, inf1=inf1):
            for k in ("x", "u", "lam"):
                w1[k].copy_(one[k], non_blocking=True)
            p1.solve(md, w1["x0hat"], w1["x"], w1["u"], w1["lam"], w1["xref"], w1["uref"],
                     w1["contact"], max_iters=ITERS, info=inf1)
        step()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            step()
        for _ in range(10):
            g.replay()
        t = event_times(torch, g.replay, reps, stream)
        lat[name + "_p50"] = pct(t, 50)
        lat[name + "_p99"] = pct(t, 99)
    # the same batch through every solver of the autotuner: the sequential
    # recursion (the fused SQP with one horizon chunk per instance, one warp,
    # 16 CTAs per SM) and the scan with 4, 8, 16 chunks
    def reset_work():
        for k in ("x", "u", "lam"):
            work[k].copy_(base[k], non_blocking=True)

    by_chunks = {}
    for w in sorted(plans):
        pw = plans[w]
        infw = {"iters": torch.zeros(pw.count, device=dev, dtype=torch.int32),
                "status": torch.zeros(pw.count, device=dev, dtype=torch.int32),
                "alpha": None, "J": None, "theta": None}

        def batch(pw=pw, infw=infw):
            pw.solve(md, work["x0hat"], work["x"], work["u"], work["lam"], work["xref"],
                     work["uref"], work["contact"], max_iters=ITERS, info=infw)
        reset_work()
        batch()
        torch.cuda.synchronize()
        t = event_times(torch, batch, 3, stream, before=reset_work)
        by_chunks[w] = {"kkt_solves_per_s": float(infw["iters"].sum().item()) / (np.mean(t) / 1e3),
                        "ms": float(np.mean(t))}
    if 1 in by_chunks:
        comp["riccati_sqp_batched"] = dict(
            by_chunks[1], warps_per_instance=1,
            note="same batch and fused SQP kernel, one horizon chunk per instance (the "
                 "sequential Riccati recursion)")
    scans = {w: v for w, v in by_chunks.items() if w > 1}
    if scans:
        wb = min(scans, key=lambda w: scans[w]["ms"])
        comp["scan_sqp_batched"] = dict(scans[wb], warps_per_instance=wb,
                                        note="same batch, the parallel scan at its best chunk count")
    comp["sqp_batched_by_chunks"] = {str(w): v for w, v in by_chunks.items()}
    # LQ KKT solves alone on the linearisation of the 4096-instance batch
    lq = plan.linearize(md, base)
    lq["S"] = None
    s = (base["x0hat"] - base["x"][torch.tensor(plan.stage_off, device=dev)]).contiguous()
    out = plan.alloc_out(device=dev)
    for name, fn in (("scan_kkt_batched", plan.kkt_scan_solve),
                     ("riccati_kkt_batched", plan.riccati_solve)):
        fn(lq, s, out=out)
        torch.cuda.synchronize()
        t = event_times(torch, lambda fn=fn: fn(lq, s, out=out), 5, stream)
        comp[name] = {"kkt_solves_per_s": plan.count / (np.mean(t) / 1e3), "ms": float(np.mean(t))}
    # the plain comparator: one sequential-Riccati KKT solve per launch
    sample = min(args.count, args.comparator_sample)
    plans1, lqs, ss, outs = [], [], [], []
    for i in range(sample):
        N, o = int(plan.N[i]), int(plan.stage_off[i])
        p1 = pdilqr.Plan(12, 12, [N], [0])
        plans1.append(p1)
        lqs.append({k: (v[o:o + N + 1].contiguous() if v is not None else None) for k, v in lq.items()})
        ss.append(s[i:i + 1].contiguous())
        outs.append(p1.alloc_out(device=dev))
    for i in range(sample):
        plans1[i].riccati_solve(lqs[i], ss[i], out=outs[i])
    torch.cuda.synchronize()

    def one_per_launch():
        for i in range(sample):
            plans1[i].riccati_solve(lqs[i], ss[i], out=outs[i])
    t = event_times(torch, one_per_launch, 3, stream)
    per = np.mean(t) / sample
    comp["riccati_kkt_one_instance_per_launch"] = {
        "kkt_solves_per_s": 1e3 / per, "ms_per_solve": per,
        "sample": f"{sample} instances of the batch, one launch each, back to back"}
    # single-instance KKT latency, scan (16 warps) vs sequential Riccati kernel
    i0 = 0
    N0 = int(plan.N[i0])
    o0 = int(plan.stage_off[i0])
    p16 = pdilqr.Plan(12, 12, [N0], [0], warps=16)
    lq0 = {k: (v[o0:o0 + N0 + 1].contiguous() if v is not None else None) for k, v in lq.items()}
    o16 = p16.alloc_out(device=dev)
    for name, fn in (("scan_kkt_single", p16.kkt_scan_solve), ("riccati_kkt_single", p16.riccati_solve)):
        fn(lq0, ss[0], out=o16)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn(lq0, ss[0], out=o16)
        for _ in range(10):
            g.replay()
        t = event_times(torch, g.replay, reps, stream)
        lat[name + "_p50"] = pct(t, 50)
        lat[name + "_p99"] = pct(t, 99)
    lat["single_horizon"] = {"sqp": 50, "kkt": N0}
    return {"latency": lat, "comparators": comp}


def measure_large_state_lq(torch, pdilqr, oracle, dev, stream, args, peak=None):
    """One instance's LQ KKT solve at the centralised multi-robot sizes (n = m =
    12 R for R = 4, 8, 16; N = 50; the whole-body LTV recipe at that size) by
    the sequential recursion (one CTA), the scan over 4 chunks inside one CTA,
    and the split scan (16 chunks on 16 CTAs), unrefined and with one
    refinement step: p50 / p99 over direct calls (CUDA events), and each
    result's error against the FP64 oracle."""
    rows = []
    reps = max(5, min(args.latency_reps, 20))
    for R in (4, 8, 16):
        n = 12 * R
        inst = synth.ltv_lq(n, n, 50, seed=500 + R, rho=0.98, b_std=0.2, q_kind="llt", r_w=0.01)
        pk, Nv1, off1 = synth.pack([inst], synth.LQ_KEYS)
        lq1 = {k: torch.tensor(np.asarray(v, np.float32), device=dev) for k, v in pk.items()}
        lq1["S"] = None
        s1 = torch.tensor(np.asarray(inst["s"][None], np.float32), device=dev)
        r32 = {k: np.asarray(inst[k], np.float32).astype(np.float64) for k in synth.LQ_KEYS}
        ref = oracle.riccati_solve(r32, np.asarray(inst["s"], np.float32).astype(np.float64))
        row = {"robots": R, "n": n, "N": 50}
        for name, kw in (("sequential", dict(warps=1)), ("scan_one_cta", dict(warps=4)),
                         ("scan_split", dict(warps=16, split=True)),
                         ("sequential_refined", dict(warps=1, refine=True)),
                         ("scan_split_refined", dict(warps=16, split=True, refine=True))):
            p1 = pdilqr.Plan(n, n, Nv1, off1, **kw)
            o1 = p1.alloc_out(device=dev)
            p1.kkt_scan_solve(lq1, s1, out=o1)
            torch.cuda.synchronize()
            t = event_times(torch, lambda: p1.kkt_scan_solve(lq1, s1, out=o1), reps, stream)
            err = 0.0
            for k, n_slots in (("dx", 51), ("du", 50), ("dlam", 51)):
                got = o1[k].double().cpu().numpy()[:n_slots]
                want = ref[k][:n_slots]
                err = max(err, float(np.abs(got - want).max() / np.abs(want).max()))
            row[name] = {"p50_ms": pct(t, 50), "p99_ms": pct(t, 99), "ctas": p1.warps if kw.get("split") else 1,
                         "status": int(o1["status"][0].item()), "max_rel_error_vs_oracle": err}
            if not kw.get("refine"):
                solver = "riccati" if kw["warps"] == 1 else "scan"
                row[name]["roofline"] = roofline_rec(51 * lq_flops_per_stage(n, n, solver), pct(t, 50),
                                                     peak, row[name]["ctas"])
            p1.close()
        row["split_speedup_vs_sequential"] = row["sequential"]["p50_ms"] / row["scan_split"]["p50_ms"]
        row["split_speedup_vs_sequential_refined"] = (row["sequential_refined"]["p50_ms"] /
                                                      row["scan_split_refined"]["p50_ms"])
        rows.append(row)
    return rows


def measure_lq_workloads(torch, pdilqr, dev, stream, args, peak=None):
    """LQ KKT solves alone: the whole-body-sized batch (n = 36, m = 24,
    N = 100, 1024 instances; 128 distinct instances replicated eight times)
    with the FP64-residual refinement step, scan vs sequential Riccati, the
    backward error of every result and the error against the oracle on a
    sample; and the single-LQR workload (n = 4, m = 2, N = 16) latency."""
    import oracle   # the error against the FP64 oracle is part of the report
    out = {}
    cfg = dict(synth.LQ_WB)
    uniq, rep = 128, 8
    insts, _, _, _, _ = synth.ltv_batch(uniq, seed=SEED, **cfg)
    allinst = [insts[i % uniq] for i in range(uniq * rep)]
    packed, Nv, off = synth.pack(allinst, synth.LQ_KEYS)
    s = np.stack([inst["s"] for inst in allinst])
    lq = {k: torch.tensor(np.asarray(v, np.float32), device=dev) for k, v in packed.items()}
    lq["S"] = None
    sd = torch.tensor(np.asarray(s, np.float32), device=dev)
    wb = {"instances": len(allinst), "distinct": uniq, "n": 36, "m": 24, "N": 100}
    refs = {}
    for i in range(uniq):                       # every distinct instance
        r32 = {k: np.asarray(allinst[i][k], np.float32).astype(np.float64) for k in synth.LQ_KEYS}
        refs[i] = oracle.riccati_solve(r32, np.asarray(s[i], np.float32).astype(np.float64))

    def run(name, warps, fn_name, refine, m_fp64=False):
        plan = pdilqr.Plan(36, 24, Nv, off, warps=warps, refine=refine, m_fp64=m_fp64)
        o = plan.alloc_out(device=dev, want_resid=True)
        fn = getattr(plan, fn_name)
        fn(lq, sd, out=o)
        torch.cuda.synchronize()
        t = event_times(torch, lambda: fn(lq, sd, out=o), 3, stream)
        bwd = pdilqr.backward_error(o["resid"]).cpu().numpy()
        z = {k: o[k].double().cpu().numpy() for k in ("dx", "du", "dlam")}
        errs = []
        for i, ref in refs.items():
            N, o0 = int(Nv[i]), int(off[i])
            e = 0.0
            for k, rk, n_slots in (("dx", "dx", N + 1), ("du", "du", N), ("dlam", "dlam", N + 1)):
                got, want = z[k][o0:o0 + n_slots], ref[rk][:n_slots]
                e = max(e, float(np.abs(got - want).max() / np.abs(want).max()))
            errs.append(e)
        rec = {"kkt_solves_per_s": len(allinst) / (np.mean(t) / 1e3), "ms": float(np.mean(t)),
               "warps": plan.warps, "max_backward_error": float(bwd.max()),
               "max_rel_error_vs_oracle": max(errs),
               "median_rel_error_vs_oracle": float(np.median(errs)),
               "within_1e-4": int(sum(e <= 1e-4 for e in errs))}
        if not refine:
            # the solve kernel alone (no residual): its algorithmic rate
            o2 = plan.alloc_out(device=dev)
            fn(lq, sd, out=o2)
            torch.cuda.synchronize()
            tk = event_times(torch, lambda: fn(lq, sd, out=o2), 3, stream)
            solver = "riccati" if warps == 1 else "scan"
            flops = float(np.sum(Nv + 1)) * lq_flops_per_stage(36, 24, solver)
            rec["roofline"] = dict(roofline_rec(flops, float(np.mean(tk)), peak),
                                   solve_ms=float(np.mean(tk)))
        plan.close()
        return rec

    for name, warps, fn_name, m64 in (("scan", 0, "kkt_scan_solve", False),
                                      ("scan_fp64_m", 0, "kkt_scan_solve", True),
                                      ("riccati", 1, "riccati_solve", False)):
        wb[name] = run(name, warps, fn_name, True, m64)
        wb[name]["unrefined"] = run(name, warps, fn_name, False, m64)
        wb[name]["oracle_compared"] = ("all 128 distinct instances; error = max over dx, du, dlam "
                                       "of |z - z_ref|_inf / |z_ref|_inf")
    wb["scan_fp64_m"]["note"] = ("the scan with its combines' M = I + C1 P2 factored and applied "
                                 "in FP64 (pdilqr_opts.m_fp64)")
    wb["note"] = ("refined: one correction solve against the FP64 KKT residual; unrefined: the "
                  "FP32 solve alone (both timings include the final FP64 residual for the "
                  "backward error)")
    out["whole_body_lq_batch"] = wb
    # single LQR (n = 4, m = 2, N = 16), graph replays
    inst = synth.ltv_lq(4, 2, 16, seed=0, **{k: v for k, v in synth.LQ_SMALL.items()
                                             if k not in ("n", "m", "N")})
    pk, Nv1, off1 = synth.pack([inst], synth.LQ_KEYS)
    lq1 = {k: torch.tensor(np.asarray(v, np.float32), device=dev) for k, v in pk.items()}
    lq1["S"] = None
    s1 = torch.tensor(np.asarray(inst["s"][None], np.float32), device=dev)
    single = {}
    for name, fn_name, refine in (("scan", "kkt_scan_solve", False), ("scan_refined", "kkt_scan_solve", True),
                                  ("riccati", "riccati_solve", False)):
        p1 = pdilqr.Plan(4, 2, Nv1, off1, refine=refine)
        o1 = p1.alloc_out(device=dev)
        fn = getattr(p1, fn_name)
        fn(lq1, s1, out=o1)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn(lq1, s1, out=o1)
        for _ in range(10):
            g.replay()
        t = event_times(torch, g.replay, args.latency_reps, stream)
        single[name] = {"p50_us": pct(t, 50) * 1e3, "p99_us": pct(t, 99) * 1e3}
    out["single_lqr_n4_N16"] = single
    out["large_state_lq"] = measure_large_state_lq(torch, pdilqr, oracle, dev, stream, args, peak)
    return out


def measure_e2e(torch, pdilqr, md, dev, stream, base, plan, args):
    """The same metric through the C ABI with host buffers: every step copies
    the problem (x0hat, warm start x, u, lam, references, contact) from pinned
    host memory, solves, and reads the solution (x, u) and status back."""
    host = {k: v.cpu().pin_memory() for k, v in base.items()}
    devb = {k: torch.empty_like(v) for k, v in base.items()}
    out_x = torch.empty_like(host["x"]).pin_memory()
    out_u = torch.empty_like(host["u"]).pin_memory()
    info = {"iters": torch.zeros(plan.count, device=dev, dtype=torch.int32),
            "status": torch.zeros(plan.count, device=dev, dtype=torch.int32),
            "alpha": None, "J": None, "theta": None}
    out_st = torch.empty(plan.count, dtype=torch.int32).pin_memory()
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    d2h = out_x.numel() * 4 + out_u.numel() * 4 + out_st.numel() * 4

    def step():
        for k in host:
            devb[k].copy_(host[k], non_blocking=True)
        plan.solve(md, devb["x0hat"], devb["x"], devb["u"], devb["lam"], devb["xref"],
                   devb["uref"], devb["contact"], max_iters=ITERS, info=info)
        out_x.copy_(devb["x"], non_blocking=True)
        out_u.copy_(devb["u"], non_blocking=True)
        out_st.copy_(info["status"], non_blocking=True)

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    t = event_times(torch, step, max(3, args.steps // 2), stream)
    kkt = int(info["iters"].sum().item())
    serial = {"value": kkt / (np.mean(t) / 1e3), "ms_per_step": float(np.mean(t)),
              "note": "one step at a time: copies in, solve, copies out, on one stream"}

    # pipelined: two device buffer sets; step i's host-to-device copies (on
    # the upload stream) and step i - 1's device-to-host copies (on the
    # download stream) overlap step i - 1's and i's solves on the compute
    # stream; every step still copies its own inputs in and its results out,
    # and the solves run one after another on the plan
    sets = [{k: torch.empty_like(v) for k, v in base.items()} for _ in range(2)]
    infos = [{"iters": torch.zeros(plan.count, device=dev, dtype=torch.int32),
              "status": torch.zeros(plan.count, device=dev, dtype=torch.int32),
              "alpha": None, "J": None, "theta": None} for _ in range(2)]
    outs = [(torch.empty_like(host["x"]).pin_memory(), torch.empty_like(host["u"]).pin_memory(),
             torch.empty(plan.count, dtype=torch.int32).pin_memory()) for _ in range(2)]
    up, down = torch.cuda.Stream(), torch.cuda.Stream()

    def pipelined(K):
        copied = [None, None]   # event: a set's inputs are on the device
        solved = [None, None]   # event: a set's solve is done
        freed = [None, None]    # event: a set's results have been read back
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        start.record(up)
        for i in range(K):
            b = i % 2
            d, inf = sets[b], infos[b]
            with torch.cuda.stream(up):
                if freed[b] is not None:
                    up.wait_event(freed[b])
                for k in host:
                    d[k].copy_(host[k], non_blocking=True)
                copied[b] = torch.cuda.Event()
                copied[b].record(up)
            stream.wait_event(copied[b])
            plan.solve(md, d["x0hat"], d["x"], d["u"], d["lam"], d["xref"], d["uref"], d["contact"],
                       max_iters=ITERS, info=inf, stream=stream)
            solved[b] = torch.cuda.Event()
            solved[b].record(stream)
            with torch.cuda.stream(down):
                down.wait_event(solved[b])
                ox, ou, ost = outs[b]
                ox.copy_(d["x"], non_blocking=True)
                ou.copy_(d["u"], non_blocking=True)
                ost.copy_(inf["status"], non_blocking=True)
                freed[b] = torch.cuda.Event()
                freed[b].record(down)
        down.wait_event(solved[(K - 1) % 2])
        end.record(down)
        end.synchronize()
        torch.cuda.synchronize()
        return start.elapsed_time(end) / K

    pipelined(4)
    K = max(6, args.steps)
    ms = pipelined(K)
    kkt = int(infos[0]["iters"].sum().item())
    return {"value": kkt / (ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": ms,
            "note": f"{K} steps pipelined on three streams (upload, solve, download) with two "
                    "device buffer sets; every step copies its own inputs in and its results "
                    "out", "serial": serial}


def client_robots(c: int, mix: str) -> int:
    """Robots of client c: "pair" alternates one and two robots; "full" gives
    60 % of the clients one robot and 10 % each two, four, eight and sixteen
    (half single-robot clients, half centralised problems with R drawn
    uniformly from {1, 2, 4, 8, 16})."""
    if mix == "pair":
        return 1 + (c % 2)
    return (1, 1, 1, 1, 1, 1, 2, 4, 8, 16)[c % 10]


def measure_serving(pdilqr, args, seconds: float, rate: float, max_batch: int, warps: int,
                    inflight: int, seed: int = 0, mix: str = "pair", large_cta_budget: int = 0,
                    split_min_robots: int = 0, split_max_batch: int = 0):
    """Poisson arrivals at ``rate`` requests/s for ``seconds``: each request is
    one real-time SQP iteration of a client's MPC problem (N = 50; robots per
    client as ``client_robots``, several robots coupled by the formation
    cost).  Returns achieved solves/s, latency percentiles (overall and per
    robot count) and the mean batch size."""
    import threading
    prm = synth.srbd_params(2)
    classes = {r: synth.srbd_params(r) for r in (1, 2, 4, 8, 16)}
    srv = pdilqr.Server(prm, hbm_budget_bytes=(1 << 30) if mix == "pair" else (16 << 30),
                        max_batch=max_batch, max_inflight=inflight, max_N=50, sqp_iters=1,
                        warps=warps, class_params=classes if mix != "pair" else None,
                        large_cta_budget=large_cta_budget, split_min_robots=split_min_robots,
                        split_max_batch=split_max_batch)
    # a client's ticks run one after another (each warm-starts the next), so
    # the full mix spreads the offered rate over more clients
    n_clients = 256 if mix == "pair" else 1024
    probs = {c: synth.srbd_problem(50, seed=10_000 + c, nrob=client_robots(c, mix))
             for c in range(n_clients)}
    g = np.random.default_rng(seed)
    gaps = g.exponential(1.0 / rate, size=int(rate * seconds * 1.2) + 16)
    picks = g.integers(0, n_clients, size=gaps.size)
    tickets = []
    lat = []
    lat_by = {}
    done = threading.Event()
    lock = threading.Lock()

    def collector():
        i = 0
        while True:
            with lock:
                have = i < len(tickets)
                tk = tickets[i] if have else None
            if not have:
                if done.is_set():
                    with lock:
                        if i >= len(tickets):
                            return
                    continue
                time.sleep(0.0002)
                continue
            r = srv.poll(tk[0], timeout_us=60_000_000)
            lat.append(r["latency_us"])
            lat_by.setdefault(tk[1], []).append(r["latency_us"])
            i += 1

    th = threading.Thread(target=collector, daemon=True)
    # admit every client once (untimed)
    first = [srv.submit(c, probs[c]["nrob"], 50, probs[c]["x0hat"], probs[c]["xref"],
                        probs[c]["uref"], probs[c]["contact"]) for c in range(n_clients)]
    for tk in first:
        srv.poll(tk, timeout_us=60_000_000)
    th.start()
    t0 = time.perf_counter()
    t_next = t0
    k = 0
    while t_next - t0 < seconds and k < gaps.size:
        now = time.perf_counter()
        if now < t_next:
            time.sleep(min(t_next - now, 0.001))
            continue
        c = int(picks[k])
        p = probs[c]
        tk = srv.submit(c, p["nrob"], 50, p["x0hat"], p["xref"], p["uref"], p["contact"])
        with lock:
            tickets.append((tk, p["nrob"]))
        t_next += gaps[k]
        k += 1
    done.set()
    th.join(timeout=120)
    t1 = time.perf_counter()
    st = srv.stats()
    srv.close()
    out = {"offered_per_s": rate, "requests": k, "solves_per_s": len(lat) / (t1 - t0),
           "p50_ms": pct(lat, 50) / 1e3, "p99_ms": pct(lat, 99) / 1e3,
           "mean_batch": st["mean_batch"], "max_batch": max_batch, "warps": warps,
           "streams": inflight, "large_cta_budget": large_cta_budget}
    if split_min_robots:
        out["split_min_robots"] = split_min_robots
        out["split_max_batch"] = split_max_batch
    if mix != "pair":
        out["by_robots"] = {str(r): {"requests": len(v), "p50_ms": pct(v, 50) / 1e3,
                                     "p99_ms": pct(v, 99) / 1e3}
                            for r, v in sorted(lat_by.items())}
    return out


# ------------------------------------------------------- horizon sweep
def run_sweep(args):
    """Single-instance latency of one SQP iteration (linearisation, LQ KKT
    solve, line search, update; CUDA-graph replays) against the horizon N
    (one robot) and against the robot count R of a centralised problem
    (n = m = 12 R, N = 50), for the scan and for the sequential recursion."""
    import torch
    from paper_2506_07823_b300 import pdilqr
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    return measure_sweep(torch, pdilqr, dev, torch.cuda.current_stream(), args.latency_reps)


def measure_sweep(torch, pdilqr, dev, stream, reps):
    """The sweep of ``run_sweep`` with ``reps`` graph replays per point."""

    def latency(nrob, N, warps, split=False):
        prm = synth.srbd_params(nrob)
        md = pdilqr.srbd_model(prm)
        pr = synth.srbd_problem(N, seed=SEED, nrob=nrob)
        pk, Nv, off = synth.pack([pr], synth.SRBD_KEYS)
        one = build_device_batch(torch, [pr], pk, Nv, off, pr["x0hat"][None], dev)
        w = {k: v.clone() for k, v in one.items()}
        n = 12 * nrob
        p = pdilqr.Plan(n, n, Nv, off, warps=warps, split=split)
        inf = {"iters": torch.zeros(1, device=dev, dtype=torch.int32),
               "status": torch.zeros(1, device=dev, dtype=torch.int32),
               "alpha": None, "J": None, "theta": None}

        def step():
            for k in ("x", "u", "lam"):
                w[k].copy_(one[k], non_blocking=True)
            p.solve(md, w["x0hat"], w["x"], w["u"], w["lam"], w["xref"], w["uref"], w["contact"],
                    max_iters=1, info=inf)
        step()
        torch.cuda.synchronize()
        if split:
            # split plans are not captured: direct calls (CUDA events)
            for _ in range(2):
                step()
            t = event_times(torch, step, max(5, min(reps, 20)), stream)
        else:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                step()
            for _ in range(5):
                g.replay()
            t = event_times(torch, g.replay, reps, stream)
        used = p.warps
        st = int(inf["status"].item())
        p.close()
        return {"p50_ms": pct(t, 50), "p99_ms": pct(t, 99), "warps": used, "status": st,
                "ctas_per_instance": used if split else 1}

    horizon = []
    for N in (25, 50, 100, 150, 200):
        sc, ri = latency(1, N, 16), latency(1, N, 1)
        horizon.append({"N": N, "scan": sc, "riccati": ri,
                        "speedup_p50": ri["p50_ms"] / sc["p50_ms"]})
    robots = []
    for R in (1, 2, 4, 8, 16):
        sc, ri = latency(R, 50, 0), latency(R, 50, 1)
        row = {"robots": R, "n": 12 * R, "scan": sc, "riccati": ri,
               "speedup_p50": ri["p50_ms"] / sc["p50_ms"]}
        if R >= 4:   # the scan's 16 chunks on 16 CTAs (unfused SQP iteration)
            row["scan_split"] = latency(R, 50, 16, split=True)
            row["split_speedup_p50"] = ri["p50_ms"] / row["scan_split"]["p50_ms"]
        robots.append(row)
    return {"sweep": "one SQP iteration, single instance, CUDA-graph replays",
            "horizon_n12": horizon, "robots_N50": robots,
            "work_ratio_scan_to_riccati": "about 50 n^3 vs 13 n^3 flop per stage (n = m)"}


# ------------------------------------------------------------ peak probes
def run_peaks(args):
    """Measured peak rates of this GPU's FP32 and FP64 FMA pipes and of its
    tensor cores on TF32 (tcgen05.mma, M = 128, N = 256, K = 8), best of five
    launches of about 50 ms each, with the SM clocks sampled meanwhile."""
    import torch
    from paper_2506_07823_b300 import pdilqr
    torch.cuda.set_device(0)
    clocks = ClockSampler(0)
    clocks.start()
    out = {}
    for name, kind in (("ffma_tflops", pdilqr.PEAK_FFMA), ("dfma_tflops", pdilqr.PEAK_DFMA),
                       ("tf32_mma_tflops", pdilqr.PEAK_TF32_MMA)):
        tf, ms = pdilqr.peak_probe(kind, 5)
        out[name] = tf
        out[name.replace("tflops", "launch_ms")] = ms
    out["clocks"] = clocks.stop()
    out["gpu"] = torch.cuda.get_device_name(0)
    out["sms"] = torch.cuda.get_device_properties(0).multi_processor_count
    return out


# --------------------------------------------------------- reference arm
def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    cores = host_cores()
    pool = oracle_pool(cores)
    insts, packed, Nv, off, x0 = synth.srbd_batch(args.count, seed=SEED, Ns_choices=HORIZONS)
    sample = insts[:sample_size(cores)]
    for _ in range(args.warmup):
        oracle_run(pool, cores, sample[:cores])
    tot_its, tot_s, per = 0, 0.0, []
    for _ in range(args.steps):
        its, secs, _ = oracle_run(pool, cores, sample)
        tot_its += its
        tot_s += secs
        per.append(secs)
    pool.close()
    value = tot_its / tot_s
    desc = (f"{len(sample)} of the {args.count} instances per step, one 10-iteration SQP "
            f"solve each, FP64 C oracle on {cores} host processes")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "instances_per_gpu": args.count,
                       "horizons": list(HORIZONS), "n": 12, "m": 12, "sqp_iters": ITERS},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--count", type=int, default=COUNT)
    ap.add_argument("--warps", type=int, default=0, choices=[0, 1, 4, 8, 16],
                    help="horizon chunks per instance of the batched solve (0: autotune over "
                         "1 = the sequential recursion and the scan's 4, 8, 16)")
    ap.add_argument("--inst-per-cta", type=int, default=0, choices=[0, 2, 4, 8],
                    help="instances per CTA of the sequential solver when --warps 1 (0: 2)")
    ap.add_argument("--latency-reps", type=int, default=200)
    ap.add_argument("--comparator-sample", type=int, default=512)
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--serve-seconds", type=float, default=5.0,
                    help="duration of each serving scenario (0 skips them)")
    ap.add_argument("--serve-rate", type=float, default=2000.0, help="Poisson arrival rate (1/s)")
    ap.add_argument("--serve-rate-sustained", type=float, default=400.0,
                    help="the equal-load rate of both servers (one the one-request-per-launch "
                         "server sustains)")
    ap.add_argument("--mix-seconds", type=float, default=60.0,
                    help="duration of the full robot-count mix (0 skips it with the others when "
                         "--serve-seconds is 0)")
    ap.add_argument("--mix-large-ctas", type=int, default=0,
                    help="large_cta_budget of the full-mix server: most instances of 4+ robots "
                         "in flight (0: no budget; with 8 streams a budget of 32 or 64 did not "
                         "bring the small classes back to their 4-stream latency)")
    ap.add_argument("--mix-split-seconds", type=float, default=30.0,
                    help="duration of the full mix with the large classes on the split scan "
                         "(0 skips it)")
    ap.add_argument("--mix-split-robots", type=int, default=16,
                    help="split_min_robots of that server: classes of this many robots or more "
                         "run the split scan (4, 8 or 16; 8 and 4 measured a higher overall p99)")
    ap.add_argument("--mix-split-batch", type=int, default=8,
                    help="split_max_batch of that server: most instances of one split batch "
                         "(4 could not keep up with 200 sixteen-robot requests/s)")
    ap.add_argument("--mix-streams", type=int, default=4,
                    help="batches in flight (streams) of the full-mix server, 1..16 (8 measured "
                         "worse than 4: large-class batches then occupy every SM and the "
                         "one-robot requests wait behind them)")
    ap.add_argument("--no-lq-workloads", dest="lq_workloads", action="store_false",
                    help="skip the whole-body LQ batch and single-LQR measurements")
    ap.add_argument("--lq-only", action="store_true",
                    help="print the LQ-solve workloads (whole-body-sized batch, single LQR) only")
    ap.add_argument("--sweep-reps", type=int, default=20,
                    help="graph replays per point of the horizon / robot-count sweep that the "
                         "bench line carries (0: leave it out)")
    ap.add_argument("--sweep", action="store_true",
                    help="print the horizon / robot-count latency sweep instead of the bench line")
    ap.add_argument("--peaks", action="store_true",
                    help="print the measured FFMA, DFMA and TF32 tensor-core peaks instead")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.sweep:
        print(json.dumps(run_sweep(args)), flush=True)
        return
    if args.peaks:
        print(json.dumps(run_peaks(args)), flush=True)
        return
    if args.lq_only:
        import torch
        from paper_2506_07823_b300 import pdilqr
        torch.cuda.set_device(0)
        peak, _ = pdilqr.peak_probe(pdilqr.PEAK_FFMA, 3)
        print(json.dumps(measure_lq_workloads(torch, pdilqr, torch.device("cuda", 0),
                                              torch.cuda.current_stream(), args, peak)), flush=True)
        return
    res = run_reference(args) if args.impl == "reference" else run_gpu(args)
    if res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
