"""Batch autotuner of the fused SQP solve.

Host logic only: it creates one plan per candidate configuration, times the
library's kernels on the caller's batch with CUDA events, and keeps the
fastest plan.  Nothing of the method is computed here.

Candidate configurations of a batch of SRBD problems (``pdilqr_opts``):

* the solver and its tiling of the horizon: ``warps = 1`` runs the sequential
  Riccati recursion of Sec. II-C (one chunk per instance); 4, 8 or 16 run the
  parallel scan of Sec. II-D over that many horizon chunks per instance;
* for the one-robot sequential solver (n = m = 12), the instances per CTA:
  2, 4 or 8 (CTAs of 1, 2 or 4 warps, two instances per warp).

A configuration that a size does not support is skipped.
"""
from __future__ import annotations

from . import pdilqr


def candidates(n: int, m: int):
    """(warps, inst_per_cta) pairs worth timing for a batch of size (n, m)."""
    if n == 12 and m == 12:
        return [(1, 2), (1, 4), (1, 8), (4, 0), (8, 0), (16, 0)]
    return [(1, 0), (4, 0), (8, 0), (16, 0)]


def label(warps: int, inst_per_cta: int) -> str:
    """Short name of a configuration: ``seq/<instances per CTA>`` or ``scan/<chunks>``."""
    if warps == 1:
        return f"seq/{inst_per_cta or 1}"
    return f"scan/{warps}"


def autotune_sqp(torch, n: int, m: int, N, stage_off, solve, reset=None, flush=None,
                 reps: int = 2, stream=None, cands=None):
    """Pick the fastest fused-SQP configuration for one batch.

    ``solve(plan)`` runs one batched solve of the caller's problem data on
    ``plan`` (``Plan.solve``); the SQP updates the trajectory in place, so
    ``reset()`` restores the warm start before every solve and ``flush()``
    (optional) evicts L2; both run outside the timed events.  Each candidate
    runs once untimed, then ``reps`` timed solves; its time is the fastest.

    Returns ``(plan, times)``: the fastest plan (the others are closed) and
    the time in ms of every candidate that ran, keyed by ``label``.
    """
    stream = stream or torch.cuda.current_stream()
    plans, times = {}, {}
    for warps, ipc in (cands or candidates(n, m)):
        try:
            p = pdilqr.Plan(n, m, N, stage_off, warps=warps, inst_per_cta=ipc)
        except pdilqr.PdilqrError:
            continue
        key = label(warps, ipc)
        if reset:
            reset()
        solve(p)
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            if reset:
                reset()
            if flush:
                flush()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            solve(p)
            e1.record(stream)
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        plans[key], times[key] = p, best
    if not plans:
        raise pdilqr.PdilqrError(pdilqr.E_INVALID_ARG, "autotune_sqp: no configuration runs")
    key = min(times, key=times.get)
    for k, p in plans.items():
        if k != key:
            p.close()
    return plans[key], times
