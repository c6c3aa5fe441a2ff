"""Parity of the GPU LQ KKT solvers (scan and sequential Riccati) with the
FP64 oracle, through the C ABI.

Tolerances (stated by the target): per block (dx, du, dlam) the relative
error |z_gpu - z_ref|_inf / |z_ref|_inf <= 1e-4, and with the FP64-residual
refinement step the normwise KKT backward error <= 1e-6.  The oracle solves
the same FP32-rounded data in FP64.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_07823_b300 import synth

pytestmark = pytest.mark.gpu

REL_TOL = 1e-4
BWD_TOL = 1e-6


def rounded(lq):
    return {k: np.asarray(v, dtype=np.float32).astype(np.float64) for k, v in lq.items()}


def lq_with_S(n, m, N, seed):
    """Random convex LQ data with a nonzero cross term S."""
    g = np.random.default_rng(seed)
    d = synth.ltv_lq(n, m, N, seed, rho=0.95, b_std=0.5, q_kind="diag", r_w=0.1)
    for k in range(N):
        L = g.normal(0, 0.3, (n + m, n + m))
        H = L @ L.T + 0.2 * np.eye(n + m)
        d["Q"][k] = H[:n, :n]
        d["R"][k] = H[n:, n:]
        d["S"][k] = H[n:, :n]
    return d


def make_batch(n, m, Ns, seed, with_S=False, **kw):
    insts = []
    for i, N in enumerate(Ns):
        if with_S:
            insts.append(lq_with_S(n, m, N, seed + i))
        else:
            args = dict(rho=0.95, b_std=0.5, q_kind="diag", r_w=0.1)
            args.update(kw)
            insts.append(synth.ltv_lq(n, m, N, seed + i, **args))
    packed, Nv, off = synth.pack(insts, synth.LQ_KEYS)
    s = np.stack([inst["s"] for inst in insts])
    return insts, packed, Nv, off, s


def to_dev(packed, s, with_S):
    lq = {k: torch.tensor(np.asarray(v, dtype=np.float32), device="cuda") for k, v in packed.items()}
    if not with_S:
        lq["S"] = None
    return lq, torch.tensor(np.asarray(s, dtype=np.float32), device="cuda")


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-30)


def check_parity(insts, Nv, off, out, s, with_S, policy=False):
    dx = out["dx"].double().cpu().numpy()
    du = out["du"].double().cpu().numpy()
    dl = out["dlam"].double().cpu().numpy()
    st = out["status"].cpu().numpy()
    assert np.all(st == 0), st
    worst = 0.0
    for i, inst in enumerate(insts):
        N, o = int(Nv[i]), int(off[i])
        lq = rounded({k: inst[k] for k in synth.LQ_KEYS})
        si = np.asarray(s[i], dtype=np.float32).astype(np.float64)
        ref = oracle.riccati_solve(lq, si)
        sl = slice(o, o + N + 1)
        e = max(rel(dx[sl], ref["dx"]), rel(du[o:o + N], ref["du"][:N]), rel(dl[sl], ref["dlam"]))
        worst = max(worst, e)
        assert rel(dx[sl], ref["dx"]) <= REL_TOL, (i, N, rel(dx[sl], ref["dx"]))
        assert rel(du[o:o + N], ref["du"][:N]) <= REL_TOL, (i, N)
        assert rel(dl[sl], ref["dlam"]) <= REL_TOL, (i, N)
        assert np.all(du[o + N] == 0.0)
        if policy:
            K = out["K"].double().cpu().numpy()[sl]
            P = out["P"].double().cpu().numpy()[sl]
            assert rel(K[:N], ref["K"][:N]) <= REL_TOL
            assert rel(P, ref["P"]) <= REL_TOL
    return worst


@pytest.mark.parametrize("solver", ["scan", "riccati"])
@pytest.mark.parametrize("warps", [4, 8, 16])
@pytest.mark.parametrize("n,m", [(1, 1), (2, 1), (3, 2), (4, 2), (12, 12), (24, 24), (36, 24)])
def test_ltv_parity_ragged(solver, warps, n, m):
    """Uneven horizons in one batch: N = 1 (degenerate), tiny, and spanning
    several chunks with a ragged tail."""
    if solver == "riccati" and warps != 4:
        pytest.skip("warp count only affects the scan")
    if n == 24 and warps != 4:
        pytest.skip("n = 24 fits shared memory with 4 warps per instance only")
    if n == 36 and warps == 16:
        pytest.skip("n = 36 runs chunks of 4 warps: at most 8 chunks per 1024-thread CTA")
    Ns = [1, 2, 3, 5, 16, 17, 50, 100]
    insts, packed, Nv, off, s = make_batch(n, m, Ns, seed=100 * n + m)
    from paper_2506_07823_b300.pdilqr import Plan
    plan = Plan(n, m, Nv, off, warps=warps)
    lq, sd = to_dev(packed, s, False)
    fn = plan.kkt_scan_solve if solver == "scan" else plan.riccati_solve
    out = fn(lq, sd, want_policy=True)
    torch.cuda.synchronize()
    check_parity(insts, Nv, off, out, s, False, policy=True)


@pytest.mark.parametrize("solver", ["scan", "riccati"])
@pytest.mark.parametrize("n,m", [(4, 2), (24, 24), (36, 24)])
def test_cross_term_S(solver, n, m):
    """A nonzero cross term S (m x n) through every path that reads it (the
    one-CTA recursion of n = 24 and 36 adds S in H and S^T [K | k] in the
    value function)."""
    insts, packed, Nv, off, s = make_batch(n, m, [7, 30, 64], seed=5 + n, with_S=True)
    from paper_2506_07823_b300.pdilqr import Plan
    plan = Plan(n, m, Nv, off, warps=8 if n == 4 else 4)
    lq, sd = to_dev(packed, s, True)
    fn = plan.kkt_scan_solve if solver == "scan" else plan.riccati_solve
    out = fn(lq, sd)
    torch.cuda.synchronize()
    check_parity(insts, Nv, off, out, s, True)


def test_single_lqr_workload_exact_config():
    """The small single-LQR workload: n=4, m=2, N=16, seed 0."""
    cfg = synth.LQ_SMALL
    inst = synth.ltv_lq(cfg["n"], cfg["m"], cfg["N"], seed=0, rho=cfg["rho"], b_std=cfg["b_std"],
                        q_kind=cfg["q_kind"], r_w=cfg["r_w"])
    packed, Nv, off = synth.pack([inst], synth.LQ_KEYS)
    from paper_2506_07823_b300.pdilqr import Plan, backward_error
    plan = Plan(4, 2, Nv, off, refine=True)
    lq, sd = to_dev(packed, inst["s"][None], False)
    out = plan.kkt_scan_solve(lq, sd, want_resid=True)
    torch.cuda.synchronize()
    check_parity([inst], Nv, off, out, inst["s"][None], False)
    assert float(backward_error(out["resid"]).max()) <= BWD_TOL


@pytest.mark.parametrize("solver", ["scan", "riccati"])
@pytest.mark.parametrize("n,m", [(4, 2), (12, 12)])
def test_refinement_backward_error(solver, n, m):
    """One refinement step against the FP64 residual brings the normwise
    backward error to <= 1e-6 and keeps the parity."""
    insts, packed, Nv, off, s = make_batch(n, m, [10, 50, 100, 33], seed=77)
    from paper_2506_07823_b300.pdilqr import Plan, backward_error
    plan0 = Plan(n, m, Nv, off, refine=False)
    plan1 = Plan(n, m, Nv, off, refine=True)
    lq, sd = to_dev(packed, s, False)
    fn0 = plan0.kkt_scan_solve if solver == "scan" else plan0.riccati_solve
    fn1 = plan1.kkt_scan_solve if solver == "scan" else plan1.riccati_solve
    o0 = fn0(lq, sd, want_resid=True)
    o1 = fn1(lq, sd, want_resid=True)
    torch.cuda.synchronize()
    b0 = backward_error(o0["resid"]).cpu().numpy()
    b1 = backward_error(o1["resid"]).cpu().numpy()
    assert np.all(b1 <= BWD_TOL), b1
    assert np.all(b1 <= b0 * 1.01 + 1e-12), (b0, b1)
    check_parity(insts, Nv, off, o1, s, False)


@pytest.mark.parametrize("solver", ["scan", "riccati"])
def test_whole_body_sized_workload(solver):
    """The whole-body-sized LTV batch recipe (n = 36, m = 24, N = 100,
    spectral radius 0.98, Q = L L^T + 0.1 I, R = 0.01 I) on a few instances,
    with the FP64-residual refinement step."""
    cfg = synth.LQ_WB
    insts, packed, Nv, off, s = make_batch(36, 24, [100, 100, 37], seed=4000, rho=cfg["rho"],
                                           b_std=cfg["b_std"], q_kind=cfg["q_kind"], r_w=cfg["r_w"])
    from paper_2506_07823_b300.pdilqr import Plan, backward_error
    plan = Plan(36, 24, Nv, off, refine=True)
    lq, sd = to_dev(packed, s, False)
    fn = plan.kkt_scan_solve if solver == "scan" else plan.riccati_solve
    out = fn(lq, sd, want_resid=True)
    torch.cuda.synchronize()
    check_parity(insts, Nv, off, out, s, False)
    assert float(backward_error(out["resid"]).max()) <= BWD_TOL


@pytest.mark.parametrize("n,m,with_S", [(4, 2, False), (12, 12, False), (24, 24, True),
                                          (36, 24, False), (36, 24, True)])
def test_residual_kernel_matches_oracle(n, m, with_S):
    """The FP64 residual kernels (one warp per stage slot at n = 4; the
    shared-memory staged form with one thread per row at n = 12, 24, 36)
    reproduce the oracle's residual norms, with and without S, over a batch
    whose slots do not fill the last block."""
    Ns = [3, 9] if n == 4 else [3, 9, 1, 6]
    insts, packed, Nv, off, s = make_batch(n, m, Ns, seed=3 + n, with_S=with_S)
    from paper_2506_07823_b300.pdilqr import Plan
    plan = Plan(n, m, Nv, off)
    lq, sd = to_dev(packed, s, with_S)
    g = np.random.default_rng(0)
    T = plan.total
    z = [g.normal(0, 1, (T, n)).astype(np.float32), g.normal(0, 1, (T, m)).astype(np.float32),
         g.normal(0, 1, (T, n)).astype(np.float32)]
    for i, N in enumerate(Nv):
        z[1][off[i] + N] = 0.0
    res = plan.kkt_residual(lq, sd, *[torch.tensor(v, device="cuda") for v in z])
    torch.cuda.synchronize()
    res = res.cpu().numpy()
    for i, inst in enumerate(insts):
        N, o = int(Nv[i]), int(off[i])
        lqr = rounded({k: inst[k] for k in synth.LQ_KEYS})
        want = oracle.kkt_residual(lqr, np.asarray(s[i], np.float32).astype(np.float64),
                                   *[v[o:o + N + 1].astype(np.float64) for v in z])
        np.testing.assert_allclose(res[i], want, rtol=1e-12)


@pytest.mark.parametrize("n,m", [(4, 2), (36, 24)])
def test_not_spd_status(n, m):
    """A control Hessian that is not positive definite is reported, not hidden
    (one-warp elimination at n = 4, the wide-group elimination at n = 36)."""
    insts, packed, Nv, off, s = make_batch(n, m, [6, 6], seed=9)
    packed["R"][off[1] + 2] = -np.eye(m)
    from paper_2506_07823_b300.pdilqr import Plan
    plan = Plan(n, m, Nv, off, warps=4)
    lq, sd = to_dev(packed, s, False)
    for fn in (plan.kkt_scan_solve, plan.riccati_solve):
        out = fn(lq, sd)
        torch.cuda.synchronize()
        st = out["status"].cpu().numpy()
        assert st[0] == 0 and st[1] != 0


def test_batch_alone_equals_in_mix():
    """An instance solved alone equals the same instance inside a batch."""
    n, m = 12, 12
    insts, packed, Nv, off, s = make_batch(n, m, [40, 25, 75, 100, 1], seed=31)
    from paper_2506_07823_b300.pdilqr import Plan
    plan = Plan(n, m, Nv, off, warps=8)
    lq, sd = to_dev(packed, s, False)
    mix = plan.kkt_scan_solve(lq, sd)
    i = 2
    pk1, Nv1, off1 = synth.pack([insts[i]], synth.LQ_KEYS)
    plan1 = Plan(n, m, Nv1, off1, warps=8)
    lq1, sd1 = to_dev(pk1, s[i:i + 1], False)
    alone = plan1.kkt_scan_solve(lq1, sd1)
    torch.cuda.synchronize()
    sl = slice(int(off[i]), int(off[i]) + int(Nv[i]) + 1)
    assert torch.equal(mix["dx"][sl], alone["dx"])
    assert torch.equal(mix["dlam"][sl], alone["dlam"])


@pytest.mark.parametrize("solver", ["scan", "riccati"])
@pytest.mark.parametrize("n,m", [(4, 2), (12, 12), (36, 24)])
def test_nonfinite_status(solver, n, m):
    """A NaN in one instance's gradient q_k, or an Inf in another's initial
    defect, is reported as E_NONFINITE for that instance only; the other
    instances of the batch keep their solution."""
    insts, packed, Nv, off, s = make_batch(n, m, [9, 12, 20, 7], seed=13)
    packed["q"][off[1] + 4, 0] = np.nan
    s = s.copy()
    s[3, 0] = np.inf
    from paper_2506_07823_b300.pdilqr import Plan, E_NONFINITE
    plan = Plan(n, m, Nv, off, warps=4)
    lq, sd = to_dev(packed, s, False)
    fn = plan.kkt_scan_solve if solver == "scan" else plan.riccati_solve
    out = fn(lq, sd)
    torch.cuda.synchronize()
    st = out["status"].cpu().numpy()
    assert st[1] == E_NONFINITE and st[3] == E_NONFINITE, st
    keep = [0, 2]
    sub = {k: out[k] for k in ("dx", "du", "dlam")}
    sub["status"] = out["status"][keep]
    check_parity([insts[i] for i in keep], Nv[keep], off[keep], sub, s[keep], False)


@pytest.mark.parametrize("n,m", [(24, 24), (36, 24)])
def test_bulk_copy_timeout_status(n, m):
    """The one-CTA recursion's stage copies go through the TMA engine with a
    bounded wait: with the test switch that issues none of them, every
    instance ends with E_TIMEOUT (nothing is in flight), and the same plan
    then solves normally."""
    from paper_2506_07823_b300 import pdilqr
    insts, packed, Nv, off, s = make_batch(n, m, [5, 3], seed=71)
    plan = pdilqr.Plan(n, m, Nv, off)
    lq, sd = to_dev(packed, s, False)
    plan.set_debug(pdilqr.DEBUG_BULK_SKIP_ISSUE)
    out = plan.riccati_solve(lq, sd)
    torch.cuda.synchronize()
    assert np.all(out["status"].cpu().numpy() == pdilqr.E_TIMEOUT)
    plan.set_debug(0)
    out = plan.riccati_solve(lq, sd)
    torch.cuda.synchronize()
    check_parity(insts, Nv, off, out, s, False)


def test_misaligned_arrays_are_rejected():
    """Every per-stage array is read with 16-byte accesses: a pointer that is
    not 16-byte aligned is an invalid argument (no launch)."""
    from paper_2506_07823_b300 import pdilqr
    n, m = 36, 24
    insts, packed, Nv, off, s = make_batch(n, m, [4], seed=72)
    plan = pdilqr.Plan(n, m, Nv, off)
    lq, sd = to_dev(packed, s, False)
    base = lq["q"]
    shifted = torch.empty(base.numel() + 1, device="cuda", dtype=torch.float32)
    shifted[1:].copy_(base.reshape(-1))
    lq["q"] = shifted[1:].reshape(base.shape)
    with pytest.raises(pdilqr.PdilqrError, match="INVALID_ARG"):
        plan.riccati_solve(lq, sd)


@pytest.mark.parametrize("warps", [4, 8])
def test_m_fp64_parity_ragged(warps):
    """The scan with its combines' M = I + C1 P2 eliminated in FP64 (the
    whole-body size): uneven horizons, policy and value function against the
    oracle."""
    from paper_2506_07823_b300.pdilqr import Plan
    Ns = [1, 2, 3, 5, 16, 17, 50, 100]
    insts, packed, Nv, off, s = make_batch(36, 24, Ns, seed=3624)
    plan = Plan(36, 24, Nv, off, warps=warps, m_fp64=True)
    lq, sd = to_dev(packed, s, False)
    out = plan.kkt_scan_solve(lq, sd, want_policy=True)
    torch.cuda.synchronize()
    check_parity(insts, Nv, off, out, s, False, policy=True)


def test_m_fp64_whole_body_workload():
    """The whole-body-sized recipe through the FP64-M scan, unrefined and
    refined, within the stated tolerances of the oracle."""
    cfg = synth.LQ_WB
    insts, packed, Nv, off, s = make_batch(36, 24, [100, 100, 37], seed=4000, rho=cfg["rho"],
                                           b_std=cfg["b_std"], q_kind=cfg["q_kind"], r_w=cfg["r_w"])
    from paper_2506_07823_b300.pdilqr import Plan, backward_error
    lq, sd = to_dev(packed, s, False)
    for refine in (False, True):
        plan = Plan(36, 24, Nv, off, m_fp64=True, refine=refine)
        out = plan.kkt_scan_solve(lq, sd, want_resid=True)
        torch.cuda.synchronize()
        check_parity(insts, Nv, off, out, s, False)
        if refine:
            assert float(backward_error(out["resid"]).max()) <= BWD_TOL


def test_m_fp64_rejected_elsewhere():
    """The FP64 elimination of M exists at (n, m) = (36, 24) only."""
    from paper_2506_07823_b300 import pdilqr
    for n, m in ((12, 12), (24, 24), (4, 2)):
        with pytest.raises(pdilqr.PdilqrError) as e:
            pdilqr.Plan(n, m, [10, 20], [0, 11], m_fp64=True)
        assert e.value.code == pdilqr.E_INVALID_ARG


@pytest.mark.parametrize("n,warps,Ns,refine", [(48, 8, [1, 3, 17, 50], False),
                                               (48, 16, [2, 16, 33, 50], False),
                                               (96, 16, [5, 50], True), (192, 16, [20], True)])
def test_split_scan_parity(n, warps, Ns, refine):
    """The scan with its horizon chunks on separate CTAs (one per chunk,
    bounded barriers between the phases): uneven horizons, horizons shorter
    than the chunk count, against the oracle.  At n = 96 and 192 the FP32
    solve of this recipe alone misses 1e-4 with every solver (the sequential
    recursion included: M = I + C1 P2 and G are ill-conditioned at these
    sizes), so there the parity is that of the precision line: one
    refinement step against the FP64 residual, and the backward error."""
    from paper_2506_07823_b300.pdilqr import Plan, backward_error
    insts, packed, Nv, off, s = make_batch(n, n, Ns, seed=7000 + n + warps)
    plan = Plan(n, n, Nv, off, warps=warps, split=True, refine=refine)
    assert plan.warps == warps
    lq, sd = to_dev(packed, s, False)
    out = plan.kkt_scan_solve(lq, sd, want_policy=not refine, want_resid=refine)
    torch.cuda.synchronize()
    check_parity(insts, Nv, off, out, s, False, policy=not refine)
    if refine:
        assert float(backward_error(out["resid"]).max()) <= BWD_TOL
    # the chunks really ran apart: the result differs from the one-chunk
    # recursion's in its rounding
    seq = Plan(n, n, Nv, off, warps=1, refine=refine).kkt_scan_solve(lq, sd)
    torch.cuda.synchronize()
    assert not torch.equal(out["dx"], seq["dx"])


def test_split_scan_refined_twice():
    """The refinement step's correction solve goes through the split scan too;
    two solves in a row on one plan (the phase counters restart at zero)."""
    from paper_2506_07823_b300.pdilqr import Plan, backward_error
    insts, packed, Nv, off, s = make_batch(96, 96, [40, 7, 25], seed=7096)
    plan = Plan(96, 96, Nv, off, split=True, refine=True)
    lq, sd = to_dev(packed, s, False)
    for _ in range(2):
        out = plan.kkt_scan_solve(lq, sd, want_resid=True)
        torch.cuda.synchronize()
        check_parity(insts, Nv, off, out, s, False)
        assert float(backward_error(out["resid"]).max()) <= BWD_TOL


def test_split_scan_rejected_elsewhere():
    """Chunks on separate CTAs exist for the 8-warp-unit sizes (n >= 48) with 8
    or 16 chunks only."""
    from paper_2506_07823_b300 import pdilqr
    for n, m, warps in ((12, 12, 16), (36, 24, 8), (48, 48, 4), (96, 96, 1)):
        with pytest.raises(pdilqr.PdilqrError) as e:
            pdilqr.Plan(n, m, [10, 20], [0, 11], warps=warps, split=True)
        assert e.value.code == pdilqr.E_INVALID_ARG


def test_split_scan_barrier_timeout_status():
    """The bounded barrier of the split scan: with the test switch that keeps
    chunk 0 from arriving at the first barrier (nothing in flight), every CTA's
    wait runs out, the instance ends with E_TIMEOUT within a few seconds, and
    the next solve on the same plan is correct."""
    import time
    from paper_2506_07823_b300 import pdilqr
    insts, packed, Nv, off, s = make_batch(48, 48, [30], seed=4848)
    plan = pdilqr.Plan(48, 48, Nv, off, warps=8, split=True)
    lq, sd = to_dev(packed, s, False)
    plan.set_debug(pdilqr.DEBUG_SPLIT_SKIP_ARRIVE)
    t0 = time.time()
    out = plan.kkt_scan_solve(lq, sd)
    torch.cuda.synchronize()
    assert out["status"].item() == pdilqr.E_TIMEOUT
    assert time.time() - t0 < 30.0
    plan.set_debug(0)
    out = plan.kkt_scan_solve(lq, sd)
    torch.cuda.synchronize()
    check_parity(insts, Nv, off, out, s, False)


def test_split_scan_with_cross_term_S():
    """The split scan with a nonzero cross term S (element build through
    R^-1 [B^T | S | r]) at n = 96, where the combines take the shared-memory LU
    of M, through the refinement step."""
    from paper_2506_07823_b300.pdilqr import Plan, backward_error
    insts, packed, Nv, off, s = make_batch(96, 96, [30, 9], seed=9696, with_S=True)
    plan = Plan(96, 96, Nv, off, warps=16, split=True, refine=True)
    lq, sd = to_dev(packed, s, True)
    out = plan.kkt_scan_solve(lq, sd, want_resid=True)
    torch.cuda.synchronize()
    check_parity(insts, Nv, off, out, s, True)
    assert float(backward_error(out["resid"]).max()) <= BWD_TOL


def test_split_scan_refuses_a_grid_that_cannot_be_resident():
    """The split scan's CTAs wait on one another, so all chunks x instances of a
    launch must be resident together: at n = 192 (one CTA per SM) ten
    instances of 16 chunks (160 CTAs) are refused on the host before any
    kernel runs, and the same plan shape with nine instances solves."""
    from paper_2506_07823_b300 import pdilqr
    Ns = [4] * 10
    insts, packed, Nv, off, s = make_batch(192, 192, Ns, seed=19210)
    lq, sd = to_dev(packed, s, False)
    plan = pdilqr.Plan(192, 192, Nv, off, warps=16, split=True)
    with pytest.raises(pdilqr.PdilqrError) as e:
        plan.kkt_scan_solve(lq, sd)
        torch.cuda.synchronize()
    assert e.value.code == pdilqr.E_CUDA
    plan9 = pdilqr.Plan(192, 192, Nv[:9], off[:9], warps=16, split=True)
    out = plan9.kkt_scan_solve(lq, sd)
    torch.cuda.synchronize()
    assert np.all(out["status"].cpu().numpy() == 0)
