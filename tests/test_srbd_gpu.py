"""Parity of the SRBD linearisation, the line-search merit and the fused SQP
with the FP64 oracle, through the C ABI.

The oracle receives the same FP32-rounded inputs in FP64.  Tolerance: the
target's 1e-4 relative error per block (normwise, infinity norm).  Full SQP
runs are compared in replay mode (the GPU takes the oracle's step sizes) and
free-running (the step sizes must agree and so must the iterates).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_07823_b300 import synth

pytestmark = pytest.mark.gpu

REL_TOL = 1e-4


def r32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-30)


def perturbed_batch(count, seed, Ns, nrob=1):
    """SRBD problems with perturbed trajectories and costates (so every term of
    the linearisation is exercised)."""
    insts = []
    g = np.random.default_rng(seed)
    for i in range(count):
        pr = synth.srbd_problem(Ns[i % len(Ns)], seed=seed + i, nrob=nrob)
        pr["x"] = pr["x"] + g.normal(0, 0.05, pr["x"].shape)
        pr["u"] = pr["u"] + g.normal(0, 4.0, pr["u"].shape)
        pr["u"][-1] = 0.0
        pr["lam"] = g.normal(0, 1.0, pr["lam"].shape)
        insts.append(pr)
    packed, Nv, off = synth.pack(insts, synth.SRBD_KEYS)
    x0 = np.stack([p["x0hat"] for p in insts])
    return insts, packed, Nv, off, x0


def dev(packed):
    out = {}
    for k, v in packed.items():
        if k == "contact":
            out[k] = torch.tensor(np.asarray(v, dtype=np.uint8), device="cuda")
        else:
            out[k] = torch.tensor(np.asarray(v, dtype=np.float32), device="cuda")
    return out


@pytest.mark.parametrize("nrob", [1, 2, 4, 8, 16])
def test_linearize_parity(nrob):
    from paper_2506_07823_b300 import pdilqr
    n = 12 * nrob
    insts, packed, Nv, off, x0 = perturbed_batch(3, 40 + nrob, [5, 9, 1], nrob)
    prm = synth.srbd_params(nrob)
    plan = pdilqr.Plan(n, n, Nv, off)
    out = plan.linearize(pdilqr.srbd_model(prm), dev(packed))
    torch.cuda.synchronize()
    got = {k: v.double().cpu().numpy() for k, v in out.items()}
    for i, pr in enumerate(insts):
        N, o = int(Nv[i]), int(off[i])
        ref = oracle.srbd_linearize(prm, r32(pr["x"]), r32(pr["u"]), r32(pr["lam"]),
                                    r32(pr["xref"]), r32(pr["uref"]), pr["contact"])
        sl = slice(o, o + N + 1)
        for k in ("A", "B", "Q", "R", "q", "r"):
            assert rel(got[k][sl], ref[k]) <= REL_TOL, (k, rel(got[k][sl], ref[k]))
        # the defect is a difference of O(1) states: compare against their scale
        assert np.abs(got["c"][sl] - ref["c"]).max() <= 1e-5 * max(1, np.abs(pr["x"]).max())
        assert np.all(got["S"][sl] == 0)


def test_merit_parity():
    from paper_2506_07823_b300 import pdilqr
    insts, packed, Nv, off, x0 = perturbed_batch(3, 7, [12, 30, 2])
    prm = synth.srbd_params()
    g = np.random.default_rng(1)
    T = int(off[-1] + Nv[-1] + 1)
    dx = (g.normal(0, 0.02, (T, 12))).astype(np.float32)
    du = (g.normal(0, 2.0, (T, 12))).astype(np.float32)
    for i, N in enumerate(Nv):
        du[off[i] + N] = 0
    d = dev(packed)
    plan = pdilqr.Plan(12, 12, Nv, off)
    mer = plan.merit_eval(pdilqr.srbd_model(prm), d, torch.tensor(x0, dtype=torch.float32, device="cuda"),
                          torch.tensor(dx, device="cuda"), torch.tensor(du, device="cuda"))
    torch.cuda.synchronize()
    mer = mer.cpu().numpy()
    for i, pr in enumerate(insts):
        N, o = int(Nv[i]), int(off[i])
        sl = slice(o, o + N + 1)
        x, u = r32(pr["x"]), r32(pr["u"])
        args = (r32(pr["xref"]), r32(pr["uref"]), pr["contact"])
        J0, th0 = oracle.srbd_merit(prm, r32(pr["x0hat"]), x, u, *args)
        assert abs(mer[i, 0] - J0) <= 1e-5 * abs(J0)
        assert abs(mer[i, 1] - th0) <= 1e-4 * th0 + 1e-5
        # directional derivative by central differences of the oracle's cost
        h = 1e-6
        Jp, _ = oracle.srbd_merit(prm, r32(pr["x0hat"]), x + h * dx[sl], u + h * du[sl], *args)
        Jm, _ = oracle.srbd_merit(prm, r32(pr["x0hat"]), x - h * dx[sl], u - h * du[sl], *args)
        fd = (Jp - Jm) / (2 * h)
        assert abs(mer[i, 2] - fd) <= 1e-3 * max(1, abs(fd))
        for t in range(10):
            a = 2.0 ** -t
            Ja, tha = oracle.srbd_merit(prm, r32(pr["x0hat"]), x + a * dx[sl].astype(np.float64),
                                        u + a * du[sl].astype(np.float64), *args)
            dJ = Ja - J0
            assert abs(mer[i, 3 + t] - dJ) <= 1e-4 * abs(dJ) + 1e-6 * abs(J0), (t, mer[i, 3 + t], dJ)
            assert abs(mer[i, 13 + t] - tha) <= 1e-4 * tha + 2e-5, (t, mer[i, 13 + t], tha)
        assert mer[i, 23] == pytest.approx(max(np.abs(dx[sl]).max(), np.abs(du[o:o + N]).max()))


def srbd_case(count, seed, Ns):
    insts, packed, Nv, off, x0 = [], None, None, None, None
    insts = [synth.srbd_problem(Ns[i % len(Ns)], seed=seed + i) for i in range(count)]
    packed, Nv, off = synth.pack(insts, synth.SRBD_KEYS)
    x0 = np.stack([p["x0hat"] for p in insts])
    return insts, packed, Nv, off, x0


def run_oracle(prm, pr, iters, alpha_replay=None):
    return oracle.srbd_sqp(prm, r32(pr["x0hat"]), r32(pr["x"]), r32(pr["u"]), r32(pr["lam"]),
                           r32(pr["xref"]), r32(pr["uref"]), pr["contact"], max_iters=iters,
                           alpha_replay=alpha_replay)


@pytest.mark.parametrize("warps", [1, 4, 8, 16])
@pytest.mark.parametrize("mode", ["replay", "free"])
def test_sqp_parity(warps, mode):
    """Fused SQP against the oracle; warps = 1 is the sequential recursion
    with two instances per warp (here pairs of unequal horizons share one)."""
    from paper_2506_07823_b300 import pdilqr
    iters = 10
    insts, packed, Nv, off, x0 = srbd_case(4, 11, [25, 50, 75, 100])
    prm = synth.srbd_params()
    refs = [run_oracle(prm, pr, iters) for pr in insts]
    d = dev(packed)
    plan = pdilqr.Plan(12, 12, Nv, off, warps=warps)
    replay = None
    if mode == "replay":
        replay = torch.tensor(np.stack([r[3]["alpha"] for r in refs]).astype(np.float32), device="cuda")
    info = plan.solve(pdilqr.srbd_model(prm), torch.tensor(x0, dtype=torch.float32, device="cuda"),
                      d["x"], d["u"], d["lam"], d["xref"], d["uref"], d["contact"],
                      max_iters=iters, alpha_replay=replay)
    torch.cuda.synchronize()
    st = info["status"].cpu().numpy()
    assert np.all(st == 0), st
    its = info["iters"].cpu().numpy()
    if mode == "replay":
        assert np.all(its == iters)
    else:
        # free-running, the FP32 iterate may stop early at its precision floor
        assert np.all((its >= 6) & (its <= iters)), its
    xs, us, ls = (d[k].double().cpu().numpy() for k in ("x", "u", "lam"))
    al = info["alpha"].cpu().numpy()
    for i, (xr, ur, lr, inf) in enumerate(refs):
        N, o = int(Nv[i]), int(off[i])
        sl = slice(o, o + N + 1)
        if mode == "replay":
            assert np.array_equal(al[i], inf["alpha"].astype(np.float32))
        else:
            # Step sizes must agree while the iterate's constraint violation is
            # well above the FP32 storage floor of the states (~1e-6 summed
            # over the horizon); below it the FP32 and FP64 filter tests may
            # legitimately differ (the final iterate is still compared).
            big = (inf["theta_it"] > 1e-4)[:its[i]]
            assert np.array_equal(al[i][:its[i]][big], inf["alpha"][:its[i]][big].astype(np.float32)), (al[i], inf)
        assert rel(xs[sl], xr) <= REL_TOL, rel(xs[sl], xr)
        assert rel(us[o:o + N], ur[:N]) <= REL_TOL, rel(us[o:o + N], ur[:N])
        assert rel(ls[sl], lr) <= REL_TOL, rel(ls[sl], lr)
        J, th = info["J"][i].item(), info["theta"][i].item()
        assert abs(J - inf["J"]) <= 1e-4 * abs(inf["J"])
        assert th <= 1e-3


def test_sqp_stops_on_tolerance():
    from paper_2506_07823_b300 import pdilqr
    insts, packed, Nv, off, x0 = srbd_case(2, 3, [30])
    prm = synth.srbd_params()
    d = dev(packed)
    plan = pdilqr.Plan(12, 12, Nv, off)
    info = plan.solve(pdilqr.srbd_model(prm), torch.tensor(x0, dtype=torch.float32, device="cuda"),
                      d["x"], d["u"], d["lam"], d["xref"], d["uref"], d["contact"],
                      max_iters=30, tol_step=1e-2, tol_theta=1e-2)
    torch.cuda.synchronize()
    it = info["iters"].cpu().numpy()
    assert np.all(it < 30) and np.all(it >= 2), it
    assert np.all(info["status"].cpu().numpy() == 0)


@pytest.mark.parametrize("warps", [1, 4])
@pytest.mark.parametrize("nrob", [2, 4, 8, 16])
def test_sqp_parity_multi_robot(nrob, warps):
    """Centralised multi-robot problems (n = m = 12 nrob, ring formation cost)
    through the fused SQP, replaying the oracle's step sizes; nrob >= 8 runs
    its work areas from the global workspace."""
    from paper_2506_07823_b300 import pdilqr
    if nrob >= 8 and warps != 1:
        pytest.skip("sizes beyond shared memory are served with one chunk")
    n = 12 * nrob
    Ns, iters = ([4, 7], 2) if nrob == 16 else ([6, 13], 3)
    insts = [synth.srbd_problem(Ns[i], seed=500 + 10 * nrob + i, nrob=nrob) for i in range(2)]
    packed, Nv, off = synth.pack(insts, synth.SRBD_KEYS)
    x0 = np.stack([p["x0hat"] for p in insts])
    prm = synth.srbd_params(nrob)
    refs = [run_oracle(prm, pr, iters) for pr in insts]
    d = dev(packed)
    plan = pdilqr.Plan(n, n, Nv, off, warps=warps)
    replay = torch.tensor(np.stack([r[3]["alpha"] for r in refs]).astype(np.float32), device="cuda")
    info = plan.solve(pdilqr.srbd_model(prm), torch.tensor(x0, dtype=torch.float32, device="cuda"),
                      d["x"], d["u"], d["lam"], d["xref"], d["uref"], d["contact"],
                      max_iters=iters, alpha_replay=replay)
    torch.cuda.synchronize()
    assert np.all(info["status"].cpu().numpy() == 0)
    assert np.all(info["iters"].cpu().numpy() == iters)
    xs, us, ls = (d[k].double().cpu().numpy() for k in ("x", "u", "lam"))
    for i, (xr, ur, lr, inf) in enumerate(refs):
        N, o = int(Nv[i]), int(off[i])
        sl = slice(o, o + N + 1)
        assert rel(xs[sl], xr) <= REL_TOL, rel(xs[sl], xr)
        assert rel(us[o:o + N], ur[:N]) <= REL_TOL, rel(us[o:o + N], ur[:N])
        assert rel(ls[sl], lr) <= REL_TOL, rel(ls[sl], lr)
        assert abs(info["J"][i].item() - inf["J"]) <= 1e-4 * abs(inf["J"])


@pytest.mark.parametrize("mode", ["replay", "free"])
def test_sqp_parity_long_horizon(mode):
    """The horizon sweep's longest problems (N = 150 and 200, one robot) through
    the 16-chunk fused SQP, 10 iterations."""
    from paper_2506_07823_b300 import pdilqr
    iters = 10
    insts, packed, Nv, off, x0 = srbd_case(2, 61, [150, 200])
    prm = synth.srbd_params()
    refs = [run_oracle(prm, pr, iters) for pr in insts]
    d = dev(packed)
    plan = pdilqr.Plan(12, 12, Nv, off, warps=16)
    replay = None
    if mode == "replay":
        replay = torch.tensor(np.stack([r[3]["alpha"] for r in refs]).astype(np.float32), device="cuda")
    info = plan.solve(pdilqr.srbd_model(prm), torch.tensor(x0, dtype=torch.float32, device="cuda"),
                      d["x"], d["u"], d["lam"], d["xref"], d["uref"], d["contact"],
                      max_iters=iters, alpha_replay=replay)
    torch.cuda.synchronize()
    assert np.all(info["status"].cpu().numpy() == 0)
    xs, us, ls = (d[k].double().cpu().numpy() for k in ("x", "u", "lam"))
    for i, (xr, ur, lr, inf) in enumerate(refs):
        N, o = int(Nv[i]), int(off[i])
        sl = slice(o, o + N + 1)
        assert rel(xs[sl], xr) <= REL_TOL, rel(xs[sl], xr)
        assert rel(us[o:o + N], ur[:N]) <= REL_TOL, rel(us[o:o + N], ur[:N])
        assert rel(ls[sl], lr) <= REL_TOL, rel(ls[sl], lr)


@pytest.mark.parametrize("warps", [1, 4])
@pytest.mark.parametrize("nrob", [8, 16])
def test_sqp_parity_multi_robot_horizon50(nrob, warps):
    """Centralised 8- and 16-robot problems at the serving horizon N = 50:
    the one-chunk recursion (tensor-core products) and the 4-chunk scan from
    the global workspace, replaying the oracle's step sizes."""
    from paper_2506_07823_b300 import pdilqr
    n = 12 * nrob
    iters = 2
    pr = synth.srbd_problem(50, seed=700 + nrob, nrob=nrob)
    packed, Nv, off = synth.pack([pr], synth.SRBD_KEYS)
    prm = synth.srbd_params(nrob)
    xr, ur, lr, inf = run_oracle(prm, pr, iters)
    d = dev(packed)
    plan = pdilqr.Plan(n, n, Nv, off, warps=warps)
    replay = torch.tensor(inf["alpha"][None].astype(np.float32), device="cuda")
    info = plan.solve(pdilqr.srbd_model(prm),
                      torch.tensor(pr["x0hat"][None], dtype=torch.float32, device="cuda"),
                      d["x"], d["u"], d["lam"], d["xref"], d["uref"], d["contact"],
                      max_iters=iters, alpha_replay=replay)
    torch.cuda.synchronize()
    assert info["status"].item() == 0
    assert info["iters"].item() == iters
    xs, us, ls = (d[k].double().cpu().numpy() for k in ("x", "u", "lam"))
    assert rel(xs, xr) <= REL_TOL, rel(xs, xr)
    assert rel(us[:50], ur[:50]) <= REL_TOL, rel(us[:50], ur[:50])
    assert rel(ls, lr) <= REL_TOL, rel(ls, lr)


def test_tensor_core_wait_timeout_status():
    """The bounded wait of the tensor-core products: with the test switch that
    issues no MMA (so nothing ever signals the barrier) the instance ends with
    E_TIMEOUT instead of hanging; the context stays usable and the next solve
    of the same plan is correct."""
    from paper_2506_07823_b300 import pdilqr
    nrob, iters = 8, 1
    pr = synth.srbd_problem(3, seed=77, nrob=nrob)
    packed, Nv, off = synth.pack([pr], synth.SRBD_KEYS)
    prm = synth.srbd_params(nrob)
    x0 = torch.tensor(pr["x0hat"][None], dtype=torch.float32, device="cuda")
    plan = pdilqr.Plan(96, 96, Nv, off, warps=1)
    d = dev(packed)
    plan.set_debug(pdilqr.DEBUG_TC_SKIP_ISSUE)
    info = plan.solve(pdilqr.srbd_model(prm), x0, d["x"], d["u"], d["lam"], d["xref"],
                      d["uref"], d["contact"], max_iters=iters)
    torch.cuda.synchronize()
    assert info["status"].item() == pdilqr.E_TIMEOUT
    plan.set_debug(0)
    xr, ur, lr, inf = run_oracle(prm, pr, iters)
    d = dev(packed)
    replay = torch.tensor(inf["alpha"][None].astype(np.float32), device="cuda")
    info = plan.solve(pdilqr.srbd_model(prm), x0, d["x"], d["u"], d["lam"], d["xref"],
                      d["uref"], d["contact"], max_iters=iters, alpha_replay=replay)
    torch.cuda.synchronize()
    assert info["status"].item() == 0
    assert rel(d["x"].double().cpu().numpy(), xr) <= REL_TOL


@pytest.mark.parametrize("ipc", [2, 4, 8])
def test_sqp_sequential_odd_batch(ipc):
    """The two-instances-per-warp sequential solver on an odd batch (the last
    warp runs one instance; at 4 and 8 instances per CTA whole warps of the
    last CTA run none) with horizons 1 (degenerate) to 100, replaying the
    oracle's step sizes."""
    from paper_2506_07823_b300 import pdilqr
    iters = 4
    insts, packed, Nv, off, x0 = srbd_case(5, 91, [1, 100, 13, 2, 50])
    prm = synth.srbd_params()
    refs = [run_oracle(prm, pr, iters) for pr in insts]
    d = dev(packed)
    plan = pdilqr.Plan(12, 12, Nv, off, warps=1, inst_per_cta=ipc)
    replay = torch.tensor(np.stack([r[3]["alpha"] for r in refs]).astype(np.float32), device="cuda")
    info = plan.solve(pdilqr.srbd_model(prm), torch.tensor(x0, dtype=torch.float32, device="cuda"),
                      d["x"], d["u"], d["lam"], d["xref"], d["uref"], d["contact"],
                      max_iters=iters, alpha_replay=replay)
    torch.cuda.synchronize()
    st = info["status"].cpu().numpy()
    want = np.array([pdilqr.E_LINESEARCH if r[3]["status"] == 1 else 0 for r in refs])
    assert np.array_equal(st, want), (st, want)
    xs, us, ls = (d[k].double().cpu().numpy() for k in ("x", "u", "lam"))
    for i, (xr, ur, lr, inf) in enumerate(refs):
        if inf["status"] != 0:
            continue
        N, o = int(Nv[i]), int(off[i])
        sl = slice(o, o + N + 1)
        assert rel(xs[sl], xr) <= REL_TOL, (i, rel(xs[sl], xr))
        assert rel(us[o:o + N], ur[:N]) <= REL_TOL, (i, rel(us[o:o + N], ur[:N]))
        assert rel(ls[sl], lr) <= REL_TOL, (i, rel(ls[sl], lr))


def test_captured_solve_replays_like_a_direct_solve():
    """The plan's own CUDA graph (pdilqr_solve_capture / pdilqr_plan_replay)
    reproduces a direct solve bit for bit, replay after replay, for both the
    sequential and the scan solver."""
    from paper_2506_07823_b300 import pdilqr
    insts, packed, Nv, off, x0 = srbd_case(5, 31, [25, 50, 75, 100, 3])
    prm = synth.srbd_params()
    md = pdilqr.srbd_model(prm)
    x0d = torch.tensor(x0, dtype=torch.float32, device="cuda")
    for warps in (1, 8):
        ref = dev(packed)
        plan = pdilqr.Plan(12, 12, Nv, off, warps=warps)
        want = plan.solve(md, x0d, ref["x"], ref["u"], ref["lam"], ref["xref"], ref["uref"],
                          ref["contact"], max_iters=4)
        torch.cuda.synchronize()
        d = dev(packed)
        base = {k: v.clone() for k, v in d.items()}
        info = plan.capture(md, x0d, d["x"], d["u"], d["lam"], d["xref"], d["uref"], d["contact"],
                            max_iters=4)
        torch.cuda.synchronize()
        assert torch.equal(d["x"], base["x"])          # the capture ran nothing
        for _ in range(2):
            for k in ("x", "u", "lam"):
                d[k].copy_(base[k])
            plan.replay()
            torch.cuda.synchronize()
            for k in ("x", "u", "lam"):
                assert torch.equal(d[k], ref[k]), (warps, k)
            assert torch.equal(info["status"], want["status"])
            assert torch.equal(info["iters"], want["iters"])


def test_instances_per_cta_same_result():
    """Packing 2, 4 or 8 instances into a CTA changes only which CTA runs an
    instance: every instance's iterate is bit-identical across the three."""
    from paper_2506_07823_b300 import pdilqr
    insts, packed, Nv, off, x0 = srbd_case(11, 7, [25, 50, 75, 100])
    md = pdilqr.srbd_model(synth.srbd_params())
    x0d = torch.tensor(x0, dtype=torch.float32, device="cuda")
    outs = []
    for ipc in (2, 4, 8):
        d = dev(packed)
        plan = pdilqr.Plan(12, 12, Nv, off, warps=1, inst_per_cta=ipc)
        info = plan.solve(md, x0d, d["x"], d["u"], d["lam"], d["xref"], d["uref"], d["contact"],
                          max_iters=3)
        torch.cuda.synchronize()
        outs.append((d["x"].clone(), d["u"].clone(), d["lam"].clone(), info["status"].clone()))
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert torch.equal(a, b)


def test_instances_per_cta_rejected_elsewhere():
    """Only the one-robot sequential solver packs several instances per CTA;
    other solvers, sizes and counts are invalid arguments."""
    from paper_2506_07823_b300 import pdilqr
    for n, warps, ipc in ((12, 4, 4), (12, 1, 3), (12, 1, 16), (24, 1, 2)):
        with pytest.raises(pdilqr.PdilqrError) as e:
            pdilqr.Plan(n, n, [10, 20], [0, 11], warps=warps, inst_per_cta=ipc)
        assert e.value.code == pdilqr.E_INVALID_ARG


def test_autotune_picks_a_timed_configuration():
    """The batch autotuner times every configuration of a one-robot batch
    and returns the plan of the fastest; its solve matches a plain plan's."""
    from paper_2506_07823_b300 import autotune, pdilqr
    insts, packed, Nv, off, x0 = srbd_case(16, 3, [25, 50, 75, 100])
    md = pdilqr.srbd_model(synth.srbd_params())
    x0d = torch.tensor(x0, dtype=torch.float32, device="cuda")
    d = dev(packed)
    base = {k: v.clone() for k, v in d.items()}

    def reset():
        for k in ("x", "u", "lam"):
            d[k].copy_(base[k])

    def solve(p):
        return p.solve(md, x0d, d["x"], d["u"], d["lam"], d["xref"], d["uref"], d["contact"],
                       max_iters=2)
    plan, times = autotune.autotune_sqp(torch, 12, 12, Nv, off, solve, reset=reset, reps=1)
    assert set(times) == {autotune.label(w, i) for w, i in autotune.candidates(12, 12)}
    assert autotune.label(plan.warps, plan.inst_per_cta) == min(times, key=times.get)
    reset()
    solve(plan)
    torch.cuda.synchronize()
    got = d["x"].clone()
    reset()
    solve(pdilqr.Plan(12, 12, Nv, off, warps=plan.warps))
    torch.cuda.synchronize()
    assert rel(got.double().cpu().numpy(), d["x"].double().cpu().numpy()) <= REL_TOL


@pytest.mark.parametrize("nrob,Ns,iters", [(4, [50], 2), (4, [13, 37], 3), (8, [50], 2), (16, [50], 2)])
def test_split_sqp_parity(nrob, Ns, iters):
    """The SQP of a split plan (the scan's 16 chunks on 16 CTAs; each iteration
    unfused: linearisation into the plan's LQ arrays, split scan, merit /
    filter / update kernel), replaying the oracle's step sizes."""
    from paper_2506_07823_b300 import pdilqr
    n = 12 * nrob
    insts = [synth.srbd_problem(N, seed=900 + 10 * nrob + i, nrob=nrob) for i, N in enumerate(Ns)]
    packed, Nv, off = synth.pack(insts, synth.SRBD_KEYS)
    x0 = np.stack([p["x0hat"] for p in insts])
    prm = synth.srbd_params(nrob)
    refs = [run_oracle(prm, pr, iters) for pr in insts]
    d = dev(packed)
    plan = pdilqr.Plan(n, n, Nv, off, warps=16, split=True)
    replay = torch.tensor(np.stack([r[3]["alpha"] for r in refs]).astype(np.float32), device="cuda")
    info = plan.solve(pdilqr.srbd_model(prm), torch.tensor(x0, dtype=torch.float32, device="cuda"),
                      d["x"], d["u"], d["lam"], d["xref"], d["uref"], d["contact"],
                      max_iters=iters, alpha_replay=replay)
    torch.cuda.synchronize()
    assert np.all(info["status"].cpu().numpy() == 0), info["status"]
    assert np.all(info["iters"].cpu().numpy() == iters), info["iters"]
    np.testing.assert_array_equal(info["alpha"].cpu().numpy(), replay.cpu().numpy())
    xs, us, ls = (d[k].double().cpu().numpy() for k in ("x", "u", "lam"))
    for i, (xr, ur, lr, inf) in enumerate(refs):
        N, o = int(Nv[i]), int(off[i])
        sl = slice(o, o + N + 1)
        assert rel(xs[sl], xr) <= REL_TOL, (i, rel(xs[sl], xr))
        assert rel(us[o:o + N], ur[:N]) <= REL_TOL, (i, rel(us[o:o + N], ur[:N]))
        assert rel(ls[sl], lr) <= REL_TOL, (i, rel(ls[sl], lr))
        assert abs(info["J"][i].item() - inf["J"]) <= 1e-4 * abs(inf["J"])
    from paper_2506_07823_b300.pdilqr import PdilqrError
    with pytest.raises(PdilqrError):
        plan.capture(pdilqr.srbd_model(prm), torch.tensor(x0, dtype=torch.float32, device="cuda"),
                     d["x"], d["u"], d["lam"], d["xref"], d["uref"], d["contact"], max_iters=iters)
