"""Pins for the FP64 CPU oracle (CPU only).

Each test checks the oracle against something other than itself: the dense
KKT system of the QP solved by LU, the sensitivity of the optimal value,
the scalar discrete Riccati closed form, brute-force minimisation of the
CVF combine, finite differences of the SRBD model, hand-derived barrier
values and one-step convergence of the SQP on a linear model.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2506_07823_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")


def rand_lq(n, m, N, seed, with_S=True):
    """Random convex LQ data (PD stage Hessians, nonzero S)."""
    g = np.random.default_rng(seed)
    A = g.normal(0, 0.5, (N + 1, n, n)) + np.eye(n)
    B = g.normal(0, 0.5, (N + 1, n, m))
    c = g.normal(0, 0.3, (N + 1, n))
    Q = np.zeros((N + 1, n, n))
    R = np.zeros((N + 1, m, m))
    S = np.zeros((N + 1, m, n))
    for k in range(N + 1):
        L = g.normal(0, 0.5, (n + m, n + m))
        H = L @ L.T + 0.3 * np.eye(n + m)
        Q[k] = H[:n, :n]
        R[k] = H[n:, n:]
        if with_S:
            S[k] = H[n:, :n]
    q = g.normal(0, 1, (N + 1, n))
    r = g.normal(0, 1, (N + 1, m))
    s = g.normal(0, 1, n)
    return {"A": A, "B": B, "c": c, "Q": Q, "R": R, "S": S, "q": q, "r": r}, s


def dense_qp(lq, s):
    """Assemble the QP of Eq. (QP) as  min 1/2 z'Hz + g'z  s.t.  E z = e,
    z = (dx_0..dx_N, du_0..du_{N-1}), with the constraints oriented as in the
    Lagrangian of Sec. II-B (lam_0 (s - dx_0), lam_{k+1}(A dx + B du + c - dx'))."""
    A, B = lq["A"], lq["B"]
    N = A.shape[0] - 1
    n, m = A.shape[1], B.shape[2]
    nz = (N + 1) * n + N * m
    ix = lambda k: slice(k * n, (k + 1) * n)
    iu = lambda k: slice((N + 1) * n + k * m, (N + 1) * n + (k + 1) * m)
    H = np.zeros((nz, nz))
    g = np.zeros(nz)
    for k in range(N):
        H[ix(k), ix(k)] = lq["Q"][k]
        H[iu(k), iu(k)] = lq["R"][k]
        H[iu(k), ix(k)] = lq["S"][k]
        H[ix(k), iu(k)] = lq["S"][k].T
        g[ix(k)] = lq["q"][k]
        g[iu(k)] = lq["r"][k]
    H[ix(N), ix(N)] = lq["Q"][N]
    g[ix(N)] = lq["q"][N]
    E = np.zeros(((N + 1) * n, nz))
    e = np.zeros((N + 1) * n)
    E[0:n, ix(0)] = -np.eye(n)          # s - dx_0 = 0
    e[0:n] = -s
    for k in range(N):
        rows = slice((k + 1) * n, (k + 2) * n)
        E[rows, ix(k)] = A[k]
        E[rows, iu(k)] = B[k]
        E[rows, ix(k + 1)] = -np.eye(n)
        e[rows] = -lq["c"][k]
    return H, g, E, e


def dense_solve(lq, s):
    H, g, E, e = dense_qp(lq, s)
    nz, nc = H.shape[0], E.shape[0]
    K = np.block([[H, E.T], [E, np.zeros((nc, nc))]])
    sol = np.linalg.solve(K, np.concatenate([-g, e]))
    return sol[:nz], sol[nz:], (H, g, E, e)


def split(lq, z, nu):
    A, B = lq["A"], lq["B"]
    N = A.shape[0] - 1
    n, m = A.shape[1], B.shape[2]
    dx = z[:(N + 1) * n].reshape(N + 1, n)
    du = z[(N + 1) * n:].reshape(N, m)
    lam = nu.reshape(N + 1, n)
    return dx, du, lam


@pytest.mark.parametrize("n,m,N", [(1, 1, 1), (2, 1, 2), (3, 2, 5), (4, 2, 8), (4, 3, 1)])
@pytest.mark.parametrize("with_S", [False, True])
def test_riccati_matches_dense_kkt(n, m, N, with_S):
    lq, s = rand_lq(n, m, N, seed=10 * n + N + with_S, with_S=with_S)
    ref = oracle.riccati_solve(lq, s)
    z, nu, _ = dense_solve(lq, s)
    dx, du, lam = split(lq, z, nu)
    np.testing.assert_allclose(ref["dx"], dx, rtol=0, atol=1e-10 * max(1, np.abs(dx).max()))
    np.testing.assert_allclose(ref["du"][:N], du, rtol=0, atol=1e-10 * max(1, np.abs(du).max()))
    np.testing.assert_allclose(ref["dlam"], lam, rtol=0, atol=1e-10 * max(1, np.abs(lam).max()))
    assert np.all(ref["du"][N] == 0.0)


def test_multipliers_are_value_sensitivities():
    """lam_0 = dV*/ds and lam_{k+1} = dV*/dc_k (V* the optimal QP value)."""
    lq, s = rand_lq(3, 2, 4, seed=7)
    H, g, _, _ = dense_qp(lq, s)

    def value(lq_, s_):
        out = oracle.riccati_solve(lq_, s_)
        N = lq_["A"].shape[0] - 1
        z = np.concatenate([out["dx"].ravel(), out["du"][:N].ravel()])
        return 0.5 * z @ H @ z + g @ z

    ref = oracle.riccati_solve(lq, s)
    h = 1e-5
    for i in range(3):
        sp, sm = s.copy(), s.copy()
        sp[i] += h
        sm[i] -= h
        fd = (value(lq, sp) - value(lq, sm)) / (2 * h)
        assert abs(fd - ref["dlam"][0, i]) < 1e-7 * max(1, abs(fd))
    for k in range(4):
        for i in range(3):
            lp = {kk: v.copy() for kk, v in lq.items()}
            lm = {kk: v.copy() for kk, v in lq.items()}
            lp["c"][k, i] += h
            lm["c"][k, i] -= h
            fd = (value(lp, s) - value(lm, s)) / (2 * h)
            assert abs(fd - ref["dlam"][k + 1, i]) < 1e-7 * max(1, abs(fd))


def test_kkt_residual_against_dense():
    lq, s = rand_lq(4, 2, 6, seed=3)
    ref = oracle.riccati_solve(lq, s)
    res, kn, zn, rn = oracle.kkt_residual(lq, s, ref["dx"], ref["du"], ref["dlam"])
    assert res / (kn * zn + rn) < 1e-13
    # perturb one component: the oracle's residual must equal the dense one
    z, nu, (H, g, E, e) = dense_solve(lq, s)
    dx = ref["dx"].copy()
    dx[3, 1] += 1e-3
    res2 = oracle.kkt_residual(lq, s, dx, ref["du"], ref["dlam"])[0]
    N = 6
    zz = np.concatenate([dx.ravel(), ref["du"][:N].ravel()])
    nz, nc = H.shape[0], E.shape[0]
    Kd = np.block([[H, E.T], [E, np.zeros((nc, nc))]])
    dense_res = np.abs(Kd @ np.concatenate([zz, ref["dlam"].ravel()]) - np.concatenate([-g, e])).max()
    assert abs(res2 - dense_res) < 1e-12
    assert kn == pytest.approx(np.abs(Kd).sum(axis=1).max(), rel=1e-12)


def test_scalar_dare_closed_form():
    gold = json.load(open(GOLDEN))["scalar_dare"]["cases"]
    for case in gold:
        a, b, q, r = case["a"], case["b"], case["q"], case["r"]
        N = 300
        lq = {"A": np.full((N + 1, 1, 1), a), "B": np.full((N + 1, 1, 1), b),
              "c": np.zeros((N + 1, 1)), "Q": np.full((N + 1, 1, 1), q),
              "R": np.full((N + 1, 1, 1), r), "S": np.zeros((N + 1, 1, 1)),
              "q": np.zeros((N + 1, 1)), "r": np.zeros((N + 1, 1))}
        lq["Q"][N] = q
        out = oracle.riccati_solve(lq, np.ones(1))
        assert abs(out["P"][0, 0, 0] - case["P"]) < 1e-12 * case["P"]
        # the closed form of the scalar DARE
        t = r * (1 - a * a) - q * b * b
        closed = (-t + np.sqrt(t * t + 4 * b * b * q * r)) / (2 * b * b)
        assert abs(out["P"][0, 0, 0] - closed) < 1e-12 * closed


# ------------------------------------------------ CVF scan (test-only code)
def cvf_element(A, B, c, Q, R, S, q, r):
    """Element V_{i->i+1} of the reverse scan (Sec. II-D initialisation)."""
    Ri = np.linalg.inv(R)
    return (A - B @ Ri @ S, c - B @ Ri @ r, B @ Ri @ B.T, q - S.T @ Ri @ r, Q - S.T @ Ri @ S)


def cvf_combine(e1, e2):
    """V_{i->k} (x) V_{k->j} with the combination rule of Sec. II-D, typos
    corrected: A = A2 M^-1 A1, b = A2 M^-1 (b1 - C1 p2) + b2,
    C = A2 M^-1 C1 A2' + C2, P = (M^-1 A1)' P2 A1 + P1,
    p = (M^-1 A1)' (p2 + P2 b1) + p1, M = I + C1 P2."""
    A1, b1, C1, p1, P1 = e1
    A2, b2, C2, p2, P2 = e2
    n = A1.shape[0]
    Mi = np.linalg.inv(np.eye(n) + C1 @ P2)
    X = Mi @ A1
    return (A2 @ X, A2 @ Mi @ (b1 - C1 @ p2) + b2, A2 @ Mi @ C1 @ A2.T + C2,
            X.T @ (p2 + P2 @ b1) + p1, X.T @ P2 @ A1 + P1)


def cvf_eval(e, xi, xj):
    """V(x_i, x_j) of Eq. (cvf) for invertible C (the max over eta in closed form)."""
    A, b, C, p, P = e
    d = xj - A @ xi - b
    return 0.5 * xi @ P @ xi + p @ xi + 0.5 * d @ np.linalg.solve(C, d)


def rand_element(n, g, c_pd=True):
    A = g.normal(0, 0.6, (n, n))
    b = g.normal(0, 1, n)
    L = g.normal(0, 0.6, (n, n))
    C = L @ L.T + (0.2 * np.eye(n) if c_pd else 0)
    L2 = g.normal(0, 0.6, (n, n))
    P = L2 @ L2.T + 0.1 * np.eye(n)
    p = g.normal(0, 1, n)
    return (A, b, C, p, P)


def test_cvf_combine_brute_force():
    """The combine equals min over x_k of V_{i->k} + V_{k->j} (Eq. otimes),
    up to the additive constant that the five-tuple of Eq. (cvf) drops."""
    g = np.random.default_rng(5)
    for trial in range(5):
        n = 3
        e1, e2 = rand_element(n, g), rand_element(n, g)
        e12 = cvf_combine(e1, e2)

        def brute(xi, xj):
            # the sum is a convex quadratic in x_k: minimise it exactly
            A1, b1, C1, _, _ = e1
            A2, b2, C2, p2, P2 = e2
            C1i, C2i = np.linalg.inv(C1), np.linalg.inv(C2)
            Hk = C1i + P2 + A2.T @ C2i @ A2
            gk = -C1i @ (A1 @ xi + b1) + p2 - A2.T @ C2i @ (xj - b2)
            xk = np.linalg.solve(Hk, -gk)
            return cvf_eval(e1, xi, xk) + cvf_eval(e2, xk, xj)

        z = np.zeros(n)
        const = brute(z, z) - cvf_eval(e12, z, z)
        for _ in range(6):
            xi, xj = g.normal(0, 1, n), g.normal(0, 1, n)
            b = brute(xi, xj)
            assert abs(cvf_eval(e12, xi, xj) + const - b) < 1e-9 * max(1, abs(b))


def test_cvf_associative():
    g = np.random.default_rng(11)
    for _ in range(5):
        e1, e2, e3 = (rand_element(4, g) for _ in range(3))
        left = cvf_combine(cvf_combine(e1, e2), e3)
        right = cvf_combine(e1, cvf_combine(e2, e3))
        for a, b in zip(left, right):
            assert np.abs(a - b).max() < 1e-10 * max(1, np.abs(a).max())


def test_cvf_deterministic_first_segment():
    """C1 = 0 pins x_k = A1 x_i + b1: the combine reduces to composition."""
    g = np.random.default_rng(2)
    e1 = list(rand_element(3, g))
    e1[2] = np.zeros((3, 3))
    e2 = rand_element(3, g)
    A1, b1, _, p1, P1 = e1
    A2, b2, C2, p2, P2 = e2
    got = cvf_combine(tuple(e1), e2)
    want = (A2 @ A1, A2 @ b1 + b2, C2, A1.T @ (p2 + P2 @ b1) + p1, A1.T @ P2 @ A1 + P1)
    for a, b in zip(got, want):
        assert np.abs(a - b).max() < 1e-12 * max(1, np.abs(b).max())


@pytest.mark.parametrize("with_S", [False, True])
def test_reverse_scan_fold_equals_riccati(with_S):
    """Suffix products e_k x ... x e_N hold (P_k, p_k) of Eq. (lqr), with
    A = b = C = 0 exactly; the trajectory scan reproduces the rollout."""
    n, m, N = 4, 2, 9
    lq, s = rand_lq(n, m, N, seed=21, with_S=with_S)
    ref = oracle.riccati_solve(lq, s)
    elems = [cvf_element(*(lq[k][i] for k in ("A", "B", "c", "Q", "R", "S", "q", "r")))
             for i in range(N)]
    elems.append((np.zeros((n, n)), np.zeros(n), np.zeros((n, n)), lq["q"][N], lq["Q"][N]))
    suffix = elems[N]
    for k in range(N, -1, -1):
        if k < N:
            suffix = cvf_combine(elems[k], suffix)
        A, b, C, p, P = suffix
        assert np.all(A == 0) and np.all(b == 0) and np.all(C == 0)
        assert np.abs(P - ref["P"][k]).max() < 1e-10 * np.abs(ref["P"][k]).max()
        assert np.abs(p - ref["p"][k]).max() < 1e-10 * max(1, np.abs(ref["p"][k]).max())
    # affine trajectory elements: (Abar_k, bbar_k), composed in order
    x = s.copy()
    for k in range(N):
        Abar = lq["A"][k] + lq["B"][k] @ ref["K"][k]
        bbar = lq["B"][k] @ ref["k"][k] + lq["c"][k]
        x = Abar @ x + bbar
        assert np.abs(x - ref["dx"][k + 1]).max() < 1e-10 * max(1, np.abs(x).max())


# ----------------------------------------------------------------- barrier
def test_barrier_golden_and_c2():
    gold = json.load(open(GOLDEN))["barrier"]["cases"]
    for case in gold:
        v = oracle.barrier(case["xi"], case["mu"], case["delta"])
        np.testing.assert_allclose(v, [case["value"], case["d1"], case["d2"]], rtol=1e-13, atol=1e-15)
    mu, d = 0.3, 0.7
    lo = oracle.barrier(d * (1 - 1e-12), mu, d)
    hi = oracle.barrier(d, mu, d)
    np.testing.assert_allclose(lo, hi, rtol=1e-9)
    for xi in (-0.4, 0.3, 1.5, 4.0):
        h = 1e-6
        v = oracle.barrier(xi, mu, d)
        vp, vm = oracle.barrier(xi + h, mu, d), oracle.barrier(xi - h, mu, d)
        assert abs((vp[0] - vm[0]) / (2 * h) - v[1]) < 1e-7
        assert abs((vp[1] - vm[1]) / (2 * h) - v[2]) < 1e-6


# ------------------------------------------- SRBD cost and merit assembly
SRBD_GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "srbd_cost_merit.json")


def _golden_params(gold, case):
    """Model constants of a golden case: its own, or another case's with overrides."""
    c = gold[case]
    base = dict(gold[c.get("params_from", case)]["params"])
    base.update(c.get("overrides", {}))
    return {k: (np.asarray(v, dtype=np.float64) if isinstance(v, list) else v)
            for k, v in base.items()}


def test_srbd_stage_cost_golden():
    """Stage and terminal cost of one robot against hand arithmetic: tracking,
    control, the five pyramid rows of two stance feet on both barrier
    branches, and a swing foot that contributes no barrier."""
    gold = json.load(open(SRBD_GOLDEN))
    c = gold["stage_cost_one_robot"]
    p = _golden_params(gold, "stage_cost_one_robot")
    ct = np.asarray(c["contact"], dtype=np.uint8)
    J = oracle.srbd_cost(p, c["x"], c["u"], ct, c["xref"], c["uref"], False)
    assert J == pytest.approx(c["stage"], rel=1e-13, abs=1e-15)
    Jt = oracle.srbd_cost(p, c["x"], None, None, c["xref"], None, True)
    assert Jt == pytest.approx(c["terminal"], rel=1e-13, abs=1e-15)


@pytest.mark.parametrize("case", ["formation_two_robots", "formation_four_robots"])
def test_srbd_formation_cost_golden(case):
    """Ring formation term against hand arithmetic (sign and owner of each
    offset d_a, wrap-around of the ring)."""
    gold = json.load(open(SRBD_GOLDEN))
    c = gold[case]
    p = _golden_params(gold, case)
    R = p["nrob"]
    x = np.zeros(12 * R)
    for a, pos in enumerate(c["positions"]):
        x[12 * a:12 * a + 3] = pos
    u = np.zeros(12 * R)
    ct = np.zeros(4 * R, dtype=np.uint8)
    J = oracle.srbd_cost(p, x, u, ct, x, u, False)
    assert J == pytest.approx(c["stage"], rel=1e-13, abs=1e-15)
    Jt = oracle.srbd_cost(p, x, None, None, x, None, True)
    assert Jt == pytest.approx(c["terminal"], rel=1e-13, abs=1e-15)


def test_srbd_merit_golden():
    """J and theta of a two-interval trajectory against hand arithmetic,
    including the initial-state term |xhat_0 - x_0|."""
    gold = json.load(open(SRBD_GOLDEN))
    c = gold["merit_free_fall"]
    p = _golden_params(gold, "merit_free_fall")
    N = c["N"]
    x = np.asarray(c["x"], dtype=np.float64)
    zeros = np.zeros((N + 1, 12))
    ct = np.zeros((N + 1, 4), dtype=np.uint8)
    J, th = oracle.srbd_merit(p, np.asarray(c["x0hat"]), x, zeros, zeros, zeros, ct)
    assert J == pytest.approx(c["J"], rel=1e-13)
    assert th == pytest.approx(c["theta"], rel=1e-13)


# -------------------------------------------------------------- SRBD model
def test_srbd_free_fall_and_torque():
    p = synth.srbd_params()
    x = np.zeros(12)
    x[2] = 0.3
    x[6] = 0.5
    u = np.zeros(12)
    nxt = oracle.srbd_step(p, x, u, np.zeros(4, dtype=np.uint8))
    dt, g = p["dt"], p["gravity"]
    assert nxt[0] == pytest.approx(0.5 * dt)
    assert nxt[8] == pytest.approx(-g * dt)
    assert nxt[6] == pytest.approx(0.5)
    # one stance foot at r = (0.2, 0.15, 0), body at (0, 0, 0.3), force (0, 0, 10):
    # torque (r - p) x f = (0.2, 0.15, -0.3) x (0, 0, 10) = (1.5, -2.0, 0)
    u[2] = 10.0
    nxt = oracle.srbd_step(p, x, u, np.array([1, 0, 0, 0], dtype=np.uint8))
    I = p["inertia"]
    np.testing.assert_allclose(nxt[9:12], dt * np.array([1.5 / I[0], -2.0 / I[1], 0.0]), rtol=1e-14)
    assert nxt[8] == pytest.approx(dt * (10.0 / p["mass"] - g))


@pytest.mark.parametrize("nrob", [1, 2])
def test_srbd_jacobians_finite_difference(nrob):
    p = synth.srbd_params(nrob)
    prob = synth.srbd_problem(4, seed=3, nrob=nrob)
    g = np.random.default_rng(0)
    n = 12 * nrob
    x = prob["x0hat"] + g.normal(0, 0.3, n)
    u = prob["uref"][0] + g.normal(0, 5.0, n)
    ct = prob["contact"][0]
    A, B = oracle.srbd_jacobians(p, x, u, ct)
    h = 1e-6
    for j in range(n):
        e = np.zeros(n)
        e[j] = h
        fa = (oracle.srbd_step(p, x + e, u, ct) - oracle.srbd_step(p, x - e, u, ct)) / (2 * h)
        fb = (oracle.srbd_step(p, x, u + e, ct) - oracle.srbd_step(p, x, u - e, ct)) / (2 * h)
        assert np.abs(fa - A[:, j]).max() < 1e-8
        assert np.abs(fb - B[:, j]).max() < 1e-8


@pytest.mark.parametrize("nrob", [1, 2])
def test_srbd_linearize_derivatives(nrob):
    """q, r are gradients of the Lagrangian; Q, R its Gauss-Newton Hessian
    (exact here: the tracking terms are quadratic and the cone rows linear)."""
    p = synth.srbd_params(nrob)
    N = 3
    prob = synth.srbd_problem(N, seed=4, nrob=nrob)
    g = np.random.default_rng(1)
    n = 12 * nrob
    x = prob["x"] + g.normal(0, 0.2, prob["x"].shape)
    u = prob["u"] + g.normal(0, 3.0, prob["u"].shape)
    lam = g.normal(0, 1.0, prob["lam"].shape)
    xr, ur, ct = prob["xref"], prob["uref"], prob["contact"]
    lq = oracle.srbd_linearize(p, x, u, lam, xr, ur, ct)

    def lagr(xx, uu):
        L = 0.0
        L += lam[0] @ (prob["x0hat"] - xx[0])
        for k in range(N):
            L += oracle.srbd_cost(p, xx[k], uu[k], ct[k], xr[k], ur[k], False)
            L += lam[k + 1] @ (oracle.srbd_step(p, xx[k], uu[k], ct[k]) - xx[k + 1])
        L += oracle.srbd_cost(p, xx[N], None, None, xr[N], None, True)
        return L

    h = 1e-5
    for k in range(N + 1):
        for i in range(n):
            xp, xm = x.copy(), x.copy()
            xp[k, i] += h
            xm[k, i] -= h
            fd = (lagr(xp, u) - lagr(xm, u)) / (2 * h)
            assert abs(fd - lq["q"][k, i]) < 2e-6 * max(1, abs(fd))
        if k == N:
            break
        for i in range(n):
            up, um = u.copy(), u.copy()
            up[k, i] += h
            um[k, i] -= h
            fd = (lagr(x, up) - lagr(x, um)) / (2 * h)
            assert abs(fd - lq["r"][k, i]) < 2e-6 * max(1, abs(fd))
        # Hessians of the cost (no dynamics curvature: Gauss-Newton)
        def gcost(xx, uu):
            lq0 = oracle.srbd_linearize(p, xx, uu, np.zeros_like(lam), xr, ur, ct)
            return lq0["q"][k], lq0["r"][k]
        for i in range(n):
            up, um = u.copy(), u.copy()
            up[k, i] += h
            um[k, i] -= h
            fd = (gcost(x, up)[1] - gcost(x, um)[1]) / (2 * h)
            assert np.abs(fd - lq["R"][k][:, i]).max() < 1e-5 * max(1, np.abs(fd).max())
            xp, xm = x.copy(), x.copy()
            xp[k, i] += h
            xm[k, i] -= h
            fdx = (gcost(xp, u)[0] - gcost(xm, u)[0]) / (2 * h)
            # the x-gradient holds -lam_k and A^T lam_{k+1}; with lam = 0 it is the cost's
            assert np.abs(fdx - lq["Q"][k][:, i]).max() < 1e-5 * max(1, np.abs(fdx).max())
    # defects
    for k in range(N):
        np.testing.assert_allclose(lq["c"][k], oracle.srbd_step(p, x[k], u[k], ct[k]) - x[k + 1],
                                   rtol=0, atol=1e-14)


def test_lambda_invariance():
    """With q, r carrying the costate terms, (dx, du) and lam + dlam do not
    depend on the current lam (Gauss-Newton Hessian)."""
    p = synth.srbd_params()
    prob = synth.srbd_problem(10, seed=9)
    xr, ur, ct = prob["xref"], prob["uref"], prob["contact"]
    s = prob["x0hat"] - prob["x"][0]
    g = np.random.default_rng(3)
    lam_a = np.zeros_like(prob["lam"])
    lam_b = g.normal(0, 5.0, prob["lam"].shape)
    sols = []
    for lam in (lam_a, lam_b):
        lq = oracle.srbd_linearize(p, prob["x"], prob["u"], lam, xr, ur, ct)
        sol = oracle.riccati_solve(lq, s)
        sols.append((sol["dx"], sol["du"], lam + sol["dlam"]))
    for a, b in zip(*sols):
        assert np.abs(a - b).max() < 1e-9 * max(1, np.abs(a).max())


# ------------------------------------------------------------ line search
def test_filter_rule_cases():
    fa = oracle.filter_accept
    # above theta_max: only theta must drop
    assert fa(1.0, 5.0, -1.0, 1.0, 1.0, 100.0, 4.9)
    assert not fa(1.0, 5.0, -1.0, 1.0, 1.0, 0.0, 5.1)
    # below theta_max, descent direction: Armijo with c = 1e-4
    assert fa(1.0, 0.1, -2.0, 1.0, 0.5, 1.0 - 1e-4, 0.2)
    assert not fa(1.0, 0.1, -2.0, 1.0, 0.5, 1.0 - 0.5e-4, 0.2)
    assert not fa(1.0, 0.1, -2.0, 1.0, 0.5, 0.0, 1.5)     # theta above theta_max
    # not a descent direction: cost or theta must drop
    assert fa(1.0, 0.1, 2.0, 1.0, 1.0, 0.9, 0.5)
    assert fa(1.0, 0.1, 2.0, 1.0, 1.0, 1.1, 0.05)
    assert not fa(1.0, 0.1, 2.0, 1.0, 1.0, 1.1, 0.2)
    assert not fa(1.0, 0.1, -2.0, 1.0, 1.0, float("nan"), 0.0)


def ltv_model(n, m, N, seed):
    lq, _ = rand_lq(n, m, N, seed)
    return {"A": lq["A"], "B": lq["B"], "e": lq["c"], "Q": lq["Q"], "R": lq["R"],
            "S": lq["S"], "gq": lq["q"], "gr": lq["r"]}


def test_ltv_sqp_one_step():
    """On a linear model with quadratic cost the first SQP step is exact:
    alpha = 1 is accepted and the next step is zero."""
    n, m, N = 3, 2, 6
    mdl = ltv_model(n, m, N, seed=2)
    g = np.random.default_rng(4)
    x0hat = g.normal(0, 1, n)
    x = g.normal(0, 1, (N + 1, n))
    u = g.normal(0, 1, (N + 1, m))
    lam = np.zeros((N + 1, n))
    x1, u1, l1, info = oracle.ltv_sqp(mdl, x0hat, x, u, lam, max_iters=2)
    assert info["alpha"][0] == 1.0
    assert info["theta"] < 1e-12
    x2, u2, l2, info2 = oracle.ltv_sqp(mdl, x0hat, x1, u1, l1, max_iters=1)
    assert np.abs(x2 - x1).max() < 1e-10 and np.abs(u2 - u1).max() < 1e-10
    assert np.abs(l2 - l1).max() < 1e-9
    # the solution equals the dense QP of the full problem in absolute variables
    lq = {"A": mdl["A"], "B": mdl["B"], "c": mdl["e"], "Q": mdl["Q"], "R": mdl["R"],
          "S": mdl["S"], "q": mdl["gq"], "r": mdl["gr"]}
    z, nu, _ = dense_solve(lq, x0hat)
    dx, du, lamd = split(lq, z, nu)
    assert np.abs(x1 - dx).max() < 1e-9 and np.abs(u1[:N] - du).max() < 1e-9
    assert np.abs(l1 - lamd).max() < 1e-8


def test_srbd_sqp_converges():
    """After 20 Gauss-Newton SQP iterations the SRBD iterate is feasible and
    stationary (the Lagrangian gradients q, r vanish)."""
    p = synth.srbd_params()
    prob = synth.srbd_problem(20, seed=1)
    x, u, lam, info = oracle.srbd_sqp(p, prob["x0hat"], prob["x"], prob["u"], prob["lam"],
                                      prob["xref"], prob["uref"], prob["contact"], max_iters=20)
    assert info["status"] == 0 and info["iters"] == 20
    assert info["theta"] < 1e-10
    lq = oracle.srbd_linearize(p, x, u, lam, prob["xref"], prob["uref"], prob["contact"])
    assert np.abs(lq["q"]).max() < 1e-6 and np.abs(lq["r"][:20]).max() < 1e-6
    # the merit decreased from the initial guess
    J0, th0 = oracle.srbd_merit(p, prob["x0hat"], prob["x"], prob["u"], prob["xref"],
                                prob["uref"], prob["contact"])
    assert th0 > info["theta"]


def test_sqp_alpha_replay_reproduces_run():
    p = synth.srbd_params()
    prob = synth.srbd_problem(12, seed=2)
    args = (p, prob["x0hat"], prob["x"], prob["u"], prob["lam"], prob["xref"], prob["uref"],
            prob["contact"])
    x, u, lam, info = oracle.srbd_sqp(*args, max_iters=5)
    x2, u2, l2, info2 = oracle.srbd_sqp(*args, max_iters=5, alpha_replay=info["alpha"])
    assert np.array_equal(x, x2) and np.array_equal(u, u2) and np.array_equal(lam, l2)
