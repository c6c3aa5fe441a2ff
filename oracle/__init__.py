"""Plain FP64 CPU oracle for the primal-dual iLQR hot path -- TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never loads it and
shares no code with it; the C source (``pdilqr_oracle.c``) follows the paper's
equations loop by loop:

* ``riccati_solve``      -- Sec. II-C, Eq. (lqr) backward/forward and the
                            costate recovery dlam_i = P_i dx_i + p_i.
* ``kkt_residual``       -- first-order conditions of Eq. (QP) with the
                            Lagrangian of Sec. II-B.
* ``barrier``            -- relaxed barrier of Sec. II-F.
* ``srbd_*``             -- single-rigid-body model of Sec. III (the paper
                            prints no equations: the reading is documented in
                            the C header).
* ``srbd_sqp``/``ltv_sqp`` -- multiple-shooting SQP with the parallel filter
                            line search of Sec. II-E.

Every function is pinned by ``tests/test_oracle_pins.py`` against something
other than itself (dense KKT solves, closed forms, finite differences, brute
force).  No function here is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pdilqr_oracle.c")
_HDR = os.path.join(_HERE, "pdilqr_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")

_dp = ctypes.POINTER(ctypes.c_double)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math)."""
    stale = (not os.path.exists(_LIB)) or any(
        os.path.getmtime(f) > os.path.getmtime(_LIB) for f in (_SRC, _HDR))
    if force or stale:
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class SrbdParams(ctypes.Structure):
    _fields_ = [("nrob", ctypes.c_int), ("w_form", ctypes.c_double),
                ("d_form", ctypes.c_double * 48),
                ("mass", ctypes.c_double), ("inertia", ctypes.c_double * 3),
                ("dt", ctypes.c_double), ("gravity", ctypes.c_double),
                ("foot", ctypes.c_double * 12), ("mu_fric", ctypes.c_double),
                ("bar_mu", ctypes.c_double), ("bar_delta", ctypes.c_double),
                ("W", ctypes.c_double * 12), ("Wu", ctypes.c_double * 12),
                ("WN", ctypes.c_double * 12)]


class SqpOpts(ctypes.Structure):
    _fields_ = [("max_iters", ctypes.c_int), ("tol_step", ctypes.c_double),
                ("tol_theta", ctypes.c_double), ("c_armijo", ctypes.c_double),
                ("theta_frac", ctypes.c_double), ("alpha_replay", _dp)]


class SqpInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("status", ctypes.c_int),
                ("alpha", ctypes.c_double * 32), ("step", ctypes.c_double * 32),
                ("theta_it", ctypes.c_double * 32),
                ("J", ctypes.c_double),
                ("theta", ctypes.c_double), ("theta_max", ctypes.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.orc_riccati_solve.restype = ctypes.c_int
        _lib.orc_srbd_cost.restype = ctypes.c_double
        _lib.orc_ltv_cost.restype = ctypes.c_double
        _lib.orc_filter_accept.restype = ctypes.c_int
        _lib.orc_filter_accept.argtypes = [ctypes.c_double] * 7 + [ctypes.c_double]
        _lib.orc_barrier.argtypes = [ctypes.c_double] * 3 + [_dp]
    return _lib


def _d(a):
    """Contiguous float64 view (or None) and its ctypes pointer."""
    if a is None:
        return None, None
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def _u8(a):
    a = np.ascontiguousarray(a, dtype=np.uint8)
    return a, a.ctypes.data_as(_u8p)


# ------------------------------------------------------------------ LQ solve
def riccati_solve(lq: dict, s):
    """Solve the LQ KKT system of one instance (Eq. lqr).

    ``lq`` holds float arrays with N+1 stage slots: A (N+1,n,n), B (N+1,n,m),
    c (N+1,n), Q (N+1,n,n), R (N+1,m,m), S (N+1,m,n), q (N+1,n), r (N+1,m).
    Returns dict(dx, du, dlam, K, k, P, p) in float64.
    """
    A = lq["A"]
    N = A.shape[0] - 1
    n = A.shape[1]
    m = lq["B"].shape[2]
    keep = [_d(lq[k]) for k in ("A", "B", "c", "Q", "R", "S", "q", "r")]
    sv = _d(s)
    out = {"dx": np.zeros((N + 1, n)), "du": np.zeros((N + 1, m)),
           "dlam": np.zeros((N + 1, n)), "K": np.zeros((N + 1, m, n)),
           "k": np.zeros((N + 1, m)), "P": np.zeros((N + 1, n, n)),
           "p": np.zeros((N + 1, n))}
    ptr = {k: v.ctypes.data_as(_dp) for k, v in out.items()}
    st = lib().orc_riccati_solve(n, m, N, *[k[1] for k in keep], sv[1],
                                 ptr["dx"], ptr["du"], ptr["dlam"], ptr["K"],
                                 ptr["k"], ptr["P"], ptr["p"])
    if st != 0:
        raise np.linalg.LinAlgError("G_k not positive definite")
    return out


def kkt_residual(lq: dict, s, dx, du, dlam):
    """Return (res_inf, K_inf, z_inf, rhs_inf) of the LQ KKT system."""
    A = lq["A"]
    N = A.shape[0] - 1
    n = A.shape[1]
    m = lq["B"].shape[2]
    keep = [_d(lq[k]) for k in ("A", "B", "c", "Q", "R", "S", "q", "r")]
    z = [_d(s), _d(dx), _d(du), _d(dlam)]
    out = np.zeros(4)
    lib().orc_kkt_residual(n, m, N, *[k[1] for k in keep], *[v[1] for v in z],
                           out.ctypes.data_as(_dp))
    return tuple(float(v) for v in out)


def kkt_backward_error(lq, s, dx, du, dlam) -> float:
    """Normwise backward error |Kz - rhs| / (|K| |z| + |rhs|), inf-norms."""
    res, kn, zn, rn = kkt_residual(lq, s, dx, du, dlam)
    return res / (kn * zn + rn)


def barrier(xi: float, mu: float, delta: float):
    out = np.zeros(3)
    lib().orc_barrier(float(xi), float(mu), float(delta), out.ctypes.data_as(_dp))
    return out


# ---------------------------------------------------------------- SRBD model
def make_params(p: dict) -> SrbdParams:
    prm = SrbdParams()
    prm.nrob = int(p.get("nrob", 1))
    prm.w_form = float(p.get("w_form", 0.0))
    d = np.zeros(48)
    if "d_form" in p:
        df = np.asarray(p["d_form"], dtype=np.float64).reshape(-1)
        d[:df.size] = df
    prm.d_form[:] = d.tolist()
    prm.mass = p["mass"]
    prm.inertia[:] = list(p["inertia"])
    prm.dt = p["dt"]
    prm.gravity = p["gravity"]
    prm.foot[:] = list(np.asarray(p["foot"], dtype=np.float64).reshape(12))
    prm.mu_fric = p["mu_fric"]
    prm.bar_mu = p["bar_mu"]
    prm.bar_delta = p["bar_delta"]
    prm.W[:] = list(p["W"])
    prm.Wu[:] = list(p["Wu"])
    prm.WN[:] = list(p["WN"])
    return prm


def srbd_step(p: dict, x, u, contact):
    prm = make_params(p)
    xv, uv, cv = _d(x), _d(u), _u8(contact)
    out = np.zeros_like(xv[0])
    lib().orc_srbd_step(ctypes.byref(prm), xv[1], uv[1], cv[1], out.ctypes.data_as(_dp))
    return out


def srbd_jacobians(p: dict, x, u, contact):
    prm = make_params(p)
    n = len(x)
    xv, uv, cv = _d(x), _d(u), _u8(contact)
    A = np.zeros((n, n))
    B = np.zeros((n, n))
    lib().orc_srbd_jacobians(ctypes.byref(prm), xv[1], uv[1], cv[1],
                             A.ctypes.data_as(_dp), B.ctypes.data_as(_dp))
    return A, B


def srbd_cost(p: dict, x, u, contact, xref, uref, terminal: bool) -> float:
    prm = make_params(p)
    xv, xr = _d(x), _d(xref)
    if terminal:
        return lib().orc_srbd_cost(ctypes.byref(prm), xv[1], None, None, xr[1], None, 1)
    uv, cv, ur = _d(u), _u8(contact), _d(uref)
    return lib().orc_srbd_cost(ctypes.byref(prm), xv[1], uv[1], cv[1], xr[1], ur[1], 0)


def srbd_linearize(p: dict, x, u, lam, xref, uref, contact) -> dict:
    prm = make_params(p)
    N = x.shape[0] - 1
    n = x.shape[1]
    m = n
    out = {"A": np.zeros((N + 1, n, n)), "B": np.zeros((N + 1, n, m)),
           "c": np.zeros((N + 1, n)), "Q": np.zeros((N + 1, n, n)),
           "R": np.zeros((N + 1, m, m)), "S": np.zeros((N + 1, m, n)),
           "q": np.zeros((N + 1, n)), "r": np.zeros((N + 1, m))}
    ins = [_d(x), _d(u), _d(lam), _d(xref), _d(uref), _u8(contact)]
    lib().orc_srbd_linearize(ctypes.byref(prm), N, *[v[1] for v in ins],
                             *[out[k].ctypes.data_as(_dp) for k in
                               ("A", "B", "c", "Q", "R", "S", "q", "r")])
    return out


def srbd_merit(p: dict, x0hat, x, u, xref, uref, contact):
    prm = make_params(p)
    N = x.shape[0] - 1
    J = ctypes.c_double()
    th = ctypes.c_double()
    ins = [_d(x0hat), _d(x), _d(u), _d(xref), _d(uref), _u8(contact)]
    lib().orc_srbd_merit(ctypes.byref(prm), N, *[v[1] for v in ins],
                         ctypes.byref(J), ctypes.byref(th))
    return J.value, th.value


def filter_accept(J0, th0, dphi, th_max, alpha, Ja, tha, c_armijo=1e-4) -> bool:
    return bool(lib().orc_filter_accept(J0, th0, dphi, th_max, alpha, Ja, tha, c_armijo))


def _opts(max_iters, tol_step, tol_theta, c_armijo, theta_frac, alpha_replay):
    o = SqpOpts()
    o.max_iters = int(max_iters)
    o.tol_step = float(tol_step)
    o.tol_theta = float(tol_theta)
    o.c_armijo = float(c_armijo)
    o.theta_frac = float(theta_frac)
    keep = None
    if alpha_replay is not None:
        keep = np.zeros(32)
        keep[:len(alpha_replay)] = alpha_replay
        o.alpha_replay = keep.ctypes.data_as(_dp)
    return o, keep


def _info(info: SqpInfo) -> dict:
    return {"iters": info.iters, "status": info.status,
            "alpha": np.array(info.alpha[:max(info.iters, 0)]),
            "step": np.array(info.step[:max(info.iters, 0)]),
            "theta_it": np.array(info.theta_it[:max(info.iters, 0)]),
            "J": info.J, "theta": info.theta, "theta_max": info.theta_max}


def srbd_sqp(p: dict, x0hat, x, u, lam, xref, uref, contact, max_iters=10,
             tol_step=0.0, tol_theta=0.0, c_armijo=1e-4, theta_frac=1e-2,
             alpha_replay=None):
    """Run the SQP; returns (x, u, lam, info) as new float64 arrays."""
    prm = make_params(p)
    N = x.shape[0] - 1
    x = np.array(x, dtype=np.float64)
    u = np.array(u, dtype=np.float64)
    lam = np.array(lam, dtype=np.float64)
    o, keep = _opts(max_iters, tol_step, tol_theta, c_armijo, theta_frac, alpha_replay)
    info = SqpInfo()
    ins = [_d(x0hat)]
    refs = [_d(xref), _d(uref), _u8(contact)]
    lib().orc_srbd_sqp(ctypes.byref(prm), N, ins[0][1], x.ctypes.data_as(_dp),
                       u.ctypes.data_as(_dp), lam.ctypes.data_as(_dp),
                       *[v[1] for v in refs], ctypes.byref(o), ctypes.byref(info))
    del keep
    return x, u, lam, _info(info)


def ltv_sqp(model: dict, x0hat, x, u, lam, max_iters=10, tol_step=0.0,
            tol_theta=0.0, c_armijo=1e-4, theta_frac=1e-2, alpha_replay=None):
    """SQP on the LTV test model; ``model`` has A, B, e, Q, R, S, gq, gr."""
    A = model["A"]
    N = A.shape[0] - 1
    n = A.shape[1]
    m = model["B"].shape[2]
    x = np.array(x, dtype=np.float64)
    u = np.array(u, dtype=np.float64)
    lam = np.array(lam, dtype=np.float64)
    o, keep = _opts(max_iters, tol_step, tol_theta, c_armijo, theta_frac, alpha_replay)
    info = SqpInfo()
    mats = [_d(model[k]) for k in ("A", "B", "e", "Q", "R", "S", "gq", "gr")]
    xh = _d(x0hat)
    lib().orc_ltv_sqp(n, m, N, *[v[1] for v in mats], xh[1], x.ctypes.data_as(_dp),
                      u.ctypes.data_as(_dp), lam.ctypes.data_as(_dp),
                      ctypes.byref(o), ctypes.byref(info))
    del keep
    return x, u, lam, _info(info)


def ltv_cost(model: dict, x, u) -> float:
    A = model["A"]
    N = A.shape[0] - 1
    n = A.shape[1]
    m = model["B"].shape[2]
    mats = [_d(model[k]) for k in ("Q", "R", "S", "gq", "gr")]
    xv, uv = _d(x), _d(u)
    return lib().orc_ltv_cost(n, m, N, *[v[1] for v in mats], xv[1], uv[1])
