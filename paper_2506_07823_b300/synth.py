"""Seeded synthetic workloads shaped like the paper's (Sec. III-IV).

This module only draws random numbers and lays them out; it holds none of the
method's arithmetic, so both the CUDA path and the CPU oracle may consume its
output.  Instance ``i`` of a workload drawn with ``seed`` uses its own Philox
stream keyed by ``seed + i``; draws happen in the order written below.

Workloads
---------
* ``ltv_lq``     -- random time-varying LQ data (the single-LQR and the
                    whole-body-sized batch workloads): A_k = I + 0.1 G rescaled
                    to a given spectral radius, B_k iid normal, diagonal or
                    L L^T + 0.1 I state weights, R_k = r_w I, terminal 10 I,
                    q, r ~ N(0, 1), defects c ~ N(0, 0.01), initial defect
                    s ~ N(0, 1), S_k = 0.  Normal draws take a standard
                    deviation as their second parameter.
* ``srbd_problem`` -- single-rigid-body quadruped MPC problems (Sec. III):
                    physical constants, a trot contact schedule of period 0.5 s
                    (diagonal pairs alternate every 12.5 steps of 0.02 s),
                    forward-velocity references U[0, 1] m/s, random initial
                    states, and the initial guess (x_k = xhat_0, u_k = the
                    gravity-compensating stance forces, lam = 0).  With
                    ``nrob > 1`` robots are stacked and coupled by a ring
                    formation cost whose offsets lie on a circle of radius 1 m.
"""
from __future__ import annotations

import numpy as np

# ---------------------------------------------------------------- batching

def pack(instances: list[dict], keys) -> tuple[dict, np.ndarray, np.ndarray]:
    """Concatenate per-instance stage arrays (N_i + 1 slots each).

    Returns (packed dict, N per instance (int32), stage offsets (int64)).
    """
    Ns = np.array([inst[keys[0]].shape[0] - 1 for inst in instances], dtype=np.int32)
    off = np.zeros(len(instances), dtype=np.int64)
    if len(instances) > 1:
        off[1:] = np.cumsum(Ns[:-1].astype(np.int64) + 1)
    packed = {k: np.concatenate([inst[k] for inst in instances], axis=0) for k in keys}
    return packed, Ns, off


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=int(seed)))


# -------------------------------------------------------------- LTV LQ data

def ltv_lq(n: int, m: int, N: int, seed: int, rho: float = 0.95,
           b_std: float = 0.5, q_kind: str = "diag", r_w: float = 0.1,
           l_std: float = 0.3, terminal_w: float = 10.0) -> dict:
    """One random LTV LQ instance; float64 arrays with N+1 stage slots."""
    g = _rng(seed)
    A = np.zeros((N + 1, n, n))
    B = np.zeros((N + 1, n, m))
    c = np.zeros((N + 1, n))
    Q = np.zeros((N + 1, n, n))
    R = np.zeros((N + 1, m, m))
    S = np.zeros((N + 1, m, n))
    q = np.zeros((N + 1, n))
    r = np.zeros((N + 1, m))
    eye = np.eye(n)
    for k in range(N):
        A[k] = eye + 0.1 * g.normal(0.0, 1.0, (n, n))
        B[k] = g.normal(0.0, b_std, (n, m))
        if q_kind == "diag":
            Q[k] = np.diag(g.uniform(0.1, 1.0, n))
        else:
            L = g.normal(0.0, l_std, (n, n))
            Q[k] = L @ L.T + 0.1 * eye
        R[k] = r_w * np.eye(m)
        q[k] = g.normal(0.0, 1.0, n)
        r[k] = g.normal(0.0, 1.0, m)
        c[k] = g.normal(0.0, 0.01, n)
    Q[N] = terminal_w * eye
    q[N] = g.normal(0.0, 1.0, n)
    s = g.normal(0.0, 1.0, n)
    # rescale every A_k to spectral radius rho (one batched eigenvalue call)
    if N > 0:
        A[:N] *= (rho / np.abs(np.linalg.eigvals(A[:N])).max(axis=1))[:, None, None]
    return {"A": A, "B": B, "c": c, "Q": Q, "R": R, "S": S, "q": q, "r": r, "s": s}


LQ_KEYS = ("A", "B", "c", "Q", "R", "S", "q", "r")

# the small single-LQR workload and the whole-body-sized batch
LQ_SMALL = dict(n=4, m=2, N=16, rho=0.95, b_std=0.5, q_kind="diag", r_w=0.1)
LQ_WB = dict(n=36, m=24, N=100, rho=0.98, b_std=0.2, q_kind="llt", r_w=0.01)


def ltv_batch(count: int, seed: int = 0, Ns=None, **kw) -> tuple[list, dict, np.ndarray, np.ndarray, np.ndarray]:
    """``count`` LTV instances; ``Ns`` optionally overrides N per instance.

    Returns (instances, packed LQ dict, N int32, stage offsets int64, s (count, n)).
    """
    insts = []
    for i in range(count):
        args = dict(kw)
        if Ns is not None:
            args["N"] = int(Ns[i])
        insts.append(ltv_lq(seed=seed + i, **args))
    packed, Nv, off = pack(insts, LQ_KEYS)
    s = np.stack([inst["s"] for inst in insts])
    return insts, packed, Nv, off, s


# --------------------------------------------------------------- SRBD model

def srbd_params(nrob: int = 1) -> dict:
    """Model constants of the single-rigid-body quadruped workload."""
    W = np.array([0, 0, 100, 10, 10, 10, 10, 10, 10, 1, 1, 1], dtype=np.float64)
    foot = np.array([[0.2, 0.15, 0.0], [0.2, -0.15, 0.0],
                     [-0.2, 0.15, 0.0], [-0.2, -0.15, 0.0]])
    p = {"nrob": nrob, "mass": 12.0, "inertia": np.array([0.07, 0.26, 0.24]),
         "dt": 0.02, "gravity": 9.81, "foot": foot, "mu_fric": 0.6,
         "bar_mu": 0.1, "bar_delta": 1.0, "W": W, "Wu": np.full(12, 1e-3),
         "WN": 10.0 * W, "w_form": 10.0 if nrob > 1 else 0.0,
         "d_form": np.zeros((16, 3))}
    if nrob > 1:
        ang = 2.0 * np.pi * np.arange(nrob) / nrob
        ring = np.stack([np.cos(ang), np.sin(ang), np.zeros(nrob)], axis=1)
        p["d_form"][:nrob] = ring - np.roll(ring, -1, axis=0)
    return p


def trot_contact(N: int, offset: int = 0) -> np.ndarray:
    """[N+1][4] stance flags; legs (FL, FR, HL, HR); period 25 steps of 0.02 s.

    Pair (FL, HR) stands during the first 12.5 steps of a period and pair
    (FR, HL) during the rest; a step j of the period is in the first half
    when 2 j < 25.
    """
    k = np.arange(N + 1) + offset
    first = (2 * (k % 25)) < 25
    c = np.zeros((N + 1, 4), dtype=np.uint8)
    c[:, 0] = first
    c[:, 3] = first
    c[:, 1] = ~first
    c[:, 2] = ~first
    return c


def srbd_problem(N: int, seed: int, nrob: int = 1, params: dict | None = None) -> dict:
    """One SRBD MPC problem.  Random draws per robot, in order: forward
    velocity reference U[0, 1], position offset N(0, 0.05) (3), linear
    velocity N(0, 0.3) (3), angular velocity N(0, 0.3) (3)."""
    prm = params if params is not None else srbd_params(nrob)
    g = _rng(seed)
    n = 12 * nrob
    x0 = np.zeros(n)
    xref = np.zeros((N + 1, n))
    uref = np.zeros((N + 1, n))
    contact = np.zeros((N + 1, nrob, 4), dtype=np.uint8)
    base = trot_contact(N)
    for b in range(nrob):
        vx = g.uniform(0.0, 1.0)
        dp = g.normal(0.0, 0.05, 3)
        dv = g.normal(0.0, 0.3, 3)
        dw = g.normal(0.0, 0.3, 3)
        o = 12 * b
        x0[o:o + 3] = np.array([0.0, 0.0, 0.3]) + dp
        x0[o + 6:o + 9] = dv
        x0[o + 9:o + 12] = dw
        xref[:, o + 2] = 0.3
        xref[:, o + 6] = vx
        contact[:, b, :] = base
        nst = base.sum(axis=1).astype(np.float64)
        for j in range(4):
            uref[:, o + 3 * j + 2] = np.where(base[:, j] > 0,
                                              prm["mass"] * prm["gravity"] / np.maximum(nst, 1.0), 0.0)
    uref[N] = 0.0
    x = np.tile(x0, (N + 1, 1))
    u = uref.copy()
    lam = np.zeros((N + 1, n))
    return {"params": prm, "N": N, "nrob": nrob, "x0hat": x0, "x": x, "u": u,
            "lam": lam, "xref": xref, "uref": uref,
            "contact": contact.reshape(N + 1, 4 * nrob)}


SRBD_KEYS = ("x", "u", "lam", "xref", "uref", "contact")


def srbd_batch(count: int, seed: int = 0, N=50, Ns_choices=None, nrob: int = 1):
    """``count`` SRBD problems.  With ``Ns_choices`` each instance first draws
    its horizon uniformly from the choices (own Philox stream, key seed+i,
    before the problem draws use key 2^32 + seed + i)."""
    insts = []
    for i in range(count):
        Ni = N
        if Ns_choices is not None:
            Ni = int(_rng(seed + i).choice(np.asarray(Ns_choices)))
        insts.append(srbd_problem(Ni, seed=(1 << 32) + seed + i if Ns_choices is not None else seed + i,
                                  nrob=nrob))
    packed, Nv, off = pack(insts, SRBD_KEYS)
    x0hat = np.stack([inst["x0hat"] for inst in insts])
    return insts, packed, Nv, off, x0hat
