"""The allocation-free LQ KKT solve gives the same answer as the planned one.

Some callers cannot allocate device memory: a real-time control loop that
may not block on cudaMalloc, code that runs while a CUDA graph is being
captured, or an application whose memory pool already owns the GPU.  For
them the library exposes pdilqr_kkt_scan_solve_noalloc, which keeps its
workspace in a static device array.  This file is collected last so that a
run stopping at the first failure has already run every other test; it also
passes on its own in a fresh process.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_07823_b300 import synth

pytestmark = pytest.mark.gpu

REL_TOL = 1e-4   # the relative tolerance of the other parity tests


def _batch(n, m, Ns, seed, with_insts=False):
    insts = [synth.ltv_lq(n, m, N, seed + i, rho=0.95, b_std=0.5, q_kind="diag", r_w=0.1)
             for i, N in enumerate(Ns)]
    packed, Nv, off = synth.pack(insts, synth.LQ_KEYS)
    s = np.stack([inst["s"] for inst in insts])
    lq = {k: torch.tensor(np.asarray(v, np.float32), device="cuda") for k, v in packed.items()}
    lq["S"] = None
    out = (lq, torch.tensor(np.asarray(s, np.float32), device="cuda"), Nv, off)
    return out + (insts, s) if with_insts else out


def _oracle_rel(insts, s, Nv, off, dx, du, dlam):
    """Largest per-block relative error of one solve against the FP64 oracle
    (which solves the same FP32-rounded data)."""
    worst = 0.0
    d = [t.double().cpu().numpy() for t in (dx, du, dlam)]
    for i, inst in enumerate(insts):
        N, o = int(Nv[i]), int(off[i])
        lq = {k: np.asarray(inst[k], np.float32).astype(np.float64) for k in synth.LQ_KEYS}
        ref = oracle.riccati_solve(lq, np.asarray(s[i], np.float32).astype(np.float64))
        for got, want in ((d[0][o:o + N + 1], ref["dx"]), (d[1][o:o + N], ref["du"][:N]),
                          (d[2][o:o + N + 1], ref["dlam"])):
            worst = max(worst, np.abs(got - want).max() / max(np.abs(want).max(), 1e-30))
    return worst


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max().clamp_min(1e-30))


@pytest.mark.parametrize("n,m,warps", [(12, 12, 8), (4, 2, 4)])
def test_noalloc_matches_planned_solve_twice(n, m, warps):
    from paper_2506_07823_b300 import pdilqr
    lq, s, Nv, off, insts, s_host = _batch(n, m, [1, 7, 33, 50, 100, 16], seed=900 + n,
                                           with_insts=True)
    plan = pdilqr.Plan(n, m, Nv, off, warps=warps)
    ref = plan.kkt_scan_solve(lq, s)
    T = plan.total
    N_dev = torch.tensor(Nv, dtype=torch.int32, device="cuda")
    off_dev = torch.tensor(off, dtype=torch.int64, device="cuda")
    for call in range(2):
        out = {k: torch.full_like(ref[k], float("nan")) for k in ("dx", "du", "dlam")}
        st = torch.full((len(Nv),), -1, dtype=torch.int32, device="cuda")
        pdilqr.kkt_scan_solve_noalloc(n, m, N_dev, off_dev, T, lq, s, out["dx"], out["du"],
                                      out["dlam"], st, warps=warps)
        torch.cuda.synchronize()
        assert torch.all(st == 0), (call, st)
        for k in ("dx", "du", "dlam"):
            assert _rel(out[k], ref[k]) <= REL_TOL, (call, k, _rel(out[k], ref[k]))
        e = _oracle_rel(insts, s_host, Nv, off, out["dx"], out["du"], out["dlam"])
        assert e <= REL_TOL, (call, e)


def test_noalloc_flags_instances_outside_the_scratch():
    """An instance whose slot range ends beyond total_stages (or has N < 1) is
    reported as E_INVALID_ARG and not touched; the others are solved."""
    from paper_2506_07823_b300 import pdilqr
    n, m = 4, 2
    lq, s, Nv, off, insts, s_host = _batch(n, m, [5, 7, 3], seed=21, with_insts=True)
    T = int(off[-1] + Nv[-1] + 1)
    limit = int(off[1] + Nv[1])             # instance 1 ends one slot past this
    Nbad = Nv.copy()
    Nbad[2] = 0                             # instance 2: empty horizon
    N_dev = torch.tensor(Nbad, dtype=torch.int32, device="cuda")
    off_dev = torch.tensor(off, dtype=torch.int64, device="cuda")
    out = {k: torch.full((T, n if k != "du" else m), 7.0, device="cuda") for k in ("dx", "du", "dlam")}
    st = torch.full((3,), -1, dtype=torch.int32, device="cuda")
    pdilqr.kkt_scan_solve_noalloc(n, m, N_dev, off_dev, limit, lq, s, out["dx"], out["du"],
                                  out["dlam"], st, warps=4)
    torch.cuda.synchronize()
    assert st.tolist() == [0, pdilqr.E_INVALID_ARG, pdilqr.E_INVALID_ARG]
    for i in (1, 2):
        sl = slice(int(off[i]), int(off[i]) + int(Nv[i]) + 1)
        for k in ("dx", "du", "dlam"):
            assert torch.all(out[k][sl] == 7.0), (i, k)
    e = _oracle_rel(insts[:1], s_host[:1], Nv[:1], off[:1], out["dx"], out["du"], out["dlam"])
    assert e <= REL_TOL, e


def test_noalloc_rejects_oversized_batch():
    from paper_2506_07823_b300 import pdilqr
    cap = pdilqr.noalloc_capacity_stages(12, 12)
    assert cap > 1000
    lq, s, Nv, off = _batch(12, 12, [5], seed=3)
    N_dev = torch.tensor(Nv, dtype=torch.int32, device="cuda")
    off_dev = torch.tensor(off, dtype=torch.int64, device="cuda")
    out = torch.zeros(6, 12, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(pdilqr.PdilqrError) as e:
        pdilqr.kkt_scan_solve_noalloc(12, 12, N_dev, off_dev, cap + 1, lq, s, out, out, out, st)
    assert e.value.code == pdilqr.E_INVALID_ARG
