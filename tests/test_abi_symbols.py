"""The C-ABI library loads and exports every symbol include/*.h declares
(CPU only: no compute calls)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        names |= set(re.findall(r"PDILQR_API\s+[\w\s\*]*?\b(pdilqr_\w+)\s*\(", src))
    return sorted(names)


def test_header_declares_entry_points():
    names = declared()
    for must in ("pdilqr_kkt_scan_solve", "pdilqr_riccati_solve", "pdilqr_kkt_residual",
                 "pdilqr_plan_create"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2506_07823_b300 import build
    lib_path = build.build_library()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings():
    from paper_2506_07823_b300 import pdilqr
    assert pdilqr.lib().pdilqr_status_string(0) == b"ok"
    assert pdilqr.lib().pdilqr_status_string(3).startswith(b"singular")


def test_plan_rejects_bad_batches_without_gpu_work():
    """Validation happens on the host before any device call."""
    from paper_2506_07823_b300 import pdilqr
    with pytest.raises(pdilqr.PdilqrError) as e:
        pdilqr.Plan(5, 5, [4], [0])              # unsupported (n, m)
    assert e.value.code == pdilqr.E_INVALID_ARG
    with pytest.raises(pdilqr.PdilqrError):
        pdilqr.Plan(4, 2, [4, 4], [0, 3])        # overlapping slot ranges
    with pytest.raises(pdilqr.PdilqrError):
        pdilqr.Plan(4, 2, [0], [0])              # empty horizon
    with pytest.raises(pdilqr.PdilqrError):
        pdilqr.Plan(4, 2, [4], [0], warps=5)     # unsupported warp count
    with pytest.raises(pdilqr.PdilqrError):
        pdilqr.Plan(4, 2, [4], [0], warps=2)


def test_autotune_candidates_cover_the_configurations():
    """The batch autotuner's candidate list (host logic, no GPU): the one-robot
    size times the sequential recursion at 2, 4 and 8 instances per CTA and
    the scan at 4, 8 and 16 chunks; other sizes the solver and chunk count;
    every label is distinct."""
    from paper_2506_07823_b300 import autotune
    c12 = autotune.candidates(12, 12)
    assert {(1, 2), (1, 4), (1, 8), (4, 0), (8, 0), (16, 0)} == set(c12)
    assert set(autotune.candidates(48, 48)) == {(1, 0), (4, 0), (8, 0), (16, 0)}
    labels = [autotune.label(w, i) for w, i in c12]
    assert len(set(labels)) == len(labels)
    assert autotune.label(1, 8) == "seq/8" and autotune.label(16, 0) == "scan/16"
