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
