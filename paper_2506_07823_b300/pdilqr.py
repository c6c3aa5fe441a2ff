"""Thin ctypes binding of ``libpdilqr.so`` (the C ABI of ``include/pdilqr.h``).

Argument marshalling only: tensors are checked (CUDA, float32/int32/float64,
contiguous) and their device pointers handed to the library; every step of
the hot path runs in the library's kernels.  There is no CPU fallback: if the
library is missing the import of this module fails.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpdilqr.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libpdilqr.so is not built; run paper_2506_07823_b300.build.build_library()")

_lib = ctypes.CDLL(LIB_PATH)

STATUS = {0: "OK", 1: "E_INVALID_ARG", 2: "E_NOT_SPD", 3: "E_SINGULAR", 4: "E_NONFINITE",
          5: "E_TIMEOUT", 6: "E_NO_MEMORY", 7: "E_ADMISSION", 8: "E_LINESEARCH", 9: "E_CUDA"}
OK, E_INVALID_ARG, E_NOT_SPD, E_SINGULAR = 0, 1, 2, 3
E_NONFINITE, E_TIMEOUT, E_NO_MEMORY, E_ADMISSION, E_LINESEARCH, E_CUDA = 4, 5, 6, 7, 8, 9

_vp = ctypes.c_void_p


class PdilqrError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {STATUS.get(code, code)} "
                         f"({_lib.pdilqr_status_string(code).decode()})")
        self.code = code


class _Batch(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("m", ctypes.c_int32), ("count", ctypes.c_int32),
                ("N", _vp), ("stage_off", _vp)]


class _Opts(ctypes.Structure):
    _fields_ = [("warps", ctypes.c_int32), ("refine", ctypes.c_int32)]


class _LQ(ctypes.Structure):
    _fields_ = [(k, _vp) for k in ("A", "B", "c", "Q", "R", "S", "q", "r")]


class _KktOut(ctypes.Structure):
    _fields_ = [(k, _vp) for k in ("dx", "du", "dlam", "K", "k", "P", "p", "status", "resid")]


_lib.pdilqr_status_string.restype = ctypes.c_char_p
_lib.pdilqr_status_string.argtypes = [ctypes.c_int]
_lib.pdilqr_plan_create.argtypes = [ctypes.POINTER(_Batch), ctypes.POINTER(_Opts), ctypes.POINTER(_vp)]
_lib.pdilqr_plan_destroy.argtypes = [_vp]
_lib.pdilqr_plan_warps.argtypes = [_vp]
_lib.pdilqr_plan_warps.restype = ctypes.c_int32
for _f in ("pdilqr_kkt_scan_solve", "pdilqr_riccati_solve"):
    getattr(_lib, _f).argtypes = [_vp, ctypes.POINTER(_LQ), _vp, ctypes.POINTER(_KktOut), _vp]
_lib.pdilqr_kkt_residual.argtypes = [_vp, ctypes.POINTER(_LQ), _vp, _vp, _vp, _vp, _vp, _vp]


def lib() -> ctypes.CDLL:
    return _lib


def _check(code: int, where: str):
    if code != 0:
        raise PdilqrError(code, where)


def _ptr(t, dtype=torch.float32, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


class Plan:
    """A batch of ``count`` instances with common (n, m) and horizons ``N``.

    ``N`` (int) and ``stage_off`` (int64) are host arrays; stage arrays of the
    batch hold ``N_i + 1`` slots per instance starting at ``stage_off[i]``.
    """

    def __init__(self, n: int, m: int, N, stage_off, warps: int = 0, refine: bool = False):
        self.n, self.m = int(n), int(m)
        self.N = np.ascontiguousarray(np.asarray(N, dtype=np.int32))
        self.stage_off = np.ascontiguousarray(np.asarray(stage_off, dtype=np.int64))
        self.count = int(self.N.size)
        self.total = int((self.stage_off + self.N + 1).max())
        b = _Batch(self.n, self.m, self.count, self.N.ctypes.data, self.stage_off.ctypes.data)
        o = _Opts(int(warps), int(bool(refine)))
        h = _vp()
        _check(_lib.pdilqr_plan_create(ctypes.byref(b), ctypes.byref(o), ctypes.byref(h)),
               "pdilqr_plan_create")
        self._h = h
        self.warps = int(_lib.pdilqr_plan_warps(h))

    def close(self):
        if getattr(self, "_h", None):
            _lib.pdilqr_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ helpers
    def _lq(self, lq: dict) -> _LQ:
        return _LQ(*[_ptr(lq.get(k), name=k) if (k != "S" or lq.get("S") is not None) else None
                     for k in ("A", "B", "c", "Q", "R", "S", "q", "r")])

    def alloc_out(self, device="cuda", want_policy=False, want_resid=False) -> dict:
        T, n, m = self.total, self.n, self.m
        f = dict(device=device, dtype=torch.float32)
        out = {"dx": torch.zeros(T, n, **f), "du": torch.zeros(T, m, **f),
               "dlam": torch.zeros(T, n, **f),
               "status": torch.full((self.count,), -1, device=device, dtype=torch.int32)}
        if want_policy:
            out.update(K=torch.zeros(T, m, n, **f), k=torch.zeros(T, m, **f),
                       P=torch.zeros(T, n, n, **f), p=torch.zeros(T, n, **f))
        if want_resid:
            out["resid"] = torch.zeros(self.count, 4, device=device, dtype=torch.float64)
        return out

    def _out(self, out: dict) -> _KktOut:
        return _KktOut(_ptr(out["dx"], name="dx"), _ptr(out["du"], name="du"),
                       _ptr(out["dlam"], name="dlam"), _ptr(out.get("K"), name="K"),
                       _ptr(out.get("k"), name="k"), _ptr(out.get("P"), name="P"),
                       _ptr(out.get("p"), name="p"),
                       _ptr(out["status"], torch.int32, "status"),
                       _ptr(out.get("resid"), torch.float64, "resid"))

    # -------------------------------------------------------------- calls
    def kkt_scan_solve(self, lq: dict, s, out: dict | None = None, stream=None, **kw) -> dict:
        out = out if out is not None else self.alloc_out(**kw)
        _check(_lib.pdilqr_kkt_scan_solve(self._h, ctypes.byref(self._lq(lq)), _ptr(s, name="s"),
                                          ctypes.byref(self._out(out)), _stream(stream)),
               "pdilqr_kkt_scan_solve")
        return out

    def riccati_solve(self, lq: dict, s, out: dict | None = None, stream=None, **kw) -> dict:
        out = out if out is not None else self.alloc_out(**kw)
        _check(_lib.pdilqr_riccati_solve(self._h, ctypes.byref(self._lq(lq)), _ptr(s, name="s"),
                                         ctypes.byref(self._out(out)), _stream(stream)),
               "pdilqr_riccati_solve")
        return out

    def kkt_residual(self, lq: dict, s, dx, du, dlam, resid=None, stream=None):
        if resid is None:
            resid = torch.zeros(self.count, 4, device=dx.device, dtype=torch.float64)
        _check(_lib.pdilqr_kkt_residual(self._h, ctypes.byref(self._lq(lq)), _ptr(s, name="s"),
                                        _ptr(dx, name="dx"), _ptr(du, name="du"),
                                        _ptr(dlam, name="dlam"),
                                        _ptr(resid, torch.float64, "resid"), _stream(stream)),
               "pdilqr_kkt_residual")
        return resid


def backward_error(resid: torch.Tensor) -> torch.Tensor:
    """Normwise backward error |Kz - rhs| / (|K| |z| + |rhs|) per instance."""
    r = resid.double()
    return r[:, 0] / (r[:, 1] * r[:, 2] + r[:, 3])
