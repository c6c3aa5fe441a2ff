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
    _fields_ = [("warps", ctypes.c_int32), ("refine", ctypes.c_int32),
                ("inst_per_cta", ctypes.c_int32), ("m_fp64", ctypes.c_int32),
                ("split", ctypes.c_int32)]


class _LQ(ctypes.Structure):
    _fields_ = [(k, _vp) for k in ("A", "B", "c", "Q", "R", "S", "q", "r")]


class _KktOut(ctypes.Structure):
    _fields_ = [(k, _vp) for k in ("dx", "du", "dlam", "K", "k", "P", "p", "status", "resid")]


class SrbdModel(ctypes.Structure):
    _fields_ = [("nrob", ctypes.c_int32), ("w_form", ctypes.c_float),
                ("d_form", ctypes.c_float * 48), ("mass", ctypes.c_float),
                ("inertia", ctypes.c_float * 3), ("dt", ctypes.c_float),
                ("gravity", ctypes.c_float), ("foot", ctypes.c_float * 12),
                ("mu_fric", ctypes.c_float), ("bar_mu", ctypes.c_float),
                ("bar_delta", ctypes.c_float), ("W", ctypes.c_float * 12),
                ("Wu", ctypes.c_float * 12), ("WN", ctypes.c_float * 12)]


class _Traj(ctypes.Structure):
    _fields_ = [(k, _vp) for k in ("x", "u", "lam", "xref", "uref", "contact")]


class _LQOut(ctypes.Structure):
    _fields_ = [(k, _vp) for k in ("A", "B", "c", "Q", "R", "S", "q", "r")]


class _SqpOpts(ctypes.Structure):
    _fields_ = [("max_iters", ctypes.c_int32), ("tol_step", ctypes.c_float),
                ("tol_theta", ctypes.c_float), ("c_armijo", ctypes.c_float),
                ("theta_frac", ctypes.c_float), ("alpha_replay", _vp)]


class _SqpInfo(ctypes.Structure):
    _fields_ = [(k, _vp) for k in ("iters", "status", "alpha", "J", "theta")]


def srbd_model(p: dict) -> SrbdModel:
    """Pack a model-constant dict (see ``synth.srbd_params``) into the C struct."""
    m = SrbdModel()
    m.nrob = int(p.get("nrob", 1))
    m.w_form = float(p.get("w_form", 0.0))
    d = np.zeros(48, dtype=np.float64)
    if "d_form" in p:
        df = np.asarray(p["d_form"], dtype=np.float64).reshape(-1)
        d[:df.size] = df
    m.d_form[:] = d.tolist()
    m.mass = p["mass"]
    m.inertia[:] = [float(v) for v in p["inertia"]]
    m.dt = p["dt"]
    m.gravity = p["gravity"]
    m.foot[:] = [float(v) for v in np.asarray(p["foot"]).reshape(12)]
    m.mu_fric = p["mu_fric"]
    m.bar_mu = p["bar_mu"]
    m.bar_delta = p["bar_delta"]
    m.W[:] = [float(v) for v in p["W"]]
    m.Wu[:] = [float(v) for v in p["Wu"]]
    m.WN[:] = [float(v) for v in p["WN"]]
    return m


_lib.pdilqr_status_string.restype = ctypes.c_char_p
_lib.pdilqr_status_string.argtypes = [ctypes.c_int]
_lib.pdilqr_plan_create.argtypes = [ctypes.POINTER(_Batch), ctypes.POINTER(_Opts), ctypes.POINTER(_vp)]
_lib.pdilqr_plan_destroy.argtypes = [_vp]
_lib.pdilqr_plan_warps.argtypes = [_vp]
_lib.pdilqr_plan_warps.restype = ctypes.c_int32
_lib.pdilqr_plan_set_debug.argtypes = [_vp, ctypes.c_int32]
DEBUG_TC_SKIP_ISSUE = 1
DEBUG_BULK_SKIP_ISSUE = 2
DEBUG_SPLIT_SKIP_ARRIVE = 4
for _f in ("pdilqr_kkt_scan_solve", "pdilqr_riccati_solve"):
    getattr(_lib, _f).argtypes = [_vp, ctypes.POINTER(_LQ), _vp, ctypes.POINTER(_KktOut), _vp]
_lib.pdilqr_kkt_residual.argtypes = [_vp, ctypes.POINTER(_LQ), _vp, _vp, _vp, _vp, _vp, _vp]
_lib.pdilqr_linearize.argtypes = [_vp, ctypes.POINTER(SrbdModel), ctypes.POINTER(_Traj),
                                  ctypes.POINTER(_LQOut), _vp]
_lib.pdilqr_merit_eval.argtypes = [_vp, ctypes.POINTER(SrbdModel), ctypes.POINTER(_Traj),
                                   _vp, _vp, _vp, _vp, _vp]
_lib.pdilqr_solve.argtypes = [_vp, ctypes.POINTER(SrbdModel), ctypes.POINTER(_SqpOpts),
                              _vp, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(_SqpInfo), _vp]
_lib.pdilqr_solve_capture.argtypes = [_vp, ctypes.POINTER(SrbdModel), ctypes.POINTER(_SqpOpts),
                                      _vp, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(_SqpInfo)]
_lib.pdilqr_plan_replay.argtypes = [_vp, _vp]


_lib.pdilqr_kkt_scan_solve_noalloc.argtypes = [
    ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, _vp, _vp, ctypes.c_int32,
    ctypes.POINTER(_LQ), _vp, _vp, _vp, _vp, _vp, _vp]
_lib.pdilqr_noalloc_capacity_stages.argtypes = [ctypes.c_int32, ctypes.c_int32]
_lib.pdilqr_noalloc_capacity_stages.restype = ctypes.c_int64
_lib.pdilqr_peak_probe.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_double)]

PEAK_FFMA, PEAK_DFMA, PEAK_TF32_MMA = 0, 1, 2


def peak_probe(kind: int, reps: int = 3) -> tuple[float, float]:
    """Measured peak rate of one pipe on the current device (pdilqr_peak_probe):
    (TFLOP/s, ms of the best launch)."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _check(_lib.pdilqr_peak_probe(int(kind), int(reps), ctypes.byref(tf), ctypes.byref(ms)),
           "pdilqr_peak_probe")
    return tf.value, ms.value


def noalloc_capacity_stages(n: int, m: int) -> int:
    """Stage slots the static workspace of the allocation-free solve holds."""
    return int(_lib.pdilqr_noalloc_capacity_stages(int(n), int(m)))


def kkt_scan_solve_noalloc(n, m, N_dev, stage_off_dev, total_stages, lq: dict, s, dx, du, dlam,
                           status, warps=0, stream=None):
    """Allocation-free LQ KKT scan solve (pdilqr_kkt_scan_solve_noalloc).

    For callers that must not allocate device memory (a real-time loop, a
    stream being captured, a host whose pool owns the GPU): every array is
    the caller's, the batch tables ``N_dev`` (int32) and ``stage_off_dev``
    (int64) are device tensors, and the workspace is the library's static
    device array.  Calls that overlap on the GPU race.
    """
    lqs = _LQ(*[_ptr(lq.get(k), name=k) if (k != "S" or lq.get("S") is not None) else None
                for k in ("A", "B", "c", "Q", "R", "S", "q", "r")])
    _check(_lib.pdilqr_kkt_scan_solve_noalloc(
        int(n), int(m), int(N_dev.numel()), int(total_stages), _ptr(N_dev, torch.int32, "N"),
        _ptr(stage_off_dev, torch.int64, "stage_off"), int(warps), ctypes.byref(lqs),
        _ptr(s, name="s"), _ptr(dx, name="dx"), _ptr(du, name="du"), _ptr(dlam, name="dlam"),
        _ptr(status, torch.int32, "status"), _stream(stream)), "pdilqr_kkt_scan_solve_noalloc")


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

    def __init__(self, n: int, m: int, N, stage_off, warps: int = 0, refine: bool = False,
                 inst_per_cta: int = 0, m_fp64: bool = False, split: bool = False):
        self.n, self.m = int(n), int(m)
        self.N = np.ascontiguousarray(np.asarray(N, dtype=np.int32))
        self.stage_off = np.ascontiguousarray(np.asarray(stage_off, dtype=np.int64))
        self.count = int(self.N.size)
        self.total = int((self.stage_off + self.N + 1).max())
        b = _Batch(self.n, self.m, self.count, self.N.ctypes.data, self.stage_off.ctypes.data)
        o = _Opts(int(warps), int(bool(refine)), int(inst_per_cta), int(bool(m_fp64)), int(bool(split)))
        h = _vp()
        _check(_lib.pdilqr_plan_create(ctypes.byref(b), ctypes.byref(o), ctypes.byref(h)),
               "pdilqr_plan_create")
        self._h = h
        self.warps = int(_lib.pdilqr_plan_warps(h))
        self.inst_per_cta = int(inst_per_cta)

    def set_debug(self, flags: int):
        """Test switches of the plan (``DEBUG_TC_SKIP_ISSUE``,
        ``DEBUG_BULK_SKIP_ISSUE``, ``DEBUG_SPLIT_SKIP_ARRIVE``); 0 clears them."""
        _check(_lib.pdilqr_plan_set_debug(self._h, int(flags)), "pdilqr_plan_set_debug")

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


    # ------------------------------------------------------- SRBD model
    def _traj(self, traj: dict) -> _Traj:
        return _Traj(_ptr(traj["x"], name="x"), _ptr(traj["u"], name="u"),
                     _ptr(traj.get("lam"), name="lam"), _ptr(traj["xref"], name="xref"),
                     _ptr(traj["uref"], name="uref"),
                     _ptr(traj["contact"], torch.uint8, "contact"))

    def linearize(self, model: SrbdModel, traj: dict, out: dict | None = None, stream=None) -> dict:
        T, n, m = self.total, self.n, self.m
        if out is None:
            f = dict(device=traj["x"].device, dtype=torch.float32)
            out = {"A": torch.empty(T, n, n, **f), "B": torch.empty(T, n, m, **f),
                   "c": torch.empty(T, n, **f), "Q": torch.empty(T, n, n, **f),
                   "R": torch.empty(T, m, m, **f), "S": torch.empty(T, m, n, **f),
                   "q": torch.empty(T, n, **f), "r": torch.empty(T, m, **f)}
        lo = _LQOut(*[_ptr(out.get(k), name=k) for k in ("A", "B", "c", "Q", "R", "S", "q", "r")])
        _check(_lib.pdilqr_linearize(self._h, ctypes.byref(model), ctypes.byref(self._traj(traj)),
                                     ctypes.byref(lo), _stream(stream)), "pdilqr_linearize")
        return out

    def merit_eval(self, model: SrbdModel, traj: dict, x0hat, dx, du, out=None, stream=None):
        if out is None:
            out = torch.zeros(self.count, 24, device=dx.device, dtype=torch.float64)
        _check(_lib.pdilqr_merit_eval(self._h, ctypes.byref(model), ctypes.byref(self._traj(traj)),
                                      _ptr(x0hat, name="x0hat"), _ptr(dx, name="dx"),
                                      _ptr(du, name="du"), _ptr(out, torch.float64, "merit"),
                                      _stream(stream)), "pdilqr_merit_eval")
        return out

    def solve(self, model: SrbdModel, x0hat, x, u, lam, xref, uref, contact, max_iters=10,
              tol_step=0.0, tol_theta=0.0, c_armijo=1e-4, theta_frac=1e-2, alpha_replay=None,
              info: dict | None = None, stream=None, capture: bool = False) -> dict:
        """Run the fused SQP in place on (x, u, lam); returns the info tensors.
        With ``capture`` the solve is captured into the plan's graph instead."""
        dev = x.device
        if info is None:
            info = {"iters": torch.zeros(self.count, device=dev, dtype=torch.int32),
                    "status": torch.full((self.count,), -1, device=dev, dtype=torch.int32),
                    "alpha": torch.zeros(self.count, max_iters, device=dev, dtype=torch.float32),
                    "J": torch.zeros(self.count, device=dev, dtype=torch.float64),
                    "theta": torch.zeros(self.count, device=dev, dtype=torch.float64)}
        o = _SqpOpts(int(max_iters), float(tol_step), float(tol_theta), float(c_armijo),
                     float(theta_frac), _ptr(alpha_replay, name="alpha_replay"))
        inf = _SqpInfo(_ptr(info["iters"], torch.int32, "iters"),
                       _ptr(info["status"], torch.int32, "status"),
                       _ptr(info.get("alpha"), name="alpha"),
                       _ptr(info.get("J"), torch.float64, "J"),
                       _ptr(info.get("theta"), torch.float64, "theta"))
        args = (_ptr(x0hat, name="x0hat"), _ptr(x, name="x"), _ptr(u, name="u"),
                _ptr(lam, name="lam"), _ptr(xref, name="xref"), _ptr(uref, name="uref"),
                _ptr(contact, torch.uint8, "contact"), ctypes.byref(inf))
        if capture:
            _check(_lib.pdilqr_solve_capture(self._h, ctypes.byref(model), ctypes.byref(o), *args),
                   "pdilqr_solve_capture")
        else:
            _check(_lib.pdilqr_solve(self._h, ctypes.byref(model), ctypes.byref(o), *args,
                                     _stream(stream)), "pdilqr_solve")
        return info

    def capture(self, *args, **kw) -> dict:
        """Capture ``solve`` with these arguments into the plan's CUDA graph
        (pdilqr_solve_capture; nothing runs); ``replay`` launches it."""
        kw.pop("stream", None)
        return self.solve(*args, capture=True, **kw)

    def replay(self, stream=None):
        """Launch the plan's captured solve (pdilqr_plan_replay)."""
        _check(_lib.pdilqr_plan_replay(self._h, _stream(stream)), "pdilqr_plan_replay")


# ------------------------------------------------------------------ serving
class _ServeOpts(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("max_batch", ctypes.c_int32),
                ("max_inflight", ctypes.c_int32), ("max_N", ctypes.c_int32),
                ("sqp_iters", ctypes.c_int32), ("warps", ctypes.c_int32),
                ("batch_window_us", ctypes.c_int32), ("model", SrbdModel),
                ("class_models", ctypes.POINTER(SrbdModel)), ("hbm_reserve_bytes", ctypes.c_int64),
                ("large_cta_budget", ctypes.c_int32), ("split_min_robots", ctypes.c_int32),
                ("split_max_batch", ctypes.c_int32)]

SERVE_NROB = (1, 2, 4, 8, 16)   # the server's size classes (robots per client)


class _Request(ctypes.Structure):
    _fields_ = [("nrob", ctypes.c_int32), ("N", ctypes.c_int32), ("reset", ctypes.c_int32),
                ("x0hat", _vp), ("xref", _vp), ("uref", _vp), ("contact", _vp)]


class _Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32),
                ("latency_ns", ctypes.c_int64), ("u0", _vp), ("x", _vp), ("u", _vp)]


class _ServeStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("submitted", "completed", "refused", "batches",
                                              "clients", "pool_bytes_used", "pool_bytes_total")] + \
               [(k, ctypes.c_double) for k in ("mean_batch", "p50_latency_us", "p99_latency_us",
                                               "solves_per_s")]


_lib.pdilqr_serve_create.argtypes = [ctypes.POINTER(_ServeOpts), ctypes.POINTER(_vp)]
_lib.pdilqr_serve_submit.argtypes = [_vp, ctypes.c_uint64, ctypes.POINTER(_Request),
                                     ctypes.POINTER(ctypes.c_uint64)]
_lib.pdilqr_serve_poll.argtypes = [_vp, ctypes.c_uint64, ctypes.POINTER(_Result), ctypes.c_int64]
_lib.pdilqr_serve_release.argtypes = [_vp, ctypes.c_uint64]
_lib.pdilqr_serve_snapshot.argtypes = [_vp, ctypes.c_uint64, _vp, _vp, _vp]
_lib.pdilqr_serve_restore.argtypes = [_vp, ctypes.c_uint64, _vp, _vp, _vp]
_lib.pdilqr_serve_stats.argtypes = [_vp, ctypes.POINTER(_ServeStats)]
_lib.pdilqr_serve_destroy.argtypes = [_vp]


def _hptr(a, dtype):
    """Host pointer of a contiguous numpy array of ``dtype`` (kept alive by the caller)."""
    if a is None:
        return None, None
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data


class Server:
    """Continuous-batching MPC server (pdilqr_serve_*) on the current device."""

    def __init__(self, model_params: dict, hbm_budget_bytes: int = 1 << 30, max_batch: int = 1024,
                 max_inflight: int = 2, max_N: int = 100, sqp_iters: int = 1, warps: int = 8,
                 batch_window_us: int = 0, class_params: dict | None = None,
                 hbm_reserve_bytes: int = 0, large_cta_budget: int = 0,
                 split_min_robots: int = 0, split_max_batch: int = 0):
        """``class_params`` optionally maps a robot count (1, 2, 4, 8, 16) to the
        model constants of that class (formation offsets differ per count);
        classes it does not name use ``model_params``.  ``hbm_reserve_bytes``:
        device memory the free-memory admission check keeps free (0: 256 MiB).
        ``large_cta_budget``: most instances of 4+ robots in flight (0: none).
        ``split_min_robots``: classes of at least this many robots (4, 8, 16) run
        the split scan, 16 CTAs per instance, one such batch in flight (0: none);
        ``split_max_batch``: most instances of one split batch (0: 8; 16 per
        instance may not exceed the SM count)."""
        cm = None
        if class_params is not None:
            cm = (SrbdModel * len(SERVE_NROB))(
                *[srbd_model(class_params.get(r, model_params)) for r in SERVE_NROB])
        o = _ServeOpts(int(hbm_budget_bytes), int(max_batch), int(max_inflight), int(max_N),
                       int(sqp_iters), int(warps), int(batch_window_us), srbd_model(model_params),
                       ctypes.cast(cm, ctypes.POINTER(SrbdModel)) if cm is not None else None,
                       int(hbm_reserve_bytes), int(large_cta_budget), int(split_min_robots),
                       int(split_max_batch))
        h = _vp()
        _check(_lib.pdilqr_serve_create(ctypes.byref(o), ctypes.byref(h)), "pdilqr_serve_create")
        self._h = h

    def submit(self, client: int, nrob: int, N: int, x0hat, xref=None, uref=None, contact=None,
               reset: bool = False) -> int:
        keep = [_hptr(x0hat, np.float32), _hptr(xref, np.float32), _hptr(uref, np.float32),
                _hptr(contact, np.uint8)]
        q = _Request(int(nrob), int(N), int(bool(reset)), *[k[1] for k in keep])
        t = ctypes.c_uint64()
        _check(_lib.pdilqr_serve_submit(self._h, ctypes.c_uint64(client), ctypes.byref(q),
                                        ctypes.byref(t)), "pdilqr_serve_submit")
        return int(t.value)

    def poll(self, ticket: int, timeout_us: int = 10_000_000, n: int | None = None,
             N: int | None = None) -> dict:
        """Wait for a ticket.  With ``n`` and ``N`` the trajectories are returned."""
        out = {}
        bufs = {}
        if n is not None:
            bufs["u0"] = np.zeros(n, np.float32)
            if N is not None:
                bufs["x"] = np.zeros((N + 1, n), np.float32)
                bufs["u"] = np.zeros((N + 1, n), np.float32)
        r = _Result(0, 0, 0, *[bufs[k].ctypes.data if k in bufs else None for k in ("u0", "x", "u")])
        _check(_lib.pdilqr_serve_poll(self._h, ctypes.c_uint64(ticket), ctypes.byref(r),
                                      int(timeout_us)), "pdilqr_serve_poll")
        out.update(status=r.status, iters=r.iters, latency_us=r.latency_ns / 1e3, **bufs)
        return out

    def release(self, client: int):
        _check(_lib.pdilqr_serve_release(self._h, ctypes.c_uint64(client)), "pdilqr_serve_release")

    def snapshot(self, client: int, n: int, N: int):
        x = np.zeros((N + 1, n), np.float32)
        u = np.zeros((N + 1, n), np.float32)
        lam = np.zeros((N + 1, n), np.float32)
        _check(_lib.pdilqr_serve_snapshot(self._h, ctypes.c_uint64(client), x.ctypes.data,
                                          u.ctypes.data, lam.ctypes.data), "pdilqr_serve_snapshot")
        return x, u, lam

    def restore(self, client: int, x, u, lam):
        k = [_hptr(v, np.float32) for v in (x, u, lam)]
        _check(_lib.pdilqr_serve_restore(self._h, ctypes.c_uint64(client), *[v[1] for v in k]),
               "pdilqr_serve_restore")

    def stats(self) -> dict:
        st = _ServeStats()
        _check(_lib.pdilqr_serve_stats(self._h, ctypes.byref(st)), "pdilqr_serve_stats")
        return {k: getattr(st, k) for k, _ in _ServeStats._fields_}

    def set_debug(self, flags: int):
        """Test switches of the plan (``DEBUG_TC_SKIP_ISSUE``); 0 clears them."""
        _check(_lib.pdilqr_plan_set_debug(self._h, int(flags)), "pdilqr_plan_set_debug")

    def close(self):
        if getattr(self, "_h", None):
            _lib.pdilqr_serve_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def backward_error(resid: torch.Tensor) -> torch.Tensor:
    """Normwise backward error |Kz - rhs| / (|K| |z| + |rhs|) per instance."""
    r = resid.double()
    return r[:, 0] / (r[:, 1] * r[:, 2] + r[:, 3])
