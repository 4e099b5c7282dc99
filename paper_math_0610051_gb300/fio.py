"""Python binding of libfio.so (include/fio.h): argument marshalling only.

Every step of the apply path runs in the library's CUDA kernels; PyTorch only
supplies device memory and the current stream.  There is no CPU fallback: if
the library is missing, every call raises ``FioError``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libfio.so")

FIO_OK, FIO_EINVAL, FIO_ENOMEM, FIO_ECUDA, FIO_ERANK, FIO_ETIMEOUT, FIO_EUNSUPPORTED = range(7)
PHASE_SHIFT_WAVE, PHASE_ELLIPSE, PHASE_TAU_MODES, PHASE_ELLIPSE_PRODUCT = 0, 1, 2, 3
AMP_ONE, AMP_SEPARABLE, AMP_HANKEL = 0, 1, 2
MIXED, FP64 = 0, 1
ALPHA_STORED, ALPHA_RECOMPUTE = 0, 1


class FioError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class _Phase(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("nmodes", ctypes.c_int),
                ("params", ctypes.POINTER(ctypes.c_double))]


class _Amp(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("a1", ctypes.c_double), ("a2", ctypes.c_double)]


class _Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("L", ctypes.c_int), ("sigma", ctypes.c_double),
                ("kb_width", ctypes.c_int), ("seed", ctypes.c_ulonglong), ("r0", ctypes.c_int),
                ("rank_cap", ctypes.c_int), ("max_batch", ctypes.c_int),
                ("surrogate", ctypes.c_void_p), ("surrogate_warp_budget", ctypes.c_double),
                ("sep_cut", ctypes.c_double), ("sep_target", ctypes.c_double),
                ("alpha_mode", ctypes.c_int), ("alpha_group", ctypes.c_int)]


class _SurInfo(ctypes.Structure):
    _fields_ = [("nparams", ctypes.c_int), ("nsamples", ctypes.c_int), ("epochs", ctypes.c_int),
                ("steps", ctypes.c_longlong), ("train_seconds", ctypes.c_double),
                ("final_loss", ctypes.c_double), ("tau_scale", ctypes.c_double),
                ("dx_scale", ctypes.c_double), ("heldout_tau_maxerr", ctypes.c_double),
                ("heldout_dx_maxerr", ctypes.c_double), ("heldout_dtheta_maxerr", ctypes.c_double),
                ("heldout_tau_relrms", ctypes.c_double)]


class _PlanInfo(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("L", ctypes.c_int), ("precision", ctypes.c_int),
                ("kb_width", ctypes.c_int), ("max_batch", ctypes.c_int),
                ("sigma", ctypes.c_double), ("kb_beta", ctypes.c_double), ("eps", ctypes.c_double),
                ("q_max", ctypes.c_int), ("q_min", ctypes.c_int), ("r_max", ctypes.c_int),
                ("q_mean", ctypes.c_double),
                ("bytes_alpha", ctypes.c_ulonglong), ("bytes_beta", ctypes.c_ulonglong),
                ("bytes_warp", ctypes.c_ulonglong), ("bytes_grid", ctypes.c_ulonglong),
                ("bytes_total", ctypes.c_ulonglong), ("grid_points", ctypes.c_ulonglong),
                ("alg_bytes_apply", ctypes.c_ulonglong), ("plan_seconds", ctypes.c_double),
                ("kernel_launches", ctypes.c_ulonglong), ("surrogate_warp", ctypes.c_int),
                ("surrogate_warp_cycles", ctypes.c_double),
                ("surrogate_residual_cycles", ctypes.c_double), ("max_bin_points", ctypes.c_int),
                ("mean_bin_points", ctypes.c_double), ("max_spread_candidates", ctypes.c_int),
                ("sep_error", ctypes.c_double), ("alpha_mode", ctypes.c_int),
                ("alpha_groups", ctypes.c_int), ("bytes_recompute", ctypes.c_ulonglong)]


class _WedgeInfo(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int * 4), ("xc1", ctypes.c_int), ("xc2", ctypes.c_int),
                ("b1", ctypes.c_int), ("n1", ctypes.c_int), ("b2", ctypes.c_int),
                ("n2", ctypes.c_int), ("m1", ctypes.c_int), ("m2", ctypes.c_int),
                ("q", ctypes.c_int), ("r", ctypes.c_int), ("npts", ctypes.c_int)]


# Every symbol include/fio.h declares (checked by the tests).
EXPORTS = [
    "fio_options_default", "fio_plan_create", "fio_apply", "fio_apply_real", "fio_apply_adjoint",
    "fio_apply_normal",
    "fio_apply_noalloc",
    "fio_plan_sync",
    "fio_plan_get_info", "fio_plan_get_wedge", "fio_plan_export_wedge", "fio_plan_export_warp",
    "fio_plan_destroy", "fio_plan_set_timing", "fio_plan_stage_times", "fio_plan_save", "fio_plan_load",
    "fio_dft2", "fio_default_wedges", "fio_wedge_map", "fio_wedge_geometry", "fio_kb_eval",
    "fio_kb_width_for", "fio_host_eigh", "fio_host_svd", "fio_host_svd_right", "fio_status_string", "fio_last_error", "fio_version",
    "fio_surrogate_train", "fio_surrogate_destroy", "fio_surrogate_get_info", "fio_surrogate_params",
    "fio_surrogate_eval", "fio_surrogate_loss_grad", "fio_surrogate_samples", "fio_surrogate_nparams",
]

_lib = None
_lock = threading.Lock()


def lib():
    """The loaded libfio.so; raises FioError if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise FioError(-1, f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
            L = ctypes.CDLL(LIB_PATH)
            P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
            L.fio_options_default.argtypes = [ctypes.POINTER(_Options)]
            L.fio_plan_create.argtypes = [I, ctypes.POINTER(_Phase), ctypes.POINTER(_Amp), D,
                                          ctypes.POINTER(_Options), ctypes.POINTER(P)]
            L.fio_apply.argtypes = [P, P, P, I, P]
            L.fio_apply_real.argtypes = [P, P, P, I, P]
            L.fio_apply_adjoint.argtypes = [P, P, P, I, P]
            L.fio_apply_normal.argtypes = [P, P, P, I, P]
            L.fio_apply_noalloc.argtypes = [P, P, P, I, P]
            L.fio_plan_sync.argtypes = [P, P]
            L.fio_plan_get_info.argtypes = [P, ctypes.POINTER(_PlanInfo)]
            L.fio_plan_get_wedge.argtypes = [P, I, ctypes.POINTER(_WedgeInfo)]
            L.fio_plan_export_wedge.argtypes = [P, I, P, P, P, P]
            L.fio_plan_export_warp.argtypes = [P, I, P]
            L.fio_plan_set_timing.argtypes = [P, I]
            L.fio_plan_stage_times.argtypes = [P, P, P]
            L.fio_plan_destroy.argtypes = [P]
            L.fio_plan_save.argtypes = [P, ctypes.c_char_p]
            L.fio_plan_load.argtypes = [ctypes.c_char_p, I, P]
            L.fio_plan_destroy.restype = None
            L.fio_dft2.argtypes = [I, I, P, P, I, I, P]
            L.fio_default_wedges.argtypes = [I]
            L.fio_wedge_map.argtypes = [I, I, P]
            L.fio_wedge_geometry.argtypes = [I, I, D, I, I, ctypes.POINTER(_WedgeInfo)]
            L.fio_kb_eval.argtypes = [I, D, I, P, P, P, P]
            L.fio_kb_width_for.argtypes = [D]
            L.fio_host_eigh.argtypes = [I, P, P, P]
            L.fio_host_svd.argtypes = [I, I, P, P, P, P]
            L.fio_host_svd_right.argtypes = [I, P, P, P]
            L.fio_surrogate_train.argtypes = [ctypes.POINTER(_Phase), I, I, I, ctypes.c_ulonglong,
                                              ctypes.POINTER(P)]
            L.fio_surrogate_destroy.argtypes = [P]
            L.fio_surrogate_destroy.restype = None
            L.fio_surrogate_get_info.argtypes = [P, ctypes.POINTER(_SurInfo)]
            L.fio_surrogate_params.argtypes = [P, P, I]
            L.fio_surrogate_eval.argtypes = [P, I, P, P, P]
            L.fio_surrogate_loss_grad.argtypes = [P, I, P, P, P, ctypes.POINTER(ctypes.c_double)]
            L.fio_surrogate_samples.argtypes = [ctypes.POINTER(_Phase), I, ctypes.c_ulonglong, P, P]
            L.fio_status_string.restype = ctypes.c_char_p
            L.fio_status_string.argtypes = [I]
            L.fio_last_error.restype = ctypes.c_char_p
            _lib = L
    return _lib


def _check(status: int, what: str):
    if status != FIO_OK:
        detail = lib().fio_last_error().decode(errors="replace")
        raise FioError(status, f"{what}: {detail}")


def _np_ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream_ptr(torch, device):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _wedge_dict(w: _WedgeInfo) -> dict:
    return {"M": list(w.M), "xc": (w.xc1, w.xc2), "b1": w.b1, "n1": w.n1, "b2": w.b2, "n2": w.n2,
            "m1": w.m1, "m2": w.m2, "q": w.q, "r": w.r, "npts": w.npts}


class Plan:
    """fio_plan_create / fio_apply / fio_apply_adjoint for one operator L.

    phase: one of PHASE_* with ``params`` (shift/wave: [x01, x02, c]; ellipse:
    [A1, B1, A2, B2]; tau modes: [K, 5] rows {a, k1, k2, m, p}; ellipse with
    product-form axes: [a1, s1, a2, s2]).
    amp: None (a = 1), (a1, a2) for a = (1 + a1 sin 2 pi x1)(1 + a2 cos theta), or
    ("hankel", s) for the Hankel amplitude of integration along ellipses (s = +1 or -1).
    """

    def __init__(self, N: int, phase: int, params, eps: float, amp=None, precision: str = "mixed",
                 L: int = 0, sigma: float = 0.0, kb_width: int = 0, seed: int = 0x5EED5EED,
                 r0: int = 0, rank_cap: int = 0, max_batch: int = 1, device=None,
                 surrogate: "Surrogate | None" = None, surrogate_warp_budget: float = 0.0,
                 sep_cut: float = 0.0, sep_target: float = 0.0, alpha_mode: str = "stored",
                 alpha_group: int = 0):
        import torch
        self._torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self._handle = ctypes.c_void_p()
        prm = np.ascontiguousarray(np.asarray(params, dtype=np.float64).ravel())
        self._params = prm
        ph = _Phase(int(phase), len(prm) // 5 if phase == PHASE_TAU_MODES else 0,
                    prm.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        if amp is None:
            am = _Amp(AMP_ONE, 0.0, 0.0)
        elif amp[0] == "hankel":
            am = _Amp(AMP_HANKEL, float(amp[1]), 0.0)
        else:
            am = _Amp(AMP_SEPARABLE, float(amp[0]), float(amp[1]))
        opt = _Options()
        lib().fio_options_default(ctypes.byref(opt))
        opt.precision = FP64 if precision in ("fp64", FP64) else MIXED
        opt.L, opt.sigma, opt.kb_width = int(L), float(sigma), int(kb_width)
        opt.seed, opt.r0, opt.rank_cap, opt.max_batch = int(seed), int(r0), int(rank_cap), int(max_batch)
        opt.surrogate = surrogate._handle if surrogate is not None else None
        opt.surrogate_warp_budget = float(surrogate_warp_budget)
        opt.sep_cut, opt.sep_target = float(sep_cut), float(sep_target)
        opt.alpha_mode = {"stored": ALPHA_STORED, "recompute": ALPHA_RECOMPUTE}.get(alpha_mode, alpha_mode)
        opt.alpha_group = int(alpha_group)
        self._surrogate = surrogate
        self.N = int(N)
        self.precision = opt.precision
        self.max_batch = max(1, int(max_batch))
        with torch.cuda.device(self.device):
            _check(lib().fio_plan_create(self.N, ctypes.byref(ph), ctypes.byref(am), float(eps),
                                         ctypes.byref(opt), ctypes.byref(self._handle)),
                   "fio_plan_create")
        self.dtype = torch.complex128 if self.precision == FP64 else torch.complex64

    # -- files
    def save(self, path: str):
        """fio_plan_save: write the plan to `path`."""
        with self._torch.cuda.device(self.device):
            _check(lib().fio_plan_save(self._handle, os.fsencode(path)), "fio_plan_save")

    @classmethod
    def load(cls, path: str, max_batch: int = 0, device=None) -> "Plan":
        """fio_plan_load: a plan rebuilt from `path` on `device` (default: current)."""
        import torch
        self = cls.__new__(cls)
        self._torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self._handle = ctypes.c_void_p()
        self._surrogate = None
        with torch.cuda.device(self.device):
            _check(lib().fio_plan_load(os.fsencode(path), int(max_batch), ctypes.byref(self._handle)),
                   "fio_plan_load")
        info = self.info()
        self.N, self.precision, self.max_batch = info["N"], info["precision"], info["max_batch"]
        self.dtype = torch.complex128 if self.precision == FP64 else torch.complex64
        return self

    # -- lifetime
    def close(self):
        if getattr(self, "_handle", None) and self._handle.value:
            lib().fio_plan_destroy(self._handle)
            self._handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- apply
    def _prep(self, x):
        torch = self._torch
        if not isinstance(x, torch.Tensor) or x.device != self.device:
            raise FioError(FIO_EINVAL, f"input must be a tensor on {self.device}")
        if x.dtype != self.dtype:
            raise FioError(FIO_EINVAL, f"input dtype must be {self.dtype}, got {x.dtype}")
        if x.shape[-2:] != (self.N, self.N):
            raise FioError(FIO_EINVAL, f"input must end with ({self.N}, {self.N})")
        # lazily conjugated / negated views keep unmodified memory: materialise them
        return x.resolve_conj().resolve_neg().contiguous()

    def _run(self, fn, x, out, what):
        torch = self._torch
        x = self._prep(x)
        batch = x.numel() // (self.N * self.N)
        if out is None:
            out = torch.empty_like(x)
        elif out.shape != x.shape or out.dtype != x.dtype or not out.is_contiguous():
            raise FioError(FIO_EINVAL, "out must be a contiguous tensor like the input")
        _check(fn(self._handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                  int(batch), _stream_ptr(torch, self.device)), what)
        return out

    def apply(self, f, out=None):
        """out = L f (fio_apply); f: complex tensor [..., N, N] on the plan's device.
        A real f (float32 for mixed plans, float64 for FP64) goes through
        fio_apply_real and gives the complex result of f + 0i."""
        torch = self._torch
        rdtype = torch.float64 if self.precision == FP64 else torch.float32
        if isinstance(f, torch.Tensor) and f.dtype == rdtype:
            if f.device != self.device or f.shape[-2:] != (self.N, self.N):
                raise FioError(FIO_EINVAL, f"input must be a tensor on {self.device} ending with "
                                           f"({self.N}, {self.N})")
            x = f.resolve_neg().contiguous()
            batch = x.numel() // (self.N * self.N)
            if out is None:
                out = torch.empty(x.shape, dtype=self.dtype, device=self.device)
            elif out.shape != x.shape or out.dtype != self.dtype or not out.is_contiguous():
                raise FioError(FIO_EINVAL, "out must be a contiguous complex tensor of f's shape")
            _check(lib().fio_apply_real(self._handle, ctypes.c_void_p(x.data_ptr()),
                                        ctypes.c_void_p(out.data_ptr()), int(batch),
                                        _stream_ptr(torch, self.device)), "fio_apply_real")
            return out
        return self._run(lib().fio_apply, f, out, "fio_apply")

    def adjoint(self, g, out=None):
        """out = L* g (fio_apply_adjoint)."""
        return self._run(lib().fio_apply_adjoint, g, out, "fio_apply_adjoint")

    def normal(self, f, out=None):
        """out = L* L f (fio_apply_normal)."""
        return self._run(lib().fio_apply_normal, f, out, "fio_apply_normal")

    def sync(self):
        _check(lib().fio_plan_sync(self._handle, _stream_ptr(self._torch, self.device)),
               "fio_plan_sync")

    # -- diagnostics
    STAGES = ["S0_dft", "S1_scatter", "S2_colfft", "S3_interp", "S4a_spread", "S4b_colfft",
              "S4b_rowfft", "S4c_gather", "S4d_idft"]

    def set_timing(self, on: bool = True):
        _check(lib().fio_plan_set_timing(self._handle, int(bool(on))), "fio_plan_set_timing")

    def stage_times(self) -> dict:
        """{stage: (total ms, executions)} since the previous call (synchronises)."""
        ms = np.zeros(len(self.STAGES))
        cnt = np.zeros(len(self.STAGES), np.int64)
        _check(lib().fio_plan_stage_times(self._handle, _np_ptr(ms), _np_ptr(cnt)),
               "fio_plan_stage_times")
        return {s: (float(ms[i]), int(cnt[i])) for i, s in enumerate(self.STAGES)}

    # -- introspection
    def info(self) -> dict:
        i = _PlanInfo()
        _check(lib().fio_plan_get_info(self._handle, ctypes.byref(i)), "fio_plan_get_info")
        return {k: getattr(i, k) for k, _ in _PlanInfo._fields_}

    def wedge(self, l: int) -> dict:
        w = _WedgeInfo()
        _check(lib().fio_plan_get_wedge(self._handle, int(l), ctypes.byref(w)), "fio_plan_get_wedge")
        return _wedge_dict(w)

    def export_wedge(self, l: int):
        """(alpha [q, N, N], beta [q, npts], k1 [npts], k2 [npts]) of wedge l, complex128."""
        w = self.wedge(l)
        q, n = w["q"], w["npts"]
        alpha = np.empty((q, self.N, self.N), np.complex128)
        beta = np.empty((q, n), np.complex128)
        k1 = np.empty(n, np.int32)
        k2 = np.empty(n, np.int32)
        _check(lib().fio_plan_export_wedge(self._handle, int(l), _np_ptr(alpha), _np_ptr(beta),
                                           _np_ptr(k1), _np_ptr(k2)), "fio_plan_export_wedge")
        return alpha, beta, k1, k2

    def export_warp(self, l: int) -> np.ndarray:
        """Warped points of wedge l: [N, N, 2] fractions y' = M^-T grad Phi mod 1."""
        y = np.empty((self.N, self.N, 2), np.float64)
        _check(lib().fio_plan_export_warp(self._handle, int(l), _np_ptr(y)), "fio_plan_export_warp")
        return y


def _tau_phase(modes):
    prm = np.ascontiguousarray(np.asarray(modes, np.float64).ravel())
    return prm, _Phase(PHASE_TAU_MODES, len(prm) // 5, prm.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))


class Surrogate:
    """fio_surrogate_*: the BF16 MLP surrogate of a tau-mode phase, trained on the GPU."""

    def __init__(self, modes, nsamples: int = 1 << 20, epochs: int = 20, batch: int = 8192,
                 seed: int = 1):
        import torch
        self._torch = torch
        self._prm, ph = _tau_phase(modes)
        self._handle = ctypes.c_void_p()
        _check(lib().fio_surrogate_train(ctypes.byref(ph), int(nsamples), int(epochs), int(batch),
                                         int(seed), ctypes.byref(self._handle)),
               "fio_surrogate_train")

    def close(self):
        if getattr(self, "_handle", None) and self._handle.value:
            lib().fio_surrogate_destroy(self._handle)
            self._handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        i = _SurInfo()
        _check(lib().fio_surrogate_get_info(self._handle, ctypes.byref(i)), "fio_surrogate_get_info")
        return {k: getattr(i, k) for k, _ in _SurInfo._fields_}

    def params(self) -> np.ndarray:
        out = np.empty(lib().fio_surrogate_nparams(), np.float32)
        _check(lib().fio_surrogate_params(self._handle, _np_ptr(out), 0), "fio_surrogate_params")
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        _check(lib().fio_surrogate_params(self._handle, _np_ptr(p), 1), "fio_surrogate_params")

    def eval(self, x4):
        """x4: CUDA float32 [n, 4] -> [n, 4] (tau, d1 tau, d2 tau, d_theta tau)."""
        torch = self._torch
        x4 = x4.contiguous()
        y = torch.empty_like(x4)
        _check(lib().fio_surrogate_eval(self._handle, x4.shape[0], ctypes.c_void_p(x4.data_ptr()),
                                        ctypes.c_void_p(y.data_ptr()),
                                        _stream_ptr(torch, x4.device)), "fio_surrogate_eval")
        return y

    def loss_grad(self, x4, t3):
        torch = self._torch
        g = torch.empty(lib().fio_surrogate_nparams(), dtype=torch.float32, device=x4.device)
        loss = ctypes.c_double()
        torch.cuda.synchronize()
        _check(lib().fio_surrogate_loss_grad(self._handle, x4.shape[0],
                                             ctypes.c_void_p(x4.contiguous().data_ptr()),
                                             ctypes.c_void_p(t3.contiguous().data_ptr()),
                                             ctypes.c_void_p(g.data_ptr()), ctypes.byref(loss)),
               "fio_surrogate_loss_grad")
        return loss.value, g


def surrogate_samples(modes, n: int, seed: int = 1):
    """The plain-evaluation training samples: (x4 float32 [n,4], t4 float64 [n,4]) on the GPU."""
    import torch
    prm, ph = _tau_phase(modes)
    x4 = torch.empty(n, 4, dtype=torch.float32, device="cuda")
    t4 = torch.empty(n, 4, dtype=torch.float64, device="cuda")
    _check(lib().fio_surrogate_samples(ctypes.byref(ph), int(n), int(seed),
                                       ctypes.c_void_p(x4.data_ptr()), ctypes.c_void_p(t4.data_ptr())),
           "fio_surrogate_samples")
    return x4, t4


def dft2(x, inverse: bool = False, out=None):
    """Unitary 2D DFT of Eq. dft on the GPU (fio_dft2); spectrum in centred order."""
    import torch
    if x.dtype not in (torch.complex64, torch.complex128) or not x.is_cuda:
        raise FioError(FIO_EINVAL, "dft2 needs a complex CUDA tensor")
    x = x.resolve_conj().resolve_neg().contiguous()
    N = x.shape[-1]
    if out is None:
        out = torch.empty_like(x)
    prec = FP64 if x.dtype == torch.complex128 else MIXED
    _check(lib().fio_dft2(N, prec, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                          x.numel() // (N * N), int(bool(inverse)), _stream_ptr(torch, x.device)),
           "fio_dft2")
    return out


# ---------------------------------------------------------------- host utils --

def default_wedges(N: int) -> int:
    return lib().fio_default_wedges(int(N))


def kb_width_for(eps: float) -> int:
    return lib().fio_kb_width_for(float(eps))


def wedge_map(N: int, L: int) -> np.ndarray:
    out = np.empty((N, N), np.int32)
    _check(lib().fio_wedge_map(int(N), int(L), _np_ptr(out)), "fio_wedge_map")
    return out


def wedge_geometry(N: int, L: int, sigma: float, kb_width: int, l: int) -> dict:
    w = _WedgeInfo()
    _check(lib().fio_wedge_geometry(int(N), int(L), float(sigma), int(kb_width), int(l),
                                    ctypes.byref(w)), "fio_wedge_geometry")
    return _wedge_dict(w)


def kb_eval(w: int, beta: float, s=None, nu=None):
    s = np.ascontiguousarray(np.zeros(0) if s is None else s, np.float64)
    nu = np.ascontiguousarray(np.zeros(len(s)) if nu is None else nu, np.float64)
    n = max(len(s), len(nu))
    if len(s) < n:
        s = np.zeros(n)
    phi, phihat = np.empty(n), np.empty(n)
    _check(lib().fio_kb_eval(int(w), float(beta), n, _np_ptr(s), _np_ptr(phi), _np_ptr(nu),
                             _np_ptr(phihat)), "fio_kb_eval")
    return phi, phihat


def host_eigh(A: np.ndarray):
    A = np.ascontiguousarray(A, np.complex128)
    n = A.shape[0]
    ev = np.empty(n)
    V = np.empty((n, n), np.complex128)
    _check(lib().fio_host_eigh(n, _np_ptr(A), _np_ptr(ev), _np_ptr(V)), "fio_host_eigh")
    return ev, V


def host_svd(A: np.ndarray):
    """(s, AV, V) of fio_host_svd: A V = AV, s descending, AV's columns s_j u_j."""
    A = np.ascontiguousarray(A, np.complex128)
    m, n = A.shape
    s = np.empty(n)
    AV = np.empty((m, n), np.complex128)
    V = np.empty((n, n), np.complex128)
    _check(lib().fio_host_svd(m, n, _np_ptr(A), _np_ptr(s), _np_ptr(AV), _np_ptr(V)), "fio_host_svd")
    return s, AV, V


def host_svd_right(R: np.ndarray):
    """(s, V) of fio_host_svd_right: singular values and right singular vectors."""
    R = np.ascontiguousarray(R, np.complex128)
    n = R.shape[0]
    s = np.empty(n)
    V = np.empty((n, n), np.complex128)
    _check(lib().fio_host_svd_right(n, _np_ptr(R), _np_ptr(s), _np_ptr(V)), "fio_host_svd_right")
    return s, V


def __getattr__(name):
    """fio.FIOApply / fio.FIOAdjoint: the autograd functions of autograd.py, imported
    on first use (they need torch, which this module imports only with a plan)."""
    if name in ("FIOApply", "FIOAdjoint", "fio_apply", "fio_adjoint"):
        from . import autograd
        return getattr(autograd, name)
    raise AttributeError(f"module {__name__!r} has no attribute {name!r}")
