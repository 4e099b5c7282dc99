"""FP64 CPU oracle for the discrete Fourier integral operator (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` leg of
``bench.py`` may import this module.  It wraps ``fio_oracle.c`` (plain C, FP64,
OpenMP), which evaluates the definitions literally:

* Eq. dft  (Sec. 1.2): fhat(xi) = (1/N) sum_x exp(-2 pi i x.xi) f(x)
* Eq. dfio (Sec. 1.2): (Lf)(x) = (1/N) sum_xi a(x,xi) exp(2 pi i Phi(x,xi)) fhat(xi)
* Sec. 3.5: (L*g)^(xi) = (1/N) sum_y conj(a) exp(-2 pi i Phi(y,xi)) g(y), then
  the inverse DFT.

It shares no code with the CUDA library.  Arrays are numpy complex128;
``fhat`` is in centred order, ``fhat[k1 + N/2, k2 + N/2]``.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fio_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# phase kinds of fio_oracle.c
SHIFT_WAVE, ELLIPSE, TAU_MODES, ELLIPSE_PRODUCT = 0, 1, 2, 3
AMP_ONE, AMP_SEPARABLE, AMP_HANKEL = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile fio_oracle.c into liboracle.so next to it (gcc, -O2, OpenMP)."""
    stamp = _LIB + ".arch"
    if not os.path.exists(stamp) or open(stamp).read().strip() != platform.machine():
        force = True  # built on another machine
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", _SRC,
                               "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
        with open(stamp, "w") as fh:
            fh.write(platform.machine())
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i, d = ctypes.c_int, ctypes.c_double
            lib.or_num_threads.restype = i
            lib.or_dft2.argtypes = [i, P, P]
            lib.or_idft2.argtypes = [i, P, P]
            lib.or_phase_eval.argtypes = [i, i, P, i, i, P, P, P, P, P]
            lib.or_amp_eval.argtypes = [i, d, d, i, P, P, P, P]
            lib.or_apply_points.argtypes = [i, i, i, P, i, i, d, d, P, i, P, P, P]
            lib.or_apply_dense.argtypes = [i, i, i, P, i, i, d, d, P, P]
            lib.or_adjoint_hat_points.argtypes = [i, i, i, P, i, i, d, d, P, i, P, P, P]
            lib.or_adjoint_dense.argtypes = [i, i, i, P, i, i, d, d, P, P]
            lib.or_matrix.argtypes = [i, i, i, P, i, i, d, d, P]
            lib.or_tau_eval.argtypes = [i, P, i, P, P, P, P]
            _lib = lib
    return _lib


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class Phase:
    """A phase Phi(x, xi) = x.xi + Psi(x, xi) given by kind and plain parameters."""

    def __init__(self, kind: int, params, grouped: bool = True):
        self.kind = int(kind)
        self.params = _c(np.asarray(params, dtype=np.float64).ravel(), np.float64)
        self.nmodes = len(self.params) // 5 if self.kind == TAU_MODES else 0
        self.grouped = bool(grouped)

    def args(self):
        return (self.kind, self.nmodes, _p(self.params), int(self.grouped))


class Amplitude:
    def __init__(self, kind: int = 0, a1: float = 0.0, a2: float = 0.0):
        self.kind, self.a1, self.a2 = int(kind), float(a1), float(a2)

    def args(self):
        return (self.kind, self.a1, self.a2)


def num_threads() -> int:
    return _load().or_num_threads()


def dft2(f: np.ndarray) -> np.ndarray:
    """Unitary 2D DFT of Eq. dft; returns fhat in centred order."""
    N = f.shape[-1]
    f = _c(f, np.complex128)
    out = np.empty((N, N), np.complex128)
    _load().or_dft2(N, _p(f), _p(out))
    return out


def idft2(fhat: np.ndarray) -> np.ndarray:
    """Inverse of Eq. dft from centred fhat."""
    N = fhat.shape[-1]
    fhat = _c(fhat, np.complex128)
    out = np.empty((N, N), np.complex128)
    _load().or_idft2(N, _p(fhat), _p(out))
    return out


def phase_eval(phase: Phase, x1, x2, k1, k2) -> np.ndarray:
    x1, x2 = _c(x1, np.float64), _c(x2, np.float64)
    k1, k2 = _c(k1, np.int32), _c(k2, np.int32)
    out = np.empty(len(x1), np.float64)
    _load().or_phase_eval(*phase.args(), len(x1), _p(x1), _p(x2), _p(k1), _p(k2), _p(out))
    return out


def amp_eval(amp: Amplitude, x1, k1, k2, psi=None) -> np.ndarray:
    """a(x, xi) (complex); psi = Phi - x.xi at the same points is read by the
    Hankel kind only."""
    x1, k1, k2 = _c(x1, np.float64), _c(k1, np.int32), _c(k2, np.int32)
    ps = _c(np.zeros(len(x1)) if psi is None else psi, np.float64)
    out = np.empty(len(x1), np.complex128)
    _load().or_amp_eval(*amp.args(), len(x1), _p(x1), _p(k1), _p(k2), _p(ps), _p(out))
    return out


def apply_points(phase: Phase, amp: Amplitude, fhat: np.ndarray, n1, n2) -> np.ndarray:
    """(Lf)(x_i) of Eq. dfio at x_i = (n1_i, n2_i)/N from centred fhat."""
    N = fhat.shape[-1]
    fhat = _c(fhat, np.complex128)
    n1, n2 = _c(n1, np.int32), _c(n2, np.int32)
    out = np.empty(len(n1), np.complex128)
    _load().or_apply_points(N, *phase.args(), *amp.args(), _p(fhat), len(n1), _p(n1), _p(n2),
                            _p(out))
    return out


def apply_dense(phase: Phase, amp: Amplitude, f: np.ndarray) -> np.ndarray:
    """(Lf) on the whole N x N grid, O(N^4)."""
    N = f.shape[-1]
    f = _c(f, np.complex128)
    out = np.empty((N, N), np.complex128)
    _load().or_apply_dense(N, *phase.args(), *amp.args(), _p(f), _p(out))
    return out


def adjoint_hat_points(phase: Phase, amp: Amplitude, g: np.ndarray, k1, k2) -> np.ndarray:
    """(L*g)^(xi_j) of Sec. 3.5 at xi_j = (k1_j, k2_j), -N/2 <= k < N/2."""
    N = g.shape[-1]
    g = _c(g, np.complex128)
    k1, k2 = _c(k1, np.int32), _c(k2, np.int32)
    out = np.empty(len(k1), np.complex128)
    _load().or_adjoint_hat_points(N, *phase.args(), *amp.args(), _p(g), len(k1), _p(k1), _p(k2),
                                  _p(out))
    return out


def adjoint_dense(phase: Phase, amp: Amplitude, g: np.ndarray) -> np.ndarray:
    """(L*g) on the whole grid, O(N^4)."""
    N = g.shape[-1]
    g = _c(g, np.complex128)
    out = np.empty((N, N), np.complex128)
    _load().or_adjoint_dense(N, *phase.args(), *amp.args(), _p(g), _p(out))
    return out


def matrix(phase: Phase, amp: Amplitude, N: int) -> np.ndarray:
    """Dense N^2 x N^2 matrix of L (tiny N only: O(N^6))."""
    out = np.empty((N * N, N * N), np.complex128)
    _load().or_matrix(N, *phase.args(), *amp.args(), _p(out))
    return out


def tau_eval(modes, x1, x2, theta) -> np.ndarray:
    """[n, 4]: tau, d tau/d x1, d tau/d x2, d tau/d theta of the tau-mode phase."""
    modes = _c(np.asarray(modes, np.float64).ravel(), np.float64)
    x1, x2, theta = _c(x1, np.float64), _c(x2, np.float64), _c(theta, np.float64)
    out = np.empty((len(x1), 4), np.float64)
    _load().or_tau_eval(len(modes) // 5, _p(modes), len(x1), _p(x1), _p(x2), _p(theta), _p(out))
    return out


def rel_l2(ref: np.ndarray, approx: np.ndarray) -> float:
    """sqrt(sum |ref - approx|^2 / sum |ref|^2): the error measure of Sec. 4."""
    ref = np.asarray(ref, np.complex128).ravel()
    approx = np.asarray(approx, np.complex128).ravel()
    return float(np.sqrt(np.sum(np.abs(ref - approx) ** 2) / np.sum(np.abs(ref) ** 2)))
