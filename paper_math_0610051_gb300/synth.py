"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module holds no arithmetic of the FIO method: it only draws inputs
(grids of samples, phase parameters, sample locations) from fixed seeds, so
that the CUDA path and the CPU oracle can be fed the same data.  numpy's
PCG64 generator is used throughout.

Workload recipes (the paper's inputs are synthetic: white noise in Sec. 4):

* ``white_noise``: i.i.d. N(0,1) samples (Sec. 4, Table 3's input).
* ``smooth_noise_discs``: Gaussian noise low-passed by exp(-|xi|^2 / (2 s^2)),
  s = N/8, scaled to unit RMS, plus 16 periodic discs with uniform centres,
  radii U[0.02, 0.08] and heights U[0.5, 1.5] (sharp edges: singularities).
* ``ellipse_params``: c1 = (2 + sin 2pi x1 sin 2pi x2)/3,
  c2 = (2 + cos 2pi x1 cos 2pi x2)/3 as {A1, B1, A2, B2}.
* ``tau_mode_params``: K modes a_j cos(2pi(k1 x1 + k2 x2) + m theta + p_j),
  integer k in [-kmax, kmax], integer m in [0, mmax], a_j proportional to
  1/|(k1, k2, m)|^2 (1 for the zero triple), normalised so sum |a_j| = scale.
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def white_noise(N: int, batch: int = 1, seed: int = 0, real: bool = True) -> np.ndarray:
    """[batch, N, N] complex128 with N(0,1) real parts (and imaginary parts if not real)."""
    g = _rng(seed)
    re = g.standard_normal((batch, N, N))
    if real:
        return re.astype(np.complex128)
    return (re + 1j * g.standard_normal((batch, N, N))) / np.sqrt(2.0)


def smooth_noise_discs(N: int, seed: int = 0, ndiscs: int = 16) -> np.ndarray:
    """[N, N] complex128 (real valued): low-passed noise plus sharp periodic discs."""
    g = _rng(seed)
    noise = g.standard_normal((N, N))
    k = np.fft.fftfreq(N) * N
    k2 = k[:, None] ** 2 + k[None, :] ** 2
    s = N / 8.0
    f = np.real(np.fft.ifft2(np.fft.fft2(noise) * np.exp(-k2 / (2 * s * s))))
    f /= np.sqrt(np.mean(f * f))
    x = np.arange(N) / N
    X1, X2 = np.meshgrid(x, x, indexing="ij")
    for _ in range(ndiscs):
        c1, c2 = g.uniform(0, 1, 2)
        rad = g.uniform(0.02, 0.08)
        h = g.uniform(0.5, 1.5)
        d1 = (X1 - c1 + 0.5) % 1.0 - 0.5
        d2 = (X2 - c2 + 0.5) % 1.0 - 0.5
        f += h * (d1 * d1 + d2 * d2 < rad * rad)
    return f.astype(np.complex128)


def ellipse_params() -> np.ndarray:
    return np.array([2.0 / 3.0, 1.0 / 3.0, 2.0 / 3.0, 1.0 / 3.0])


def tau_mode_params(K: int, seed: int = 0, kmax: int = 4, mmax: int = 4,
                    scale: float = 0.05) -> np.ndarray:
    """[K, 5] rows {a_j, k1_j, k2_j, m_j, p_j}."""
    g = _rng(seed)
    k1 = g.integers(-kmax, kmax + 1, K)
    k2 = g.integers(-kmax, kmax + 1, K)
    m = g.integers(0, mmax + 1, K)
    norm2 = k1.astype(float) ** 2 + k2.astype(float) ** 2 + m.astype(float) ** 2
    a = np.where(norm2 > 0, 1.0 / np.maximum(norm2, 1.0), 1.0)
    a = a * g.choice([-1.0, 1.0], K)
    a *= scale / np.sum(np.abs(a))
    p = g.uniform(0.0, 2 * np.pi, K)
    return np.stack([a, k1, k2, m, p], axis=1).astype(np.float64)


def sample_points(N: int, s: int, seed: int = 0):
    """s distinct grid points (n1, n2) drawn uniformly."""
    g = _rng(seed)
    idx = g.choice(N * N, size=min(s, N * N), replace=False)
    return (idx // N).astype(np.int32), (idx % N).astype(np.int32)


def sample_freqs(N: int, s: int, seed: int = 0):
    """s distinct frequencies (k1, k2) in [-N/2, N/2)^2."""
    n1, n2 = sample_points(N, s, seed)
    return (n1 - N // 2).astype(np.int32), (n2 - N // 2).astype(np.int32)


def unit_directions(N: int, count: int, seed: int = 0, real: bool = True) -> np.ndarray:
    """[count, N, N] complex128 directions of unit Frobenius norm."""
    d = white_noise(N, count, seed, real=real)
    return d / np.sqrt(np.sum(np.abs(d) ** 2, axis=(1, 2), keepdims=True))


def complex_noise_like(a: np.ndarray, rel: float, seed: int = 0) -> np.ndarray:
    """Complex Gaussian noise with RMS = rel * RMS(a)."""
    g = _rng(seed)
    n = (g.standard_normal(a.shape) + 1j * g.standard_normal(a.shape)) / np.sqrt(2.0)
    return n * rel * np.sqrt(np.mean(np.abs(a) ** 2))


def circle_grt_modes(sign: int = 1) -> np.ndarray:
    """Tau modes of sign * r(x) with r = (3 + sin 4 pi x1)(3 + sin 4 pi x2) / 16, the
    circle radius of the variable-amplitude experiment (Sec. 4, Eq. circlerad):
    r = 9/16 + (3/16) sin 4 pi x1 + (3/16) sin 4 pi x2
        + (1/32) cos 2 pi (2 x1 - 2 x2) - (1/32) cos 2 pi (2 x1 + 2 x2).
    With these modes the tau-mode phase is Phi = x.xi + sign r(x) |xi|."""
    h = np.pi / 2
    rows = [[9 / 16, 0, 0, 0, 0.0], [3 / 16, 2, 0, 0, -h], [3 / 16, 0, 2, 0, -h],
            [1 / 32, 2, -2, 0, 0.0], [1 / 32, 2, 2, 0, np.pi]]
    m = np.array(rows, dtype=np.float64)
    m[:, 0] *= sign
    return m


def paper_ellipse_params() -> np.ndarray:
    """{a1, s1, a2, s2} of the product-form ellipse phase of the paper's own
    separation experiments (Sec. 4, Eq. nrphase): r1 = (2 + sin 4 pi x1)(2 + sin 4 pi x2)/9,
    r2 = (2 + cos 4 pi x1)(2 + cos 4 pi x2)/9."""
    return np.array([2.0, 1.0 / 9.0, 2.0, 1.0 / 9.0])
