"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: numpy's FFT
(a library routine), closed forms of special phases (identity, translation,
Fourier multipliers: Sec. 1.1-1.2), hand-derived values (tests/golden), and
identities (Parseval, adjointness, homogeneity of the phase).
"""
import os

import numpy as np
import pytest

from paper_math_0610051_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "phase_values.txt")


def _centred_k(N):
    k = np.arange(N) - N // 2
    return np.meshgrid(k, k, indexing="ij")


def _multiplier_apply(f, mult):
    """Apply a Fourier multiplier with numpy: IDFT(mult * DFT f) in Eq. dft's unitary scaling."""
    N = f.shape[-1]
    fh = np.fft.fftshift(np.fft.fft2(f)) / N
    return np.fft.ifft2(np.fft.ifftshift(fh * mult)) * N


# ---------------------------------------------------------------- P6: DFT ---

@pytest.mark.parametrize("N", [8, 16, 32])
def test_dft_matches_numpy(orc, N):
    f = synth.white_noise(N, 1, seed=N, real=False)[0]
    ref = np.fft.fftshift(np.fft.fft2(f)) / N
    got = orc.dft2(f)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))
    back = orc.idft2(got)
    assert np.max(np.abs(back - f)) < 1e-12 * np.max(np.abs(f))
    # numpy's inverse on the same centred spectrum
    ref_inv = np.fft.ifft2(np.fft.ifftshift(got)) * N
    assert np.max(np.abs(back - ref_inv)) < 1e-12 * np.max(np.abs(f))


def test_parseval(orc):
    f = synth.white_noise(24, 1, seed=3, real=False)[0]
    fh = orc.dft2(f)
    assert abs(np.linalg.norm(fh) - np.linalg.norm(f)) < 1e-12 * np.linalg.norm(f)


# ------------------------------------------------------ phase golden values ---

def _golden_rows():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            kind, params, x, k, val, _ = [s.strip() for s in line.split("|", 5)]
            rows.append((kind, [float(v) for v in params.split()], [float(v) for v in x.split()],
                         [int(v) for v in k.split()], float(val)))
    return rows


@pytest.mark.parametrize("row", _golden_rows(), ids=lambda r: f"{r[0]}-{r[2]}-{r[3]}")
def test_phase_golden(orc, row):
    kind, params, (x1, x2), (k1, k2), val = row
    if kind == "amp":
        got = orc.amp_eval(orc.Amplitude(1, *params), [x1], [k1], [k2])[0]
    else:
        kinds = {"ellipse": orc.ELLIPSE, "tau": orc.TAU_MODES}
        got = []
        for grouped in (False, True):
            ph = orc.Phase(kinds[kind], params, grouped=grouped)
            got.append(orc.phase_eval(ph, [x1], [x2], [k1], [k2])[0])
        assert abs(got[0] - got[1]) < 1e-12
        got = got[0]
    assert abs(got - val) < 1e-12, (got, val)


def test_phase_homogeneous(orc):
    """Phi(x, lambda xi) = lambda Phi(x, xi) for lambda > 0 (Sec. 1, after Eq. FIO)."""
    g = np.random.default_rng(5)
    n = 200
    x1, x2 = g.uniform(0, 1, n), g.uniform(0, 1, n)
    k1, k2 = g.integers(-20, 21, n), g.integers(-20, 21, n)
    for ph in [orc.Phase(orc.ELLIPSE, synth.ellipse_params()),
               orc.Phase(orc.TAU_MODES, synth.tau_mode_params(8, seed=1)),
               orc.Phase(orc.SHIFT_WAVE, [0.1, -0.3, 0.7])]:
        p1 = orc.phase_eval(ph, x1, x2, k1, k2)
        p3 = orc.phase_eval(ph, x1, x2, 3 * k1, 3 * k2)
        assert np.max(np.abs(p3 - 3 * p1)) < 1e-11


def test_tau_grouping_is_exact(orc):
    """The regrouping of tau by m used for speed equals the literal sum over modes."""
    g = np.random.default_rng(6)
    n = 500
    x1, x2 = g.uniform(0, 1, n), g.uniform(0, 1, n)
    k1, k2 = g.integers(-30, 31, n), g.integers(-30, 31, n)
    prm = synth.tau_mode_params(32, seed=2)
    a = orc.phase_eval(orc.Phase(orc.TAU_MODES, prm, grouped=False), x1, x2, k1, k2)
    b = orc.phase_eval(orc.Phase(orc.TAU_MODES, prm, grouped=True), x1, x2, k1, k2)
    assert np.max(np.abs(a - b)) < 1e-11


# ------------------------------------------------------------ closed forms ---

def test_identity_phase_is_identity(orc):
    """Phi = x.xi, a = 1: L is the identity (the isometry remark after Eq. dft)."""
    N = 16
    f = synth.white_noise(N, 1, seed=7, real=False)[0]
    out = orc.apply_dense(orc.Phase(orc.SHIFT_WAVE, [0, 0, 0]), orc.Amplitude(), f)
    assert np.max(np.abs(out - f)) < 1e-12


def test_shift_phase_translates(orc):
    """Phi = (x - x0).xi with x0 = (3, 5)/N on the grid: (Lf)(x) = f(x - x0)."""
    N = 16
    f = synth.white_noise(N, 1, seed=8, real=False)[0]
    out = orc.apply_dense(orc.Phase(orc.SHIFT_WAVE, [3 / N, 5 / N, 0]), orc.Amplitude(), f)
    assert np.max(np.abs(out - np.roll(f, (3, 5), axis=(0, 1)))) < 1e-12


@pytest.mark.parametrize("c", [0.37, 1.9])
def test_wave_phase_is_fourier_multiplier(orc, c):
    """Phi = x.xi + c|xi| (the wave propagator, Sec. 1.1): L = IDFT exp(2 pi i c|xi|) DFT."""
    N = 16
    f = synth.white_noise(N, 1, seed=9, real=False)[0]
    K1, K2 = _centred_k(N)
    ref = _multiplier_apply(f, np.exp(2j * np.pi * c * np.hypot(K1, K2)))
    out = orc.apply_dense(orc.Phase(orc.SHIFT_WAVE, [0, 0, c]), orc.Amplitude(), f)
    assert np.max(np.abs(out - ref)) < 1e-11


def test_constant_ellipse_is_anisotropic_multiplier(orc):
    """Ellipse phase with constant axes (B1 = B2 = 0): multiplier exp(2 pi i sqrt(A1^2 xi1^2 + A2^2 xi2^2))."""
    N = 16
    f = synth.white_noise(N, 1, seed=10, real=False)[0]
    K1, K2 = _centred_k(N)
    A1, A2 = 0.45, 1.3
    ref = _multiplier_apply(f, np.exp(2j * np.pi * np.sqrt((A1 * K1) ** 2 + (A2 * K2) ** 2)))
    out = orc.apply_dense(orc.Phase(orc.ELLIPSE, [A1, 0, A2, 0]), orc.Amplitude(), f)
    assert np.max(np.abs(out - ref)) < 1e-11


@pytest.mark.parametrize("grouped", [False, True])
def test_angular_tau_is_multiplier(orc, grouped):
    """tau = a cos(m theta + p) with k = 0 is x-independent: multiplier exp(2 pi i |xi| tau(theta))."""
    N = 16
    f = synth.white_noise(N, 1, seed=11, real=False)[0]
    K1, K2 = _centred_k(N)
    a, m, p = 0.21, 3, 0.4
    th = np.arctan2(K2, K1)
    ref = _multiplier_apply(f, np.exp(2j * np.pi * np.hypot(K1, K2) * a * np.cos(m * th + p)))
    ph = orc.Phase(orc.TAU_MODES, [[a, 0, 0, m, p]], grouped=grouped)
    out = orc.apply_dense(ph, orc.Amplitude(), f)
    assert np.max(np.abs(out - ref)) < 1e-11


def test_separable_amplitude(orc):
    """a = (1 + a1 sin 2pi x1)(1 + a2 cos theta), Phi = x.xi: Lf = a_x IDFT(a_xi fhat)."""
    N = 16
    f = synth.white_noise(N, 1, seed=12, real=False)[0]
    K1, K2 = _centred_k(N)
    a1, a2 = 0.5, 0.3
    r = np.hypot(K1, K2)
    cth = np.where(r > 0, K1 / np.where(r > 0, r, 1), 1.0)
    ax = 1 + a1 * np.sin(2 * np.pi * np.arange(N) / N)[:, None]
    ref = ax * _multiplier_apply(f, 1 + a2 * cth)
    out = orc.apply_dense(orc.Phase(orc.SHIFT_WAVE, [0, 0, 0]), orc.Amplitude(1, a1, a2), f)
    assert np.max(np.abs(out - ref)) < 1e-12


# -------------------------------------------------------------- identities ---

def _phases(orc):
    return [orc.Phase(orc.ELLIPSE, synth.ellipse_params()),
            orc.Phase(orc.TAU_MODES, synth.tau_mode_params(6, seed=4))]


def test_adjoint_identity_dense(orc):
    """<Lf, g> = <f, L*g> for the dense forward and adjoint sums (Sec. 3.5)."""
    N = 16
    f = synth.white_noise(N, 1, seed=13, real=False)[0]
    g = synth.white_noise(N, 1, seed=14, real=False)[0]
    for ph in _phases(orc):
        for amp in (orc.Amplitude(), orc.Amplitude(1, 0.5, 0.3)):
            lf = orc.apply_dense(ph, amp, f)
            lsg = orc.adjoint_dense(ph, amp, g)
            a, b = np.vdot(g, lf), np.vdot(lsg, f)
            assert abs(a - b) < 1e-11 * abs(a)


def test_adjoint_is_conjugate_transpose(orc):
    """At N = 8 the adjoint applied to each delta equals the conjugate transpose of L's matrix."""
    N = 8
    ph = orc.Phase(orc.ELLIPSE, synth.ellipse_params())
    amp = orc.Amplitude(1, 0.5, 0.3)
    M = orc.matrix(ph, amp, N)
    g = synth.white_noise(N, 1, seed=15, real=False)[0]
    ref = (M.conj().T @ g.ravel()).reshape(N, N)
    got = orc.adjoint_dense(ph, amp, g)
    assert np.max(np.abs(got - ref)) < 1e-12


def test_adjoint_hat_is_dft_of_adjoint(orc):
    N = 16
    ph = orc.Phase(orc.TAU_MODES, synth.tau_mode_params(5, seed=9))
    amp = orc.Amplitude(1, 0.2, -0.4)
    g = synth.white_noise(N, 1, seed=16, real=False)[0]
    full = orc.dft2(orc.adjoint_dense(ph, amp, g))
    k1, k2 = synth.sample_freqs(N, 40, seed=1)
    pts = orc.adjoint_hat_points(ph, amp, g, k1, k2)
    assert np.max(np.abs(pts - full[k1 + N // 2, k2 + N // 2])) < 1e-12


def test_linearity(orc):
    N = 16
    ph = orc.Phase(orc.ELLIPSE, synth.ellipse_params())
    amp = orc.Amplitude()
    f = synth.white_noise(N, 1, seed=17, real=False)[0]
    g = synth.white_noise(N, 1, seed=18, real=False)[0]
    a, b = 0.7 - 0.2j, -1.3 + 0.5j
    lhs = orc.apply_dense(ph, amp, a * f + b * g)
    rhs = a * orc.apply_dense(ph, amp, f) + b * orc.apply_dense(ph, amp, g)
    assert np.max(np.abs(lhs - rhs)) < 1e-12


def test_points_equal_dense(orc):
    """Sampled per-point sums agree with the full grid evaluation."""
    N = 32
    ph = orc.Phase(orc.ELLIPSE, synth.ellipse_params())
    amp = orc.Amplitude()
    f = synth.white_noise(N, 1, seed=19)[0]
    full = orc.apply_dense(ph, amp, f)
    n1, n2 = synth.sample_points(N, 50, seed=2)
    pts = orc.apply_points(ph, amp, orc.dft2(f), n1, n2)
    assert np.max(np.abs(pts - full[n1, n2])) < 1e-12


def test_rel_l2_definition(orc):
    a = np.array([3.0, 4.0], complex)
    assert orc.rel_l2(a, a) == 0.0
    assert abs(orc.rel_l2(a, np.array([3.0, 4.5])) - 0.1) < 1e-15
