"""Pins of the oracle's integration-along-ellipses workload (Sec. 4 variable
amplitude experiment, Appendix A): the circle radius as tau modes, and the
identity L+ f + L- f = (1/N) sum_xi J0(2 pi r(x)|xi|)/(2 pi) e^{2 pi i x.xi} fhat(xi),
the kernel of Appendix A, evaluated here directly with scipy's J0."""
import numpy as np
import pytest

from paper_math_0610051_gb300 import synth

sp = pytest.importorskip("scipy.special")


def _radius(x1, x2):
    return (3 + np.sin(4 * np.pi * x1)) * (3 + np.sin(4 * np.pi * x2)) / 16


def test_circle_modes_are_the_radius(orc):
    g = np.random.default_rng(1)
    x1, x2, th = g.uniform(0, 1, 200), g.uniform(0, 1, 200), g.uniform(0, 2 * np.pi, 200)
    for sign in (1, -1):
        tau = orc.tau_eval(synth.circle_grt_modes(sign), x1, x2, th)[:, 0]
        assert np.max(np.abs(tau - sign * _radius(x1, x2))) < 1e-14


def test_hankel_pair_sums_to_the_j0_kernel(orc):
    N = 32
    f = synth.white_noise(N, 1, seed=3, real=False)[0]
    fh = orc.dft2(f)
    n1, n2 = synth.sample_points(N, 48, seed=2)
    got = sum(orc.apply_points(orc.Phase(orc.TAU_MODES, synth.circle_grt_modes(s)),
                               orc.Amplitude(orc.AMP_HANKEL, s), fh, n1, n2) for s in (1, -1))
    k = np.arange(N) - N // 2
    K1, K2 = np.meshgrid(k, k, indexing="ij")
    ref = np.empty(len(n1), complex)
    for i, (a, b) in enumerate(zip(n1, n2)):
        x1, x2 = a / N, b / N
        kern = sp.j0(2 * np.pi * _radius(x1, x2) * np.hypot(K1, K2)) / (2 * np.pi)
        ref[i] = np.sum(kern * np.exp(2j * np.pi * (x1 * K1 + x2 * K2)) * fh) / N
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_hankel_amplitude_envelope(orc):
    """|a+-| -> sqrt(2 / (pi z)) / (4 pi) with z = 2 pi rho (Hankel asymptotics),
    the order -1/2 of Appendix A; the two signs are complex conjugates."""
    rho = np.array([50.0, 200.0, 800.0])
    ap = orc.amp_eval(orc.Amplitude(orc.AMP_HANKEL, 1), np.zeros(3), [1] * 3, [0] * 3, rho)
    am = orc.amp_eval(orc.Amplitude(orc.AMP_HANKEL, -1), np.zeros(3), [1] * 3, [0] * 3, -rho)
    env = np.sqrt(2 / (np.pi * 2 * np.pi * rho)) / (4 * np.pi)
    assert np.all(np.abs(np.abs(ap) / env - 1) < 2e-3)
    assert np.allclose(am, np.conj(ap), rtol=0, atol=1e-15)


def test_paper_ellipse_phase_hand_values(orc):
    """Eq. nrphase with the axes of the paper's experiments (Sec. 4):
    r1 = (2 + sin 4 pi x1)(2 + sin 4 pi x2)/9, r2 = (2 + cos 4 pi x1)(2 + cos 4 pi x2)/9.
    At x = (0, 0): r1 = 4/9, r2 = 1, so Phi(x, (9, 4)) = sqrt(16 + 16).
    At x = (1/8, 1/8): r1 = 1, r2 = 4/9, so Phi(x, (4, 9)) = 13/8 + sqrt(16 + 16).
    At x = (1/4, 0): r1 = 4/9, r2 = 1/3, so Phi(x, (9, 3)) = 9/4 + sqrt(16 + 1)."""
    ph = orc.Phase(orc.ELLIPSE_PRODUCT, synth.paper_ellipse_params())
    got = orc.phase_eval(ph, [0.0, 0.125, 0.25], [0.0, 0.125, 0.0], [9, 4, 9], [4, 9, 3])
    want = [np.sqrt(32.0), 13 / 8 + np.sqrt(32.0), 9 / 4 + np.sqrt(17.0)]
    assert np.max(np.abs(got - want)) < 1e-13
    # homogeneity of degree 1 in xi
    g = np.random.default_rng(3)
    x1, x2 = g.uniform(0, 1, 20), g.uniform(0, 1, 20)
    k1, k2 = g.integers(-30, 31, 20), g.integers(-30, 31, 20)
    a = orc.phase_eval(ph, x1, x2, k1, k2)
    b = orc.phase_eval(ph, x1, x2, 3 * k1, 3 * k2)
    assert np.max(np.abs(b - 3 * a)) < 1e-11


def test_hankel_amplitude_is_the_hankel_function(orc):
    """Appendix A, Eq. ellipses_amp: a+ = H0^(1)(2 pi rho) e^{-2 pi i rho} / (4 pi) and
    a- = H0^(2)(2 pi rho) e^{+2 pi i rho} / (4 pi), since J0 + i Y0 = H0^(1) and
    J0 - i Y0 = H0^(2).  scipy's Hankel functions are an independent evaluation, and a
    flipped sign of the Y0 term (H0^(2) in a+) fails this at every rho."""
    rho = np.array([0.1, 0.37, 1.0, 2.5, 7.3, 31.0, 120.0])
    z = 2 * np.pi * rho
    zeros, ones = np.zeros(len(rho)), [1] * len(rho)
    ap = orc.amp_eval(orc.Amplitude(orc.AMP_HANKEL, 1), zeros, ones, [0] * len(rho), rho)
    am = orc.amp_eval(orc.Amplitude(orc.AMP_HANKEL, -1), zeros, ones, [0] * len(rho), -rho)
    want_p = sp.hankel1(0, z) * np.exp(-1j * z) / (4 * np.pi)
    want_m = sp.hankel2(0, z) * np.exp(1j * z) / (4 * np.pi)
    assert np.max(np.abs(ap - want_p) / np.abs(want_p)) < 1e-13
    assert np.max(np.abs(am - want_m) / np.abs(want_m)) < 1e-13


def test_hankel_amplitude_is_demodulated(orc):
    """The point of Appendix A's split: a+ is the smooth envelope of the outgoing wave,
    H0^(1)(z) ~ sqrt(2 / (pi z)) e^{i (z - pi/4)}, so arg a+ -> -pi/4 and arg a- -> +pi/4
    as rho grows (with the sign flipped, a+ would oscillate like e^{-2 i z})."""
    rho = np.array([40.0, 160.0, 640.0, 2560.0])
    n = len(rho)
    ap = orc.amp_eval(orc.Amplitude(orc.AMP_HANKEL, 1), np.zeros(n), [1] * n, [0] * n, rho)
    am = orc.amp_eval(orc.Amplitude(orc.AMP_HANKEL, -1), np.zeros(n), [1] * n, [0] * n, -rho)
    # next term of the expansion: the phase error is about 1 / (8 z)
    tol = 1.0 / (8 * 2 * np.pi * rho) * 1.5
    assert np.all(np.abs(np.angle(ap) + np.pi / 4) < tol)
    assert np.all(np.abs(np.angle(am) - np.pi / 4) < tol)
