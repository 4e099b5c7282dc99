"""The seeded input generators (no GPU): reproducible, and with the structure the
workloads state (tau modes: integer wave numbers in range, amplitudes summing
to the scale; distinct sample points; unit directions)."""
import numpy as np

from paper_math_0610051_gb300 import synth


def test_tau_modes_structure_and_seed():
    m = synth.tau_mode_params(256, seed=7, kmax=8, mmax=4)
    assert m.shape == (256, 5)
    a, k1, k2, mm, p = m.T
    assert np.all(k1 == np.round(k1)) and np.all(np.abs(k1) <= 8) and np.all(np.abs(k2) <= 8)
    assert np.all(mm == np.round(mm)) and np.all((mm >= 0) & (mm <= 4))
    assert abs(np.sum(np.abs(a)) - 0.05) < 1e-15
    assert np.all((p >= 0) & (p < 2 * np.pi))
    # amplitudes fall as 1/|(k1, k2, m)|^2
    n2 = k1 ** 2 + k2 ** 2 + mm ** 2
    nz = n2 > 0
    r = np.abs(a[nz]) * n2[nz]
    assert np.allclose(r, r[0])
    assert np.array_equal(m, synth.tau_mode_params(256, seed=7, kmax=8, mmax=4))
    assert not np.array_equal(m, synth.tau_mode_params(256, seed=8, kmax=8, mmax=4))


def test_sample_points_distinct_and_in_range():
    n1, n2 = synth.sample_points(64, 500, seed=3)
    assert len(set(zip(n1.tolist(), n2.tolist()))) == 500
    assert n1.min() >= 0 and n1.max() < 64 and n2.min() >= 0 and n2.max() < 64
    k1, k2 = synth.sample_freqs(64, 100, seed=3)
    assert k1.min() >= -32 and k1.max() < 32 and k2.min() >= -32 and k2.max() < 32


def test_white_noise_and_directions():
    f = synth.white_noise(32, 2, seed=1)
    assert f.shape == (2, 32, 32) and np.all(f.imag == 0)
    g = synth.white_noise(32, 1, seed=1, real=False)
    assert abs(np.mean(np.abs(g) ** 2) - 1.0) < 0.1
    d = synth.unit_directions(16, 4, seed=2)
    assert np.allclose(np.sum(np.abs(d) ** 2, axis=(1, 2)), 1.0)


def test_complex_noise_level():
    a = synth.white_noise(64, 1, seed=5)
    n = synth.complex_noise_like(a, 0.01, seed=6)
    rel = np.sqrt(np.mean(np.abs(n) ** 2) / np.mean(np.abs(a) ** 2))
    assert abs(rel - 0.01) < 0.001
