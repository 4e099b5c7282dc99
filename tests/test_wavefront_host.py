"""Host helpers of the Figure 2 experiment (numpy only, no GPU): the test images,
the band of cells near a jump, and the share of high-frequency energy in it."""
import numpy as np

from paper_math_0610051_gb300 import wavefront


def test_inputs_are_indicator_images():
    imgs = wavefront.inputs(64)
    assert set(imgs) == {"disc", "lines", "rectangle"}
    for a in imgs.values():
        assert a.shape == (64, 64) and set(np.unique(a)) <= {0.0, 1.0} and a.sum() > 0
    # the disc of radius 0.2 covers about pi 0.04 of the unit square
    assert abs(imgs["disc"].mean() - np.pi * 0.04) < 0.01


def test_jump_band_of_a_half_plane():
    N = 32
    f = np.zeros((N, N))
    f[:, N // 2:] = 1.0  # jumps at columns N/2 and 0 (periodic)
    b = wavefront.jump_band(f, 2)
    cols = np.where(b.any(axis=0))[0]
    # a jump is marked at the cell after it (columns 0 and N/2), then widened by 2 cells
    assert set(cols) == {N - 2, N - 1, 0, 1, 2, N // 2 - 2, N // 2 - 1, N // 2, N // 2 + 1, N // 2 + 2}
    assert b.all(axis=0)[cols].all()


def test_band_energy_limits():
    N = 64
    k = np.arange(N)
    # a single high-frequency plane wave: its energy is spread evenly over the grid
    g = np.exp(2j * np.pi * 20 * k / N)[None, :] * np.ones((N, 1))
    band = np.zeros((N, N), bool)
    band[:, :16] = True
    assert abs(wavefront.band_energy(g, band, N / 5) - 0.25) < 1e-12
    assert abs(wavefront.band_energy(g, np.ones((N, N), bool), N / 5) - 1.0) < 1e-12
