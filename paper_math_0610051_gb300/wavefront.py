"""The imaging experiment of Sec. 4 (Figure 2): the normal operator L*L keeps
the singularities of its input, WF(L*L f) = WF(f), for the phase
Phi(x, xi) = x.xi + r(x)|xi| with the circle radius
r(x) = (3 + sin 4 pi x1)(3 + sin 4 pi x2) / 16 and a = 1.

``run`` applies L and L*L (fio_apply_normal) on the GPU to three inputs with
different singularities -- a disc (a jump along a circle), three thin line
segments and a rectangle (jumps along straight edges with corners) -- and writes
headless arrays instead of the paper's images: for each input, f, |L f| and
|L*L f| as .npy files.  The property is qualitative (the paper compares
pictures), so nothing here is a parity check.  As a number to read beside the
arrays, ``band_energy`` gives the share of an image's high-frequency energy that
lies within a few cells of the jump set of f.

Usage: python -m paper_math_0610051_gb300.wavefront --N 512 --out DIR
"""
from __future__ import annotations

import argparse
import os

import numpy as np


def inputs(N: int) -> dict:
    """The three test images on the N x N grid (cell centres), values 0 / 1."""
    x = (np.arange(N) + 0.5) / N
    X1, X2 = np.meshgrid(x, x, indexing="ij")
    disc = ((X1 - 0.5) ** 2 + (X2 - 0.5) ** 2 < 0.2 ** 2).astype(float)
    lines = np.zeros((N, N))
    for a, b, c in ((1.0, 0.3, 0.0), (0.4, 1.0, -0.55), (1.0, -1.0, 0.1)):
        lines = np.maximum(lines, (np.abs(a * (X1 - 0.5) + b * (X2 - 0.5) + c) < 1.0 / N).astype(float))
    rect = ((np.abs(X1 - 0.45) < 0.18) & (np.abs(X2 - 0.55) < 0.12)).astype(float)
    return {"disc": disc, "lines": lines, "rectangle": rect}


def jump_band(f: np.ndarray, width: int) -> np.ndarray:
    """Cells within `width` grid steps (periodic) of a jump of f."""
    s = np.zeros(f.shape, bool)
    for d in (0, 1):
        s |= np.abs(f - np.roll(f, 1, d)) > 1e-9
    b = s.copy()
    for _ in range(width):
        b = b | np.roll(b, 1, 0) | np.roll(b, -1, 0) | np.roll(b, 1, 1) | np.roll(b, -1, 1)
    return b


def band_energy(g: np.ndarray, band: np.ndarray, cut: float) -> float:
    """Share of the energy of g above frequency |xi| > cut that lies in `band`."""
    N = g.shape[0]
    k = np.fft.fftfreq(N) * N
    K1, K2 = np.meshgrid(k, k, indexing="ij")
    h = np.fft.ifft2(np.fft.fft2(g) * (np.hypot(K1, K2) > cut))
    e = np.abs(h) ** 2
    return float(e[band].sum() / e.sum())


def run(N: int = 512, out: str | None = None, eps: float = 1e-4) -> dict:
    """Apply L and L*L to the three inputs; write the arrays to `out` (if given)
    and return {input: {"band": ..., "f": E, "Lf": E, "LsLf": E}}."""
    import torch

    from . import fio, synth

    imgs = inputs(N)
    names = list(imgs)
    f = np.stack([imgs[n] for n in names])
    with fio.Plan(N, fio.PHASE_TAU_MODES, synth.circle_grt_modes(1), eps, max_batch=len(names)) as plan:
        x = torch.from_numpy(f).to(torch.complex64).cuda()
        lf = plan.apply(x).cpu().numpy()
        llf = plan.normal(x).cpu().numpy()
        plan.sync()
    res = {}
    if out:
        os.makedirs(out, exist_ok=True)
    for i, n in enumerate(names):
        band = jump_band(imgs[n], 3)
        cut = N / 5
        res[n] = {"band": float(band.mean()), "f": band_energy(imgs[n], band, cut),
                  "Lf": band_energy(lf[i], band, cut), "LsLf": band_energy(llf[i], band, cut)}
        if out:
            np.save(os.path.join(out, f"{n}_f.npy"), imgs[n].astype(np.float32))
            np.save(os.path.join(out, f"{n}_abs_Lf.npy"), np.abs(lf[i]).astype(np.float32))
            np.save(os.path.join(out, f"{n}_abs_LsLf.npy"), np.abs(llf[i]).astype(np.float32))
    return res


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--N", type=int, default=512)
    ap.add_argument("--eps", type=float, default=1e-4)
    ap.add_argument("--out", default="wavefront_arrays")
    a = ap.parse_args()
    for n, r in run(a.N, a.out, a.eps).items():
        print(f"{n:10s} band {r['band']:.3f} of the grid; high-frequency energy in the band: "
              f"f {r['f']:.3f}, |Lf| {r['Lf']:.3f}, |L*Lf| {r['LsLf']:.3f}")


if __name__ == "__main__":
    main()
