"""Differentiation through the fast operator (the inverse-problem use of Sec. 4's
ellipse transform): loss = ||L f - g||^2, g = L f_true + 1% noise, gradient by the
hand-written adjoint inside torch.autograd.

A quadratic's central difference [Q(f + h d) - Q(f - h d)] / (2h) equals its
directional derivative exactly (up to rounding) for any h, so the check is
tight; it runs on the FP64 path, whose rounding is far below the tolerance.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_math_0610051_gb300 import autograd, fio
    return fio, autograd, torch


def _problem(fio, torch, N, prec, eps, seed=0):
    from paper_math_0610051_gb300 import synth
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    plan = fio.Plan(N, fio.PHASE_ELLIPSE, synth.ellipse_params(), eps, precision=prec)
    f_true = torch.from_numpy(synth.smooth_noise_discs(N, seed=seed)).to(dt).cuda()[None]
    g = plan.apply(f_true)
    g = g + torch.from_numpy(synth.complex_noise_like(g.cpu().numpy(), 0.01, seed=seed + 1)).to(dt).cuda()
    f0 = torch.from_numpy(synth.white_noise(N, 1, seed=seed + 2)).to(dt).cuda()
    return plan, g, f0


def test_gradient_matches_central_differences(env):
    """N = 512: <grad, d> against central differences with h = 1e-3 in 64 seeded
    real unit directions."""
    fio, ag, torch = env
    from paper_math_0610051_gb300 import synth
    N = 512
    plan, g, f0 = _problem(fio, torch, N, "fp64", 1e-4)

    def loss(fr):
        r = ag.fio_apply(fr.to(torch.complex128), plan) - g
        return (r.real ** 2 + r.imag ** 2).sum()

    fr = f0.real.clone().requires_grad_(True)
    Q = loss(fr)
    Q.backward()
    grad = fr.grad.detach()
    dirs = torch.from_numpy(synth.unit_directions(N, 64, seed=9).real).cuda()
    h = 1e-3
    errs = []
    with torch.no_grad():
        for k in range(64):
            d = dirs[k][None]
            fd = (loss(fr + h * d) - loss(fr - h * d)) / (2 * h)
            an = (grad * d).sum()
            errs.append(abs(float(fd - an)) / max(abs(float(an)), 1e-30))
    plan.close()
    assert max(errs) < 1e-6, max(errs)


def test_mixed_gradient_tracks_fp64(env):
    """The mixed-precision gradient agrees with the FP64 one to 1e-4."""
    fio, ag, torch = env
    N = 256
    grads = []
    for prec in ("fp64", "mixed"):
        plan, g, f0 = _problem(fio, torch, N, prec, 1e-4, seed=3)
        f = f0.clone().requires_grad_(True)
        r = ag.fio_apply(f, plan) - g
        (r.abs() ** 2).sum().backward()
        grads.append(f.grad.detach().to(torch.complex128).cpu().numpy())
        plan.close()
    e = np.linalg.norm(grads[0] - grads[1]) / np.linalg.norm(grads[0])
    assert e < 1e-4, e


def test_gradient_is_dense_adjoint(env, orc):
    """N = 64: the autograd gradient 2 L*(L f - g) against the oracle's dense adjoint."""
    fio, ag, torch = env
    N = 64
    plan, g, f0 = _problem(fio, torch, N, "fp64", 1e-6, seed=5)
    f = f0.clone().requires_grad_(True)
    r = ag.fio_apply(f, plan) - g
    (r.abs() ** 2).sum().backward()
    grad = f.grad.detach().cpu().numpy()[0]
    res = r.detach().cpu().numpy()[0]
    from paper_math_0610051_gb300 import synth
    ref = 2 * orc.adjoint_dense(orc.Phase(orc.ELLIPSE, synth.ellipse_params()), orc.Amplitude(), res)
    plan.close()
    assert np.linalg.norm(grad - ref) / np.linalg.norm(ref) < 1e-6


def test_adjoint_function_gradient(env):
    """FIOAdjoint's backward is the forward operator: <L* g, u> = <g, L u>."""
    fio, ag, torch = env
    from paper_math_0610051_gb300 import synth
    N = 64
    plan = fio.Plan(N, fio.PHASE_ELLIPSE, synth.ellipse_params(), 1e-6, precision="fp64")
    g = torch.from_numpy(synth.white_noise(N, 1, seed=7, real=False)).cuda().requires_grad_(True)
    u = torch.from_numpy(synth.white_noise(N, 1, seed=8, real=False)).cuda()
    out = ag.fio_adjoint(g, plan)
    (out.conj() * u).real.sum().backward()
    # d/dg Re<L* g, u> = L u in PyTorch's convention for C-linear maps
    lu = plan.apply(u)
    e = (g.grad - lu).abs().max().item() / lu.abs().max().item()
    plan.close()
    assert e < 1e-12


def test_real_input_gradient(env):
    """A real f goes through fio_apply_real; its gradient is the real part of
    the complex path's gradient (PyTorch's real-to-complex rule), and a central
    difference of the quadratic loss along a real direction matches it."""
    fio, ag, torch = env
    from paper_math_0610051_gb300 import synth
    N = 64
    plan = fio.Plan(N, fio.PHASE_ELLIPSE, synth.ellipse_params(), 1e-6, precision="fp64")
    g = torch.from_numpy(synth.white_noise(N, 1, seed=3, real=False)).cuda()
    fr = torch.from_numpy(synth.white_noise(N, 1, seed=4).real.copy()).cuda().requires_grad_(True)
    fc = fr.detach().to(torch.complex128).requires_grad_(True)

    def loss(f):
        return ((ag.fio_apply(f, plan) - g).abs() ** 2).sum()

    loss(fr).backward()
    loss(fc).backward()
    assert fr.grad.dtype == torch.float64
    e = (fr.grad - fc.grad.real).abs().max().item() / fc.grad.real.abs().max().item()
    assert e < 1e-12
    d = torch.from_numpy(np.random.default_rng(5).standard_normal((1, N, N))).cuda()
    h = 1e-3
    with torch.no_grad():
        fd = (loss(fr + h * d) - loss(fr - h * d)).item() / (2 * h)
    dd = (fr.grad * d).sum().item()
    plan.close()
    assert abs(fd - dd) <= 1e-9 * abs(dd)
