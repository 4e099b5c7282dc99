"""The normal operator L* L in one call (fio_apply_normal): against the two
separate calls, against the oracle's dense L* L, and its defining identity
<L* L f, f> = ||L f||^2 (real, non-negative)."""
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
    from paper_math_0610051_gb300 import fio
    return fio, torch


def _rel(a, b):
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(a))


def test_normal_equals_adjoint_of_apply(env):
    fio, torch = env
    from paper_math_0610051_gb300 import synth
    N, B = 256, 2
    f = torch.from_numpy(synth.smooth_noise_discs(N, seed=4)[None].repeat(B, 0)).to(torch.complex64).cuda()
    f[1] *= 1j
    with fio.Plan(N, fio.PHASE_ELLIPSE, synth.ellipse_params(), 1e-4, max_batch=B) as plan:
        two = plan.adjoint(plan.apply(f)).cpu().numpy()
        one = plan.normal(f).cpu().numpy()
        plan.sync()
    # the forward's atomic sum over wedges may round in another order
    assert _rel(two, one) < 1e-6


def test_normal_matches_dense_oracle_fp64(env, orc):
    fio, torch = env
    from paper_math_0610051_gb300 import synth
    N = 64
    prm = synth.ellipse_params()
    f = synth.white_noise(N, 1, seed=8)
    with fio.Plan(N, fio.PHASE_ELLIPSE, prm, 1e-6, precision="fp64") as plan:
        got = plan.normal(torch.from_numpy(f).cuda()).cpu().numpy()[0]
    ph, amp = orc.Phase(orc.ELLIPSE, prm), orc.Amplitude()
    ref = orc.adjoint_dense(ph, amp, orc.apply_dense(ph, amp, f[0]))
    assert _rel(ref, got) < 2e-6


def test_normal_is_positive_semidefinite(env):
    fio, torch = env
    from paper_math_0610051_gb300 import synth
    N = 128
    f = torch.from_numpy(synth.white_noise(N, 1, seed=9, real=False)).cuda()
    with fio.Plan(N, fio.PHASE_TAU_MODES, synth.tau_mode_params(16, seed=2), 1e-6,
                  amp=(0.5, 0.3), precision="fp64") as plan:
        n = plan.normal(f)
        lf = plan.apply(f)
    ip = torch.vdot(f.flatten(), n.flatten()).item()  # <f, L* L f> = ||L f||^2
    nrm = torch.linalg.vector_norm(lf).item() ** 2
    assert abs(ip.imag) < 1e-10 * nrm
    assert abs(ip.real - nrm) < 1e-10 * nrm
