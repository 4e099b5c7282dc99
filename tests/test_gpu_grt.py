"""Integration along circles (the variable-amplitude experiment of Sec. 4 with
the Hankel amplitudes of Appendix A) through the CUDA path, against the oracle:
L+ dense in FP64, L+ + L- dense in mixed precision, L+ sampled at N = 256."""
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


def _plan(fio, N, sign, eps, prec):
    from paper_math_0610051_gb300 import synth
    return fio.Plan(N, fio.PHASE_TAU_MODES, synth.circle_grt_modes(sign), eps, amp=("hankel", sign),
                    precision=prec)


def test_grt_plus_dense_fp64(env, orc):
    fio, torch = env
    from paper_math_0610051_gb300 import synth
    N = 64
    f = synth.white_noise(N, 1, seed=21)
    g = synth.white_noise(N, 1, seed=22, real=False)
    ph = orc.Phase(orc.TAU_MODES, synth.circle_grt_modes(1))
    am = orc.Amplitude(orc.AMP_HANKEL, 1)
    with _plan(fio, N, 1, 1e-6, "fp64") as plan:
        out = plan.apply(torch.from_numpy(f).cuda()).cpu().numpy()[0]
        adj = plan.adjoint(torch.from_numpy(g).cuda()).cpu().numpy()[0]
        plan.sync()
    assert _rel(orc.apply_dense(ph, am, f[0]), out) < 1e-6
    assert _rel(orc.adjoint_dense(ph, am, g[0]), adj) < 1e-6


def test_grt_sum_dense_mixed(env, orc):
    fio, torch = env
    from paper_math_0610051_gb300 import synth
    N = 64
    f = synth.white_noise(N, 1, seed=23)
    got = 0
    ref = 0
    for s in (1, -1):
        with _plan(fio, N, s, 1e-4, "mixed") as plan:
            got = got + plan.apply(torch.from_numpy(f).to(torch.complex64).cuda()).cpu().numpy()[0]
        ph = orc.Phase(orc.TAU_MODES, synth.circle_grt_modes(s))
        ref = ref + orc.apply_dense(ph, orc.Amplitude(orc.AMP_HANKEL, s), f[0])
    assert _rel(ref, got) < 1e-4


def test_grt_plus_sampled_256(env, orc):
    fio, torch = env
    from paper_math_0610051_gb300 import synth
    N = 256
    f = synth.white_noise(N, 1, seed=24)
    with _plan(fio, N, 1, 1e-4, "mixed") as plan:
        out = plan.apply(torch.from_numpy(f).to(torch.complex64).cuda()).cpu().numpy()[0]
        info = plan.info()
    n1, n2 = synth.sample_points(N, 256, seed=6)
    ph = orc.Phase(orc.TAU_MODES, synth.circle_grt_modes(1))
    ref = orc.apply_points(ph, orc.Amplitude(orc.AMP_HANKEL, 1), orc.dft2(f[0]), n1, n2)
    err = _rel(ref, out[n1, n2])
    print(f"\nGRT L+ N=256 eps=1e-4: rel-L2 {err:.2e}, q mean {info['q_mean']:.1f}, "
          f"q max {info['q_max']}, plan {info['plan_seconds']:.2f} s")
    assert err < 1e-4
