"""GPU parity of the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances (rel-L2 over all compared outputs, the error measure of Sec. 4):
the mixed path (complex64 FFT/NUFFT) must stay within 1e-4 at eps = 1e-4, the
FP64 path within 1e-6 at eps = 1e-6.  Phases whose residual is exactly rank 1
(identity, translation, wave multiplier) carry no separation error, so they
must reach the NUFFT accuracy alone (eps / 3).
"""
import os

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


def dev(torch, a, prec):
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    return torch.from_numpy(np.ascontiguousarray(a)).to(dt).cuda()


def rel(ref, got):
    ref = np.asarray(ref).ravel()
    got = np.asarray(got).ravel()
    return float(np.linalg.norm(ref - got) / np.linalg.norm(ref))


PREC_EPS = [("mixed", 1e-4), ("fp64", 1e-6)]


# ------------------------------------------------------------------ S0 -------

@pytest.mark.parametrize("N", [8, 16, 64, 96, 120, 1024])
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_dft2_matches_oracle(env, orc, N, prec):
    fio, torch = env
    from paper_math_0610051_gb300 import synth
    B = 3 if N <= 128 else 1
    f = synth.white_noise(N, B, seed=N, real=False)
    fh = fio.dft2(dev(torch, f, prec)).cpu().numpy()
    back = fio.dft2(dev(torch, fh, prec), inverse=True).cpu().numpy()
    tol = 1e-12 if prec == "fp64" else 2e-6
    for b in range(B):
        assert rel(orc.dft2(f[b]), fh[b]) < tol
        assert rel(f[b], back[b]) < 2 * tol


# ------------------------------------------------- exact rank-1 phases -------

@pytest.mark.parametrize("prec,eps", PREC_EPS)
@pytest.mark.parametrize("name,params", [("identity", [0, 0, 0]), ("shift", [3 / 64, 5 / 64, 0]),
                                         ("wave", [0, 0, 0.3]), ("shift_wave", [0.11, -0.27, 1.7])])
def test_rank_one_phases(env, orc, prec, eps, name, params):
    fio, torch = env
    from paper_math_0610051_gb300 import synth
    N, B = 64, 2
    f = synth.white_noise(N, B, seed=5, real=False)
    with fio.Plan(N, fio.PHASE_SHIFT_WAVE, params, eps, precision=prec, max_batch=B) as plan:
        assert plan.info()["q_max"] == 1
        out = plan.apply(dev(torch, f, prec)).cpu().numpy()
    ph = orc.Phase(orc.SHIFT_WAVE, params)
    for b in range(B):
        ref = orc.apply_dense(ph, orc.Amplitude(), f[b])
        assert rel(ref, out[b]) < eps / 3, (name, b)


# ----------------------------------------------- configs: dense at N = 64 ----

@pytest.mark.parametrize("prec,eps", PREC_EPS)
@pytest.mark.parametrize("N", [48, 64])
def test_ellipse_dense(env, orc, prec, eps, N):
    """Ellipse phase, a = 1, f ~ N(0,1): the whole grid against the O(N^4) oracle."""
    fio, torch = env
    from paper_math_0610051_gb300 import synth
    prm = synth.ellipse_params()
    f = synth.white_noise(N, 1, seed=11)
    with fio.Plan(N, fio.PHASE_ELLIPSE, prm, eps, precision=prec) as plan:
        out = plan.apply(dev(torch, f, prec)).cpu().numpy()[0]
    ref = orc.apply_dense(orc.Phase(orc.ELLIPSE, prm), orc.Amplitude(), f[0])
    assert rel(ref, out) < eps


@pytest.mark.parametrize("N", [8, 16])
def test_tiny_grids(env, orc, N):
    fio, torch = env
    from paper_math_0610051_gb300 import synth
    prm = synth.ellipse_params()
    f = synth.white_noise(N, 1, seed=3, real=False)
    with fio.Plan(N, fio.PHASE_ELLIPSE, prm, 1e-6, precision="fp64") as plan:
        out = plan.apply(dev(torch, f, "fp64")).cpu().numpy()[0]
        adj = plan.adjoint(dev(torch, f, "fp64")).cpu().numpy()[0]
        plan.sync()
    ph = orc.Phase(orc.ELLIPSE, prm)
    assert rel(orc.apply_dense(ph, orc.Amplitude(), f[0]), out) < 1e-6
    assert rel(orc.adjoint_dense(ph, orc.Amplitude(), f[0]), adj) < 1e-6


# ------------------------------------------- configs: sampled at N = 256/512 -

@pytest.mark.parametrize("N", [256, 512])
@pytest.mark.parametrize("prec,eps", PREC_EPS)
def test_ellipse_sampled(env, orc, N, prec, eps):
    """Smooth noise plus sharp discs; the oracle's direct sums at 512 random x."""
    fio, torch = env
    from paper_math_0610051_gb300 import synth
    prm = synth.ellipse_params()
    f = synth.smooth_noise_discs(N, seed=N)
    with fio.Plan(N, fio.PHASE_ELLIPSE, prm, eps, precision=prec) as plan:
        out = plan.apply(dev(torch, f[None], prec)).cpu().numpy()[0]
        plan.sync()  # raises if an in-kernel bounds check fired
    n1, n2 = synth.sample_points(N, 512, seed=1)
    ref = orc.apply_points(orc.Phase(orc.ELLIPSE, prm), orc.Amplitude(), orc.dft2(f), n1, n2)
    assert rel(ref, out[n1, n2]) < eps


def test_mixed_vs_fp64_full_grid(env):
    """At N = 512 the mixed path tracks the FP64 path on every output to 1e-4."""
    fio, torch = env
    from paper_math_0610051_gb300 import synth
    N = 512
    prm = synth.ellipse_params()
    f = synth.white_noise(N, 1, seed=21)
    with fio.Plan(N, fio.PHASE_ELLIPSE, prm, 1e-6, precision="fp64") as p64:
        ref = p64.apply(dev(torch, f, "fp64")).cpu().numpy()
    with fio.Plan(N, fio.PHASE_ELLIPSE, prm, 1e-4) as p32:
        out = p32.apply(dev(torch, f, "mixed")).cpu().numpy()
    assert rel(ref, out) < 1e-4


def test_tau_modes_amplitude_batch(env, orc):
    """N = 512, tau with 32 modes, a = (1 + 0.5 sin 2pi x1)(1 + 0.3 cos theta), 8 inputs in one launch."""
    fio, torch = env
    from paper_math_0610051_gb300 import synth
    N, B = 512, 8
    prm = synth.tau_mode_params(32, seed=3)
    f = synth.white_noise(N, B, seed=31)
    with fio.Plan(N, fio.PHASE_TAU_MODES, prm, 1e-4, amp=(0.5, 0.3), max_batch=B) as plan:
        x = dev(torch, f, "mixed")
        out = plan.apply(x).cpu().numpy()
        one = plan.apply(x[5:6].clone()).cpu().numpy()
        adj = plan.adjoint(x).cpu().numpy()
        adj_one = plan.adjoint(x[5:6].clone()).cpu().numpy()
        adj_again = plan.adjoint(x).cpu().numpy()
        plan.sync()
    # Batching changes only the order of the sums: the forward sum over wedges is
    # an atomic add, and the spread's lane layout depends on how many channels a
    # grid cell holds.  The adjoint has no atomics: a repeated call is bit-identical.
    assert rel(out[5], one[0]) < 1e-6
    assert rel(adj[5], adj_one[0]) < 1e-6
    assert np.array_equal(adj, adj_again)
    ph, amp = orc.Phase(orc.TAU_MODES, prm), orc.Amplitude(1, 0.5, 0.3)
    n1, n2 = synth.sample_points(N, 256, seed=2)
    for b in (0, 7):
        ref = orc.apply_points(ph, amp, orc.dft2(f[b]), n1, n2)
        assert rel(ref, out[b][n1, n2]) < 1e-4


# ------------------------------------------------------------ adjoint --------

@pytest.mark.parametrize("prec,eps", PREC_EPS)
def test_adjoint_dense(env, orc, prec, eps):
    fio, torch = env
    from paper_math_0610051_gb300 import synth
    N = 64
    prm = synth.tau_mode_params(8, seed=5)
    g = synth.white_noise(N, 2, seed=41, real=False)
    with fio.Plan(N, fio.PHASE_TAU_MODES, prm, eps, amp=(0.5, 0.3), precision=prec,
                  max_batch=2) as plan:
        adj = plan.adjoint(dev(torch, g, prec)).cpu().numpy()
    ph, amp = orc.Phase(orc.TAU_MODES, prm), orc.Amplitude(1, 0.5, 0.3)
    for b in range(2):
        assert rel(orc.adjoint_dense(ph, amp, g[b]), adj[b]) < eps


@pytest.mark.parametrize("prec,tol", [("mixed", 2e-5), ("fp64", 1e-12)])
def test_adjoint_identity_fast_path(env, prec, tol):
    """<L f, g> = <f, L* g> for the fast operators themselves (to rounding)."""
    fio, torch = env
    from paper_math_0610051_gb300 import synth
    N = 256
    prm = synth.ellipse_params()
    f = synth.white_noise(N, 1, seed=51, real=False)
    g = synth.white_noise(N, 1, seed=52, real=False)
    with fio.Plan(N, fio.PHASE_ELLIPSE, prm, 1e-4, amp=(0.2, -0.4), precision=prec) as plan:
        lf = plan.apply(dev(torch, f, prec)).cpu().numpy()
        lsg = plan.adjoint(dev(torch, g, prec)).cpu().numpy()
    a, b = np.vdot(g, lf), np.vdot(lsg, f)
    assert abs(a - b) / (np.linalg.norm(lf) * np.linalg.norm(g)) < tol


def test_adjoint_sampled_spectrum(env, orc):
    """N = 512: the spectrum of L* g at 256 random xi against the oracle's direct sums."""
    fio, torch = env
    from paper_math_0610051_gb300 import synth
    N = 512
    prm = synth.ellipse_params()
    g = synth.white_noise(N, 1, seed=61, real=False)
    with fio.Plan(N, fio.PHASE_ELLIPSE, prm, 1e-4) as plan:
        adj = plan.adjoint(dev(torch, g, "mixed")).cpu().numpy()[0]
    k1, k2 = synth.sample_freqs(N, 256, seed=3)
    ref = orc.adjoint_hat_points(orc.Phase(orc.ELLIPSE, prm), orc.Amplitude(), g[0], k1, k2)
    got = orc.dft2(adj)[k1 + N // 2, k2 + N // 2]
    assert rel(ref, got) < 1e-4


def test_full_size_bench_configuration(env, orc):
    """N = 1024, the bench's launch configuration (batch of 8 white-noise inputs,
    eps = 1e-4, mixed): the forward at 256 random x of inputs 0 and 7 and the
    adjoint spectrum at 128 random xi of input 3, against the oracle's direct sums."""
    fio, torch = env
    from paper_math_0610051_gb300 import synth
    N, B = 1024, 8
    prm = synth.ellipse_params()
    ph = orc.Phase(orc.ELLIPSE, prm)
    f = synth.white_noise(N, B, seed=10)
    g = synth.white_noise(N, B, seed=5000, real=False)
    with fio.Plan(N, fio.PHASE_ELLIPSE, prm, 1e-4, max_batch=B) as plan:
        out = plan.apply(dev(torch, f, "mixed")).cpu().numpy()
        adj = plan.adjoint(dev(torch, g, "mixed")).cpu().numpy()
        plan.sync()
    n1, n2 = synth.sample_points(N, 256, seed=4)
    for b in (0, 7):
        ref = orc.apply_points(ph, orc.Amplitude(), orc.dft2(f[b]), n1, n2)
        assert rel(ref, out[b][n1, n2]) < 1e-4
    k1, k2 = synth.sample_freqs(N, 128, seed=5)
    ref = orc.adjoint_hat_points(ph, orc.Amplitude(), g[3], k1, k2)
    got = orc.dft2(adj[3])[k1 + N // 2, k2 + N // 2]
    assert rel(ref, got) < 1e-4


# ------------------------------------------------ separation (Table 1) -------

@pytest.mark.parametrize("eps", [1e-4, 1e-6])
def test_separation_error_estimator(env, orc, eps):
    """The estimator of Sec. 4 (Table 1): s x s random submatrix, relative Frobenius
    error of the factors against the exact kernel, must be below eps."""
    fio, torch = env
    from paper_math_0610051_gb300 import synth
    N, s = 128, 200
    prm = synth.ellipse_params()
    ph = orc.Phase(orc.ELLIPSE, prm)
    rng = np.random.default_rng(9)
    with fio.Plan(N, fio.PHASE_ELLIPSE, prm, eps, precision="fp64") as plan:
        L = plan.info()["L"]
        for l in (0, L // 8, L // 4 + 1):
            w = plan.wedge(l)
            alpha, beta, k1, k2 = plan.export_wedge(l)
            y = plan.export_warp(l)
            rows = rng.choice(N * N, s, replace=False)
            cols = rng.choice(w["npts"], min(s, w["npts"]), replace=False)
            n1, n2 = rows // N, rows % N
            M = np.array(w["M"]).reshape(2, 2)
            kk = M @ np.stack([k1[cols], k2[cols]])
            X1 = np.repeat(n1 / N, len(cols))
            X2 = np.repeat(n2 / N, len(cols))
            K1 = np.tile(k1[cols], s)
            K2 = np.tile(k2[cols], s)
            phi = orc.phase_eval(ph, X1, X2, K1, K2).reshape(s, len(cols))
            lin = y[n1, n2, 0][:, None] * kk[0][None, :] + y[n1, n2, 1][:, None] * kk[1][None, :]
            A = np.exp(2j * np.pi * (phi - lin))
            UT = alpha[:, n1, n2].T @ beta[:, cols]
            err = np.linalg.norm(A - UT) / np.linalg.norm(A)
            assert err < eps, (l, err, w["q"])


# ----------------------------------------------------------- error paths -----

@pytest.mark.parametrize("prec,eps", PREC_EPS)
def test_real_input_entry(env, orc, prec, eps):
    """fio_apply_real on a real batch against the O(N^4) oracle, and against
    fio_apply on the same values as complex (the sum over wedges is an atomic
    float sum, so the two agree to rounding, not bit for bit)."""
    fio, torch = env
    from paper_math_0610051_gb300 import synth
    N, B = 48, 3
    prm = synth.ellipse_params()
    f = synth.white_noise(N, B, seed=12).real
    rdt = torch.float64 if prec == "fp64" else torch.float32
    with fio.Plan(N, fio.PHASE_ELLIPSE, prm, eps, precision=prec, max_batch=B) as plan:
        fr = torch.from_numpy(np.ascontiguousarray(f)).to(rdt).cuda()
        out_r = plan.apply(fr).cpu().numpy()
        out_c = plan.apply(dev(torch, f, prec)).cpu().numpy()
        assert out_r.dtype == (np.complex128 if prec == "fp64" else np.complex64)
        # an output that overlaps the real input is refused before any launch
        buf = torch.zeros(B * N * N, dtype=plan.dtype, device="cuda")
        tail = torch.view_as_real(buf).view(-1)[B * N * N:]
        st = fio.lib().fio_apply_real(plan._handle, tail.data_ptr(), buf.data_ptr(), B, None)
        assert st == fio.FIO_EINVAL
    ref = orc.apply_dense(orc.Phase(orc.ELLIPSE, prm), orc.Amplitude(), f[1])
    assert rel(ref, out_r[1]) < eps
    assert rel(out_c, out_r) < (1e-12 if prec == "fp64" else 1e-6)


def test_batch_limit_and_dtype_errors(env):
    fio, torch = env
    from paper_math_0610051_gb300 import synth
    with fio.Plan(32, fio.PHASE_ELLIPSE, synth.ellipse_params(), 1e-3) as plan:
        x = torch.zeros(2, 32, 32, dtype=torch.complex64, device="cuda")
        with pytest.raises(fio.FioError) as e:
            plan.apply(x)
        assert e.value.status == fio.FIO_EINVAL
        with pytest.raises(fio.FioError):
            plan.apply(torch.zeros(1, 32, 32, dtype=torch.complex128, device="cuda"))


def test_injected_allocation_failure_leaks_nothing(env):
    """FIO_FAULT_ALLOC=k makes the k-th device allocation of fio_plan_create fail:
    FIO_ENOMEM, and every allocation made before it is released."""
    fio, torch = env
    from paper_math_0610051_gb300 import synth
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for k in (1, 3, 6, 9):
        os.environ["FIO_FAULT_ALLOC"] = str(k)
        try:
            with pytest.raises(fio.FioError) as e:
                fio.Plan(64, fio.PHASE_ELLIPSE, synth.ellipse_params(), 1e-4)
            assert e.value.status == fio.FIO_ENOMEM
        finally:
            del os.environ["FIO_FAULT_ALLOC"]
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) < (8 << 20)
