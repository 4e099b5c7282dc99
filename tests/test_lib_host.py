"""CPU tests of the C-ABI library: it loads, exports what include/fio.h declares,
and its host logic (wedges of Sec. 1.3, boxes of Sec. 3.4, Kaiser-Bessel kernel,
Hermitian eigensolver of Sec. 3.2, argument checks) is right.  No CUDA call."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fio():
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_math_0610051_gb300 import fio
    return fio


def _declared():
    with open(os.path.join(ROOT, "include", "fio.h")) as fh:
        src = fh.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fio_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(fio):
    lib = fio.lib()
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(fio.EXPORTS) == names


def test_version_and_status_strings(fio):
    lib = fio.lib()
    assert lib.fio_version() >= 100
    for s in range(7):
        assert lib.fio_status_string(s)


def test_default_wedges(fio):
    assert [fio.default_wedges(N) for N in (64, 256, 512, 1024)] == [8, 16, 24, 32]


def test_kb_width_rule(fio):
    assert fio.kb_width_for(1e-4) == 6
    assert fio.kb_width_for(1e-6) == 8


@pytest.mark.parametrize("N,L", [(64, 8), (128, 16), (256, 16), (512, 24)])
def test_wedge_partition(fio, N, L):
    """W_l = {(2l-1) pi/L <= arg xi < (2l+1) pi/L}: every xi in exactly one wedge, by angle."""
    wm = fio.wedge_map(N, L)
    k = np.arange(N) - N // 2
    K1, K2 = np.meshgrid(k, k, indexing="ij")
    th = np.mod(np.arctan2(K2, K1) + np.pi / L, 2 * np.pi)
    expect = np.floor(th / (2 * np.pi / L)).astype(int) % L
    expect[N // 2, N // 2] = 0
    assert np.array_equal(wm, expect)
    counts = np.bincount(wm.ravel(), minlength=L)
    assert counts.sum() == N * N and counts.min() > 0.5 * N * N / L


@pytest.mark.parametrize("N,L", [(64, 8), (256, 16), (1024, 32)])
def test_wedge_boxes(fio, N, L):
    """Sec. 3.4: xi' = M xi - xi_c maps the wedge into its box; M unimodular; grid >= sigma * box."""
    wm = fio.wedge_map(N, L)
    k = np.arange(N) - N // 2
    K1, K2 = np.meshgrid(k, k, indexing="ij")
    sigma, w = 2.0, 6
    total = 0
    for l in range(L):
        g = fio.wedge_geometry(N, L, sigma, w, l)
        M = np.array(g["M"]).reshape(2, 2)
        assert round(np.linalg.det(M)) == 1
        sel = wm == l
        pts = np.stack([K1[sel], K2[sel]])
        xp = M @ pts - np.array(g["xc"])[:, None]
        assert xp[0].min() == g["b1"] and xp[0].max() == g["b1"] + g["n1"] - 1
        assert xp[1].min() == g["b2"] and xp[1].max() == g["b2"] + g["n2"] - 1
        assert len({(a, b) for a, b in xp.T}) == g["npts"] == sel.sum()
        for m, n in ((g["m1"], g["n1"]), (g["m2"], g["n2"])):
            assert m >= sigma * n and m % 2 == 0
            r = m
            for p in (2, 3, 5):
                while r % p == 0:
                    r //= p
            assert r == 1
        total += g["n1"] * g["n2"]
    if N == 1024:
        # the sheared boxes cover about 2.9 N^2 frequencies in total
        assert total < 3.2 * N * N


def test_kb_kernel_matches_bessel_and_quadrature(fio):
    """phi(s) = I0(beta sqrt(1-(2s/w)^2))/I0(beta); phihat is its Fourier transform."""
    from scipy import integrate, special
    w, beta = 6, 13.855
    s = np.linspace(-3.2, 3.2, 41)
    phi, _ = fio.kb_eval(w, beta, s=s)
    z = 1 - (2 * s / w) ** 2
    ref = np.where(z > 0, special.i0(beta * np.sqrt(np.maximum(z, 0))) / special.i0(beta), 0)
    assert np.max(np.abs(phi - ref)) < 1e-13
    nu = np.array([0.0, 0.05, 0.1, 0.2, 0.25, 0.4, 0.7, 1.2])
    _, ph = fio.kb_eval(w, beta, nu=nu)
    for v, got in zip(nu, ph):
        f = lambda t: special.i0(beta * np.sqrt(max(1 - (2 * t / w) ** 2, 0))) / special.i0(beta) \
            * np.cos(2 * np.pi * v * t)
        q, _ = integrate.quad(f, -w / 2, w / 2, limit=200, epsabs=1e-14, epsrel=1e-13)
        assert abs(got - q) < 1e-10 * max(1.0, abs(q)), (v, got, q)


@pytest.mark.parametrize("eps", [1e-4, 1e-6])
def test_kb_nufft_accuracy(fio, eps):
    """The default width/shape for eps gives a 1D type-2 NUFFT error below eps / 5
    (sigma = 2), measured against the direct sum."""
    w = fio.kb_width_for(eps)
    g = np.random.default_rng(1)
    n, m = 120, 240
    k = np.arange(-n // 2, n // 2)
    F = g.standard_normal(n) + 1j * g.standard_normal(n)
    y = g.uniform(0, 1, 800)
    exact = np.exp(2j * np.pi * np.outer(y, k)) @ F
    _, ph = fio.kb_eval(w, 0.0, nu=k / m)
    G = np.zeros(m, complex)
    G[k % m] = F / ph
    Gg = np.fft.ifft(G) * m
    u = y * m
    j0 = np.floor(u - w / 2).astype(int) + 1
    res = np.zeros_like(exact)
    for a in range(w):
        j = j0 + a
        phi, _ = fio.kb_eval(w, 0.0, s=u - j)
        res += phi * Gg[j % m]
    err = np.linalg.norm(res - exact) / np.linalg.norm(exact)
    assert err < eps / 5, err


@pytest.mark.parametrize("n", [1, 5, 24, 70])
def test_host_eigh_matches_numpy(fio, n):
    g = np.random.default_rng(n)
    X = g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))
    A = X @ X.conj().T
    ev, V = fio.host_eigh(A)
    ref = np.sort(np.linalg.eigvalsh(A))[::-1]
    assert np.max(np.abs(ev - ref)) < 1e-11 * ref[0]
    assert np.max(np.abs(V.conj().T @ V - np.eye(n))) < 1e-11
    assert np.max(np.abs(A @ V - V * ev)) < 1e-10 * ref[0]


def test_host_eigh_rank_deficient(fio):
    """A Gram matrix of rank 3 (the situation of oversampled columns, Sec. 3.2)."""
    g = np.random.default_rng(7)
    B = g.standard_normal((40, 3)) + 1j * g.standard_normal((40, 3))
    A = B.conj().T @ B
    A = np.pad(A, ((0, 9), (0, 9)))
    C = g.standard_normal((12, 12)) + 1j * g.standard_normal((12, 12))
    Q, _ = np.linalg.qr(C)
    A = Q @ A @ Q.conj().T
    ev, V = fio.host_eigh(A)
    assert np.all(ev[3:] < 1e-12 * ev[0])
    assert np.max(np.abs(A @ V[:, :3] - V[:, :3] * ev[:3])) < 1e-10 * ev[0]


@pytest.mark.parametrize("case", ["plan_gram", "clusters", "diagonal", "zero", "tiny"])
def test_host_eigh_structured(fio, case):
    """Matrices of the kinds the separation meets: Gram matrices of unit-modulus
    phase columns (A_[C]^H A_[C]), two tight eigenvalue clusters, an already
    diagonal matrix, the zero matrix and the 1 x 1 and 2 x 2 cases."""
    g = np.random.default_rng(11)
    if case == "plan_gram":
        x = g.uniform(0, 1, (300, 1))
        k = g.uniform(-40, 40, (1, 96))
        Am = np.exp(2j * np.pi * (x * k + 0.3 * np.sin(2 * np.pi * x) * np.abs(k)))
        mats = [Am.conj().T @ Am]
    elif case == "clusters":
        X = g.standard_normal((120, 120)) + 1j * g.standard_normal((120, 120))
        Q, _ = np.linalg.qr(X)
        lam = np.concatenate([np.ones(60), 1e-9 * np.ones(60)])
        mats = [(Q * lam) @ Q.conj().T]
    elif case == "diagonal":
        mats = [np.diag(np.arange(16.0)).astype(complex)]
    elif case == "zero":
        mats = [np.zeros((7, 7), complex)]
    else:
        mats = [np.array([[2.5]], complex), np.array([[1.0, 2 - 1j], [2 + 1j, -3.0]])]
    for A in mats:
        n = A.shape[0]
        ev, V = fio.host_eigh(A)
        ref = np.sort(np.linalg.eigvalsh(A))[::-1]
        scale = max(np.max(np.abs(ref)), 1e-300)
        assert np.all(np.diff(ev) <= 1e-12 * scale)          # descending
        assert np.max(np.abs(ev - ref)) < 1e-12 * scale
        assert np.max(np.abs(V.conj().T @ V - np.eye(n))) < 1e-11
        assert np.max(np.abs(A @ V - V * ev)) < 1e-11 * scale + 1e-300


def test_plan_create_rejects_bad_arguments_before_cuda(fio):
    """Argument errors are reported before any CUDA call (FIO_EINVAL), with a message."""
    lib = fio.lib()
    prm = np.array([2 / 3, 1 / 3, 2 / 3, 1 / 3])
    bad = np.array([np.nan, 0, 1, 0])
    tau = np.array([[0.1, 1, 0, 2.5, 0.0]])

    def create(N, params, kind=fio.PHASE_ELLIPSE, eps=1e-4, nmodes=0):
        ph = fio._Phase(kind, nmodes, params.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        h = ctypes.c_void_p()
        st = lib.fio_plan_create(N, ctypes.byref(ph), None, eps, None, ctypes.byref(h))
        return st, h.value

    assert create(63, prm) == (fio.FIO_EINVAL, None)
    assert create(4, prm) == (fio.FIO_EINVAL, None)
    assert create(64, prm, eps=0.5)[0] == fio.FIO_EINVAL
    assert create(64, bad)[0] == fio.FIO_EINVAL
    assert b"non-finite" in lib.fio_last_error()
    assert create(64, tau.ravel().copy(), fio.PHASE_TAU_MODES, nmodes=1)[0] == fio.FIO_EINVAL
    assert lib.fio_apply(None, None, None, 1, None) == fio.FIO_EINVAL
    assert lib.fio_apply_normal(None, None, None, 1, None) == fio.FIO_EINVAL
    assert lib.fio_dft2(100 + 14, 0, None, None, 1, 0, None) == fio.FIO_EINVAL
    # phase kinds: unknown kind, and a non-finite product-form ellipse parameter
    assert create(64, prm, kind=4)[0] == fio.FIO_EINVAL
    assert create(64, bad, kind=fio.PHASE_ELLIPSE_PRODUCT)[0] == fio.FIO_EINVAL


def test_alpha_mode_options_are_validated_before_cuda(fio):
    """An unknown storage mode or a negative group size is FIO_EINVAL; the
    recompute mode of a complex64 plan with the Hankel amplitude is
    FIO_EUNSUPPORTED; all before any CUDA call."""
    lib = fio.lib()
    prm = np.array([2 / 3, 1 / 3, 2 / 3, 1 / 3])
    ph = fio._Phase(fio.PHASE_ELLIPSE, 0, prm.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))

    def create(mode, group=0, amp=None, precision=fio.MIXED):
        opt = fio._Options()
        lib.fio_options_default(ctypes.byref(opt))
        opt.alpha_mode, opt.alpha_group, opt.precision = mode, group, precision
        h = ctypes.c_void_p()
        st = lib.fio_plan_create(64, ctypes.byref(ph), ctypes.byref(amp) if amp else None, 1e-4,
                                 ctypes.byref(opt), ctypes.byref(h))
        return st, h.value

    opt = fio._Options()
    assert lib.fio_options_default(ctypes.byref(opt)) == fio.FIO_OK
    assert opt.alpha_mode == fio.ALPHA_STORED and opt.alpha_group == 0
    assert create(2) == (fio.FIO_EINVAL, None)
    assert create(-1) == (fio.FIO_EINVAL, None)
    assert create(fio.ALPHA_RECOMPUTE, group=-3) == (fio.FIO_EINVAL, None)
    hank = fio._Amp(fio.AMP_HANKEL, 1.0, 0.0)
    assert create(fio.ALPHA_RECOMPUTE, amp=hank) == (fio.FIO_EUNSUPPORTED, None)
    assert b"FP64" in lib.fio_last_error()


def test_hankel_amplitude_sign_is_validated(fio):
    """FIO_AMP_HANKEL takes its sign from a1, which must be +1 or -1."""
    lib = fio.lib()
    prm = np.ascontiguousarray(fio_synth().circle_grt_modes(1).ravel())
    ph = fio._Phase(fio.PHASE_TAU_MODES, 5, prm.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    for a1 in (0.5, 0.0, 2.0, np.nan):
        am = fio._Amp(fio.AMP_HANKEL, a1, 0.0)
        h = ctypes.c_void_p()
        st = lib.fio_plan_create(64, ctypes.byref(ph), ctypes.byref(am), 1e-4, None, ctypes.byref(h))
        assert (st, h.value) == (fio.FIO_EINVAL, None), a1
        assert b"amplitude" in lib.fio_last_error()


def fio_synth():
    from paper_math_0610051_gb300 import synth
    return synth


def _unitary(g, n):
    q, r = np.linalg.qr(g.standard_normal((n, n)) + 1j * g.standard_normal((n, n)))
    return q * (np.diag(r) / np.abs(np.diag(r)))


@pytest.mark.parametrize("m,n", [(1, 1), (5, 3), (40, 40), (200, 24), (7, 12)])
def test_host_svd_matches_numpy(fio, m, n):
    """One-sided Jacobi SVD (the solver of the randomized separation, Sec. 3.2)
    against LAPACK's: singular values, A V = AV, orthonormal V, orthogonal
    columns of AV with norms s."""
    g = np.random.default_rng(m * 131 + n)
    A = g.standard_normal((m, n)) + 1j * g.standard_normal((m, n))
    s, AV, V = fio.host_svd(A)
    ref = np.linalg.svd(A, compute_uv=False)
    k = min(m, n)
    assert np.all(np.diff(s) <= 0)
    assert np.max(np.abs(s[:k] - ref[:k])) < 1e-13 * ref[0]
    assert np.all(np.abs(s[k:]) < 1e-13 * ref[0])
    assert np.max(np.abs(A @ V - AV)) < 1e-13 * ref[0]
    assert np.max(np.abs(V.conj().T @ V - np.eye(n))) < 1e-13
    G = AV.conj().T @ AV
    assert np.max(np.abs(G - np.diag(s ** 2))) < 1e-13 * ref[0] ** 2


def test_host_svd_small_singular_values_keep_absolute_accuracy(fio):
    """A = U diag(s) V^H with s from 1 down to 1e-12: every computed singular value
    is within a few 1e-16 s_1 of the true one, as for a QR-based SVD.  The square
    roots of the eigenvalues of A^H A (the Gram route) miss the small ones: their
    error grows like 1e-16 s_1^2 / s_k."""
    g = np.random.default_rng(7)
    n, m = 16, 64
    sv = np.logspace(0, -12, n)
    U = _unitary(g, m)[:, :n]
    Vt = _unitary(g, n)
    A = (U * sv) @ Vt.conj().T
    s, AV, V = fio.host_svd(A)
    assert np.max(np.abs(s - sv)) < 2e-15
    # the Gram route, for contrast
    ev = np.linalg.eigvalsh(A.conj().T @ A)[::-1]
    gram = np.sqrt(np.maximum(ev, 0))
    assert np.max(np.abs(gram - sv)) > 1e-10
    # right singular vectors of well-separated singular values are accurate
    for k in range(4):
        assert abs(abs(np.vdot(V[:, k], Vt[:, k])) - 1) < 1e-12


def test_host_svd_rank_deficient_and_zero(fio):
    g = np.random.default_rng(3)
    B = g.standard_normal((30, 4)) + 1j * g.standard_normal((30, 4))
    A = B @ (g.standard_normal((4, 9)) + 1j * g.standard_normal((4, 9)))
    s, AV, V = fio.host_svd(A)
    ref = np.linalg.svd(A, compute_uv=False)
    assert np.max(np.abs(s[:4] - ref[:4])) < 1e-13 * ref[0]
    assert np.max(s[4:]) < 1e-13 * ref[0]
    s0, AV0, V0 = fio.host_svd(np.zeros((6, 3)))
    assert np.all(s0 == 0) and np.all(AV0 == 0)
    assert np.allclose(V0.conj().T @ V0, np.eye(3))


@pytest.mark.parametrize("n", [1, 7, 48, 130])
def test_host_svd_right_matches_numpy(fio, n):
    """The column-pivoted preconditioned Jacobi SVD applied to triangular factors
    (Sec. 3.2): singular values as LAPACK's, R V orthogonal columns of norms s,
    V unitary; graded factors keep the small singular values."""
    g = np.random.default_rng(n)
    R = np.triu(g.standard_normal((n, n)) + 1j * g.standard_normal((n, n)))
    R = R * np.logspace(0, -10, n)[None, :]
    s, V = fio.host_svd_right(R)
    ref = np.linalg.svd(R, compute_uv=False)
    assert np.max(np.abs(s - ref)) < 1e-13 * ref[0]
    # a singular vector is determined to about 1e-16 s_1 / s_k: check those of
    # singular values above 1e-8 s_1 (the separation keeps s_k > 0.25 eps s_1)
    k = int(np.sum(s > 1e-8 * s[0]))
    Vk = V[:, :k]
    assert np.max(np.abs(Vk.conj().T @ Vk - np.eye(k))) < 1e-7
    RV = R @ Vk
    assert np.max(np.abs(RV.conj().T @ RV - np.diag(s[:k] ** 2))) < 1e-13 * ref[0] ** 2


def test_host_svd_right_rank_deficient(fio):
    g = np.random.default_rng(5)
    R = (g.standard_normal((20, 3)) + 1j * g.standard_normal((20, 3))) @ (g.standard_normal((3, 20)))
    s, V = fio.host_svd_right(R)
    ref = np.linalg.svd(R, compute_uv=False)
    assert np.max(np.abs(s[:3] - ref[:3])) < 1e-13 * ref[0]
    assert np.all(s[3:] < 1e-13 * ref[0])
    RV = R @ V[:, :3]
    assert np.max(np.abs(RV.conj().T @ RV - np.diag(s[:3] ** 2))) < 1e-12 * ref[0] ** 2


def test_plan_load_rejects_bad_files_without_a_gpu(fio, tmp_path):
    """fio_plan_load reads and checks the file's header before any CUDA call: a
    missing file, a foreign file and a plan file of a truncated header are
    FIO_EINVAL, and no plan is returned."""
    lib = fio.lib()
    bad = os.path.join(tmp_path, "bad.fioplan")
    with open(bad, "wb") as fh:
        fh.write(b"NOTAPLAN" + bytes(64))
    short = os.path.join(tmp_path, "short.fioplan")
    with open(short, "wb") as fh:
        fh.write(b"FIOPLAN1" + (1).to_bytes(4, "little"))
    # a file of the previous format version, and a current header whose storage
    # mode is unknown: both rejected from the header alone
    import struct

    def header(version, alpha_mode):
        ints = [64, 8, 0, 1, 6, 10, 8, 64, 0, 100, 500, 10, 10, 10, 40, 0]
        dbl = [1e-4, 2.0, 14.0, 5e-5, 9.0, 1.0, 0.0, 0.0, 50.0]
        i64 = [1000, 1000, 1000, 1000, 100, 1000]
        return (b"FIOPLAN1" + struct.pack("<II", version, 0x01020304) +
                struct.pack("<16i9d6q", *ints, *dbl, *i64) +
                struct.pack("<2i3q", alpha_mode, 0, 0, 0, 0))

    old_ver = os.path.join(tmp_path, "v1.fioplan")
    with open(old_ver, "wb") as fh:
        fh.write(header(1, 0))
    bad_mode = os.path.join(tmp_path, "mode.fioplan")
    with open(bad_mode, "wb") as fh:
        fh.write(header(2, 7))
    for path in (bad, short, os.path.join(tmp_path, "missing.fioplan"), old_ver, bad_mode):
        h = ctypes.c_void_p(1)
        assert lib.fio_plan_load(os.fsencode(path), 0, ctypes.byref(h)) == fio.FIO_EINVAL
        assert not h.value
        assert b"fio_plan_load" in lib.fio_last_error()
    assert b"corrupt plan header" in lib.fio_last_error()
    # control: the same header with a valid mode passes the header checks and
    # stops at the missing tables, so the check above is the mode's
    good_mode = os.path.join(tmp_path, "good.fioplan")
    with open(good_mode, "wb") as fh:
        fh.write(header(2, fio.ALPHA_RECOMPUTE))
    h = ctypes.c_void_p(1)
    assert lib.fio_plan_load(os.fsencode(good_mode), 0, ctypes.byref(h)) == fio.FIO_EINVAL
    assert not h.value
    assert b"host tables" in lib.fio_last_error()


def test_autograd_functions_reachable_from_fio(fio):
    """fio.FIOApply / fio.FIOAdjoint are the autograd functions (imported on use)."""
    pytest.importorskip("torch")
    from paper_math_0610051_gb300 import autograd
    assert fio.FIOApply is autograd.FIOApply and fio.FIOAdjoint is autograd.FIOAdjoint
    with pytest.raises(AttributeError):
        fio.no_such_name
