"""Reproduction, on the GPU plan, of the separation experiments of Sec. 4 on the
paper's own phase (Eq. nrphase, product-form axes): Table 1 (the randomized
separation's relative error stays below eps) and Table 2 (ranks for
eps = N^-p grow with p and gently with N).  Ranks are random-sample dependent
and our acceptance test is stricter, so Table 2 is a shape check, not parity;
the paper's values are printed beside ours.  At N = 64 the wedges are small
enough that tight eps samples every column; the separation then takes the
exact projection T = S V^H of the full block."""
import numpy as np
import pytest

PAPER_RANKS = {64: [7, 10, 14, 18, 22], 128: [9, 12, 17, 21, 24], 256: [9, 12, 17, 21, 25],
               512: [10, 15, 19, 24, 27]}  # Table 2, p = 1, 1.5, 2, 2.5, 3


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_math_0610051_gb300 import fio
    return fio, torch


@pytest.mark.gpu
def test_paper_phase_dense(env, orc):
    fio, torch = env
    from paper_math_0610051_gb300 import synth
    N = 64
    prm = synth.paper_ellipse_params()
    f = synth.white_noise(N, 1, seed=31)
    with fio.Plan(N, fio.PHASE_ELLIPSE_PRODUCT, prm, 1e-4) as plan:
        out = plan.apply(torch.from_numpy(f).to(torch.complex64).cuda()).cpu().numpy()[0]
    ref = orc.apply_dense(orc.Phase(orc.ELLIPSE_PRODUCT, prm), orc.Amplitude(), f[0])
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) < 1e-4


def _plan_or_cap(fio, N, prm, eps):
    """The plan's info, or None when the separation needs more than rank_cap
    columns (FIO_ERANK)."""
    try:
        with fio.Plan(N, fio.PHASE_ELLIPSE_PRODUCT, prm, eps) as plan:
            return plan.info()
    except fio.FioError as e:
        if e.status != fio.FIO_ERANK:
            raise
        return None


@pytest.mark.gpu_long
def test_table1_separation_error(env):
    """Every plan that is built meets eps; the ones that would need more than
    rank_cap sampled columns are reported (FIO_ERANK), and there are none up to
    N = 256."""
    fio, _ = env
    from paper_math_0610051_gb300 import synth
    prm = synth.paper_ellipse_params()
    rows, capped = [], []
    for N in (64, 128, 256, 512):
        errs = []
        for eps in (1e-3, 1e-4, 1e-5, 1e-6):
            info = _plan_or_cap(fio, N, prm, eps)
            if info is None:
                capped.append((N, eps))
                errs.append(float("nan"))
                print(f"Table 1: N={N} eps={eps:g} needs more than rank_cap columns", flush=True)
                continue
            errs.append(info["sep_error"])
            print(f"Table 1: N={N} eps={eps:g} error {errs[-1]:.2e} q mean {info['q_mean']:.1f} "
                  f"r max {info['r_max']} plan {info['plan_seconds']:.1f} s", flush=True)
            assert errs[-1] <= eps, (N, eps, errs[-1])
        rows.append(f"N={N:4d}  " + "  ".join(f"{e:.2e}" for e in errs))
    print("\nTable 1 (largest per-wedge separation error, eps = 1e-3 .. 1e-6):\n" + "\n".join(rows))
    assert all(N > 256 for N, _ in capped), capped


@pytest.mark.gpu_long
def test_table2_ranks(env):
    fio, _ = env
    from paper_math_0610051_gb300 import synth
    prm = synth.paper_ellipse_params()
    lines = []
    for N, paper in PAPER_RANKS.items():
        qs = []
        for p in (1.0, 1.5, 2.0, 2.5, 3.0):
            info = _plan_or_cap(fio, N, prm, float(N) ** -p)
            if info is None:  # needs more than rank_cap columns: the rest of the row too
                print(f"Table 2: N={N} p={p} needs more than rank_cap columns", flush=True)
                break
            qs.append((info["q_max"], info["q_mean"]))
            print(f"Table 2: N={N} p={p} q max {qs[-1][0]} mean {qs[-1][1]:.1f} "
                  f"error {info['sep_error']:.2e} plan {info['plan_seconds']:.1f} s", flush=True)
        assert len(qs) >= 3, (N, qs)
        assert all(b[0] >= a[0] for a, b in zip(qs, qs[1:])), (N, qs)  # grows with p
        lines.append(f"N={N:4d}  ours (max/mean) " +
                     "  ".join(f"{m:2d}/{a:4.1f}" for m, a in qs) + "   paper " + " ".join(map(str, paper)))
    print("\nTable 2 (ranks for eps = N^-p, p = 1, 1.5, 2, 2.5, 3):\n" + "\n".join(lines))
