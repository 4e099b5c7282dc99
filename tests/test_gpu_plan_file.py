"""fio_plan_save / fio_plan_load: a saved plan rebuilt in place of the
preprocessing of Sec. 3.2.  The loaded plan must apply the same operator with
the same arithmetic: its adjoint (no atomics) is bit-identical, its forward
equal up to the rounding order of the atomic sum over wedges, and saving it
again gives the same file, byte for byte."""
import filecmp
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
    __graft_entry__.build_library()
    from paper_math_0610051_gb300 import fio
    return fio, torch


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_save_load_round_trip(env, tmp_path, prec):
    fio, torch = env
    from paper_math_0610051_gb300 import synth
    N, B = 64, 2
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    f = torch.from_numpy(synth.white_noise(N, B, seed=4, real=False)).to(dt).cuda()
    p1 = os.path.join(tmp_path, "a.fioplan")
    p2 = os.path.join(tmp_path, "b.fioplan")
    with fio.Plan(N, fio.PHASE_ELLIPSE, synth.ellipse_params(), 1e-4, precision=prec,
                  max_batch=B) as plan:
        ref_f = plan.apply(f).cpu().numpy()
        ref_a = plan.adjoint(f).cpu().numpy()
        info = plan.info()
        plan.save(p1)
    loaded = fio.Plan.load(p1)
    try:
        got_a = loaded.adjoint(f).cpu().numpy()
        got_f = loaded.apply(f).cpu().numpy()
        li = loaded.info()
        loaded.save(p2)
    finally:
        loaded.close()
    assert np.array_equal(got_a, ref_a)
    tol = 1e-12 if prec == "fp64" else 1e-6
    assert np.linalg.norm(got_f - ref_f) <= tol * np.linalg.norm(ref_f)
    for k in ("N", "L", "q_mean", "q_max", "r_max", "sep_error", "grid_points", "bytes_alpha",
              "max_batch", "kb_width"):
        assert li[k] == info[k], k
    assert filecmp.cmp(p1, p2, shallow=False)


def test_load_with_a_larger_batch(env, tmp_path):
    fio, torch = env
    from paper_math_0610051_gb300 import synth
    N = 64
    path = os.path.join(tmp_path, "p.fioplan")
    with fio.Plan(N, fio.PHASE_ELLIPSE, synth.ellipse_params(), 1e-4) as plan:
        plan.save(path)
        g = torch.from_numpy(synth.white_noise(N, 3, seed=9, real=False)).to(torch.complex64).cuda()
        one = [plan.adjoint(g[b:b + 1]).cpu().numpy()[0] for b in range(3)]
    with fio.Plan.load(path, max_batch=3) as big:
        assert big.info()["max_batch"] == 3
        got = big.adjoint(g).cpu().numpy()
    for b in range(3):
        assert np.linalg.norm(got[b] - one[b]) <= 1e-6 * np.linalg.norm(one[b])


def test_load_rejects_bad_files(env, tmp_path):
    fio, _ = env
    bad = os.path.join(tmp_path, "bad.fioplan")
    with open(bad, "wb") as fh:
        fh.write(b"NOTAPLAN" + bytes(64))
    for path in (bad, os.path.join(tmp_path, "missing.fioplan")):
        with pytest.raises(fio.FioError) as e:
            fio.Plan.load(path)
        assert e.value.status == fio.FIO_EINVAL
