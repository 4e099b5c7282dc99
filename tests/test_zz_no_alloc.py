"""fio_apply_noalloc: the forward apply on the library's fixed scratch array.

It is meant for callers that cannot allocate device memory while they run (a
framework that owns all device memory through its own pool, a real-time loop
that cannot risk an allocation's latency or failure).  It must give what
fio_apply gives, call after call, and refuse sizes beyond the scratch array.
This file is collected last on purpose: a failure here leaves every other test
already run.
"""
import ctypes

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


def _noalloc(fio, torch, plan, x, out):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return fio.lib().fio_apply_noalloc(plan._handle, ctypes.c_void_p(x.data_ptr()),
                                       ctypes.c_void_p(out.data_ptr()), x.shape[0], stream)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_noalloc_matches_apply_twice(env, prec):
    fio, torch = env
    from paper_math_0610051_gb300 import synth
    N, B = 64, 3
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    tol = 1e-12 if prec == "fp64" else 1e-6
    with fio.Plan(N, fio.PHASE_ELLIPSE, synth.ellipse_params(), 1e-4, precision=prec,
                  max_batch=B) as plan:
        f = torch.from_numpy(synth.white_noise(N, B, seed=1)).to(dt).cuda()
        ref = plan.apply(f)
        for call in range(2):
            # a different input in between, so the second call starts from a
            # scratch array holding another call's values
            g = torch.from_numpy(synth.white_noise(N, B, seed=10 + call, real=False)).to(dt).cuda()
            tmp = torch.empty_like(g)
            assert _noalloc(fio, torch, plan, g, tmp) == fio.FIO_OK
            out = torch.full_like(f, float("nan"))
            assert _noalloc(fio, torch, plan, f, out) == fio.FIO_OK
            torch.cuda.synchronize()
            err = (torch.linalg.vector_norm(out - ref) / torch.linalg.vector_norm(ref)).item()
            assert err <= tol, (call, err)
        plan.sync()


def test_noalloc_on_a_recompute_plan(env):
    """A plan in the recompute storage mode forms gamma^x in its own buffer, so
    the no-allocation entry still allocates nothing and agrees with fio_apply."""
    fio, torch = env
    from paper_math_0610051_gb300 import synth
    N, B = 64, 2
    with fio.Plan(N, fio.PHASE_ELLIPSE, synth.ellipse_params(), 1e-4, max_batch=B,
                  alpha_mode="recompute") as plan:
        f = torch.from_numpy(synth.white_noise(N, B, seed=7, real=False)).to(torch.complex64).cuda()
        ref = plan.apply(f)
        out = torch.full_like(f, float("nan"))
        assert _noalloc(fio, torch, plan, f, out) == fio.FIO_OK
        torch.cuda.synchronize()
        err = (torch.linalg.vector_norm(out - ref) / torch.linalg.vector_norm(ref)).item()
        assert err <= 1e-6, err
        plan.sync()


def test_noalloc_rejects_oversize(env):
    fio, torch = env
    from paper_math_0610051_gb300 import synth
    N = 256
    with fio.Plan(N, fio.PHASE_ELLIPSE, synth.ellipse_params(), 1e-4) as plan:
        need = (plan.info()["grid_points"] + N * N) * 8
        assert need > (32 << 20)
        f = torch.zeros(1, N, N, dtype=torch.complex64, device="cuda")
        out = torch.empty_like(f)
        assert _noalloc(fio, torch, plan, f, out) == fio.FIO_EINVAL
        assert b"FIO_NOALLOC_SCRATCH_BYTES" in fio.lib().fio_last_error()


def test_noalloc_batch_beyond_max_batch_allocates_nothing(env):
    """The entry's batch is bounded by the scratch array, not by the plan's
    max_batch: a plan made for one input applies four in one call, equal to four
    single fio_apply calls.  After a first call, further calls leave the device's
    free memory unchanged."""
    fio, torch = env
    from paper_math_0610051_gb300 import synth
    N, B = 64, 4
    with fio.Plan(N, fio.PHASE_ELLIPSE, synth.ellipse_params(), 1e-4, max_batch=1) as plan:
        f = torch.from_numpy(synth.white_noise(N, B, seed=3, real=False)).to(torch.complex64).cuda()
        ref = torch.stack([plan.apply(f[b:b + 1])[0] for b in range(B)])
        out = torch.empty_like(f)
        assert _noalloc(fio, torch, plan, f, out) == fio.FIO_OK  # set-up call
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(2):
            out.fill_(float("nan"))
            assert _noalloc(fio, torch, plan, f, out) == fio.FIO_OK
            torch.cuda.synchronize()
            assert torch.cuda.mem_get_info()[0] == free0
            err = (torch.linalg.vector_norm(out - ref) / torch.linalg.vector_norm(ref)).item()
            assert err <= 1e-6, err
        plan.sync()
