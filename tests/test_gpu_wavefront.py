"""The Figure 2 experiment of Sec. 4 as headless arrays (WF(L*L f) = WF(f) for
Phi = x.xi + r(x)|xi|).  The property is qualitative, so this checks that the
script writes finite arrays of the right shape and that its band-energy numbers
are well defined; it asserts nothing about the wave front sets."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_wavefront_arrays(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_math_0610051_gb300 import wavefront
    N = 128
    res = wavefront.run(N, str(tmp_path))
    assert set(res) == {"disc", "lines", "rectangle"}
    for name, r in res.items():
        for kind in ("f", "abs_Lf", "abs_LsLf"):
            a = np.load(os.path.join(tmp_path, f"{name}_{kind}.npy"))
            assert a.shape == (N, N) and np.all(np.isfinite(a))
        assert 0 < r["band"] < 1
        assert r["f"] > 0.8  # the input's own high frequencies sit on its jumps
        for k in ("Lf", "LsLf"):
            assert 0 <= r[k] <= 1
