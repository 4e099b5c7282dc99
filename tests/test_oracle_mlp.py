"""Pins of the CPU references used to check the phase surrogate: the FP64 MLP's
gradients and angular derivative against finite differences, and the tau-mode
derivatives against finite differences and against the oracle's phase."""
import numpy as np

from oracle import mlp
from paper_math_0610051_gb300 import synth


def _params(seed):
    return np.random.default_rng(seed).standard_normal(mlp.NPARAMS) * 0.3


def _inputs(n, seed):
    g = np.random.default_rng(seed)
    th = g.uniform(0, 2 * np.pi, n)
    return np.stack([g.uniform(0, 1, n), g.uniform(0, 1, n), np.cos(th), np.sin(th)], 1), th


def test_mlp_zero_weights_give_bias():
    p = np.zeros(mlp.NPARAMS)
    p[-3:] = [0.5, -1.0, 2.0]
    X, _ = _inputs(5, 0)
    y, _ = mlp.forward(p, X)
    assert np.allclose(y, [[0.5, -1.0, 2.0]] * 5)


def test_mlp_gradient_matches_central_differences():
    p = _params(1)
    X, _ = _inputs(40, 2)
    T = np.random.default_rng(3).standard_normal((40, 3))
    g = mlp.grad(p, X, T)
    rng = np.random.default_rng(4)
    idx = rng.choice(mlp.NPARAMS, 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros(mlp.NPARAMS)
        e[i] = h
        fd = (mlp.loss(p + e, X, T) - mlp.loss(p - e, X, T)) / (2 * h)
        assert abs(fd - g[i]) < 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_mlp_dtheta_matches_finite_difference():
    p = _params(5)
    _, th = _inputs(30, 6)
    x = np.random.default_rng(7).uniform(0, 1, (30, 2))

    def y0(t):
        X = np.stack([x[:, 0], x[:, 1], np.cos(t), np.sin(t)], 1)
        return mlp.forward(p, X)[0][:, 0]

    h = 1e-6
    X = np.stack([x[:, 0], x[:, 1], np.cos(th), np.sin(th)], 1)
    fd = (y0(th + h) - y0(th - h)) / (2 * h)
    assert np.max(np.abs(fd - mlp.dtheta(p, X))) < 1e-7


def test_tau_derivatives_match_finite_differences(orc):
    modes = synth.tau_mode_params(16, seed=3)
    g = np.random.default_rng(8)
    x1, x2, th = g.uniform(0, 1, 50), g.uniform(0, 1, 50), g.uniform(0, 2 * np.pi, 50)
    t = orc.tau_eval(modes, x1, x2, th)
    h = 1e-6
    for col, (dx1, dx2, dth) in zip((1, 2, 3), ((h, 0, 0), (0, h, 0), (0, 0, h))):
        fd = (orc.tau_eval(modes, x1 + dx1, x2 + dx2, th + dth)[:, 0] -
              orc.tau_eval(modes, x1 - dx1, x2 - dx2, th - dth)[:, 0]) / (2 * h)
        assert np.max(np.abs(fd - t[:, col])) < 1e-7


def test_tau_matches_phase(orc):
    """Phi(x, xi) - x.xi = |xi| tau(x, arg xi) for the tau-mode phase."""
    modes = synth.tau_mode_params(12, seed=4)
    g = np.random.default_rng(9)
    n = 80
    x1, x2 = g.uniform(0, 1, n), g.uniform(0, 1, n)
    k1, k2 = g.integers(-40, 41, n), g.integers(-40, 41, n)
    k1[k1 == 0] = 1
    phi = orc.phase_eval(orc.Phase(orc.TAU_MODES, modes), x1, x2, k1, k2)
    tau = orc.tau_eval(modes, x1, x2, np.arctan2(k2, k1))[:, 0]
    assert np.max(np.abs(phi - (x1 * k1 + x2 * k2) - np.hypot(k1, k2) * tau)) < 1e-11


def test_mlp_forward_hand_value():
    """A worked value of the 4 -> 64 -> 64 -> 3 tanh network with one non-zero weight per
    layer, reached at points where tanh(z) differs from z (a dropped activation, a
    missing input map 2x - 1 or a transposed weight index fails it).
    Input x = (0.75, 0.25, cos t, sin t) -> first-layer input (0.5, -0.5, cos t, sin t).
      h1[5]  = tanh(1.5 * 0.5 + 0.2)           (W1[0][5] = 1.5, b1[5] = 0.2)
      h2[7]  = tanh(-2.0 * h1[5] + 0.1)        (W2[5][7] = -2.0, b2[7] = 0.1)
      y      = (0.3, 0.7 h2[7] - 0.4, 0)       (W3[7][1] = 0.7, b3 = (0.3, -0.4, 0))
    Every other unit is tanh(0) = 0 and adds nothing."""
    W1, b1, W2, b2, W3, b3 = [np.zeros(s) for s in mlp.SIZES]
    W1[0, 5], b1[5] = 1.5, 0.2
    W2[5, 7], b2[7] = -2.0, 0.1
    W3[7, 1] = 0.7
    b3[:] = [0.3, -0.4, 0.0]
    p = np.concatenate([a.ravel() for a in (W1, b1, W2, b2, W3, b3)])
    X = np.array([[0.75, 0.25, np.cos(0.3), np.sin(0.3)]])
    h1 = np.tanh(1.5 * 0.5 + 0.2)
    h2 = np.tanh(-2.0 * h1 + 0.1)
    y, _ = mlp.forward(p, X)
    assert np.allclose(y[0], [0.3, 0.7 * h2 - 0.4, 0.0], rtol=0, atol=1e-15)
    # the numbers themselves (tanh 0.95 = 0.739783..., tanh(-1.379566) = -0.880854...)
    assert abs(y[0, 1] - (0.7 * -0.88085407 - 0.4)) < 1e-7
    # d y / d theta: the angular inputs carry no weight here, so it vanishes
    assert abs(mlp.dtheta(p, X)[0]) < 1e-15


def test_mlp_dtheta_hand_value():
    """An angular weight: W1[3][0] = 1 (sin t -> unit 0), W2[0][0] = 1, W3[0][0] = 1:
    y0 = tanh(tanh(sin t)), so d y0 / d t = (1 - y0^2)(1 - tanh(sin t)^2) cos t."""
    W1, b1, W2, b2, W3, b3 = [np.zeros(s) for s in mlp.SIZES]
    W1[3, 0] = W2[0, 0] = W3[0, 0] = 1.0
    p = np.concatenate([a.ravel() for a in (W1, b1, W2, b2, W3, b3)])
    t = 1.1
    X = np.array([[0.1, 0.9, np.cos(t), np.sin(t)]])
    u = np.tanh(np.sin(t))
    y0 = np.tanh(u)
    assert abs(mlp.forward(p, X)[0][0, 0] - y0) < 1e-15
    assert abs(mlp.dtheta(p, X)[0] - (1 - y0 ** 2) * (1 - u ** 2) * np.cos(t)) < 1e-15
