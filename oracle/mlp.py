"""FP64 CPU reference of the phase-surrogate MLP (test infrastructure).

The network maps (x1, x2, cos theta, sin theta) through two tanh layers of 64
units to three outputs (tau, d tau/d x1, d tau/d x2); x1 and x2 in [0, 1) enter
the first layer as 2 x - 1.  Parameters are one flat
vector, in this order: W1 [4][64], b1 [64], W2 [64][64], b2 [64], W3 [64][3],
b3 [3] (row-major, input index first).  The loss is the mean over samples of
the squared output error summed over the three outputs.  Gradients are the
chain rule written out; tests pin them with finite differences.
"""
from __future__ import annotations

import numpy as np

SIZES = [(4, 64), (64,), (64, 64), (64,), (64, 3), (3,)]
NPARAMS = sum(int(np.prod(s)) for s in SIZES)


def unpack(params):
    params = np.asarray(params, np.float64)
    out, o = [], 0
    for s in SIZES:
        n = int(np.prod(s))
        out.append(params[o:o + n].reshape(s))
        o += n
    return out


def net_input(X):
    """The first layer's input: (2 x1 - 1, 2 x2 - 1, cos theta, sin theta)."""
    Z = np.array(X, np.float64, copy=True)
    Z[:, :2] = 2.0 * Z[:, :2] - 1.0
    return Z


def forward(params, X):
    W1, b1, W2, b2, W3, b3 = unpack(params)
    h1 = np.tanh(net_input(X) @ W1 + b1)
    h2 = np.tanh(h1 @ W2 + b2)
    return h2 @ W3 + b3, (h1, h2)


def loss(params, X, T):
    y, _ = forward(params, X)
    return float(np.mean(np.sum((y - T) ** 2, axis=1)))


def grad(params, X, T):
    W1, b1, W2, b2, W3, b3 = unpack(params)
    y, (h1, h2) = forward(params, X)
    n = X.shape[0]
    dy = 2.0 * (y - T) / n
    gW3 = h2.T @ dy
    gb3 = dy.sum(0)
    dz2 = (dy @ W3.T) * (1 - h2 ** 2)
    gW2 = h1.T @ dz2
    gb2 = dz2.sum(0)
    dz1 = (dz2 @ W2.T) * (1 - h1 ** 2)
    gW1 = net_input(X).T @ dz1
    gb1 = dz1.sum(0)
    return np.concatenate([g.ravel() for g in (gW1, gb1, gW2, gb2, gW3, gb3)])


def dtheta(params, X):
    """d y0 / d theta with (x3, x4) = (cos theta, sin theta): forward-mode tangent."""
    W1, b1, W2, b2, W3, b3 = unpack(params)
    d = np.zeros_like(X)
    d[:, 2] = -X[:, 3]
    d[:, 3] = X[:, 2]
    h1 = np.tanh(net_input(X) @ W1 + b1)
    dh1 = (1 - h1 ** 2) * (d @ W1)
    h2 = np.tanh(h1 @ W2 + b2)
    dh2 = (1 - h2 ** 2) * (dh1 @ W2)
    return (dh2 @ W3)[:, 0]
