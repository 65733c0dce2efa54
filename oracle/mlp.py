"""CPU oracle of the node scorer: a 12 -> 64 -> 64 -> 2 ReLU perceptron.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain numpy in float64.

Definition (the same one the CUDA kernels implement):
  z1 = W1 x + b1, h1 = relu(z1)      W1: 64 x 12
  z2 = W2 h1 + b2, h2 = relu(z2)     W2: 64 x 64
  y  = W3 h2 + b3                    W3: 2 x 64
  y[r] is the predicted cost of branching a node with rule r (regression).
  Per-sample loss: m0 * (y0 - t0)^2 / 2 + m1 * (y1 - t1)^2 / 2;
  the batch loss is the mean over samples.
The forward and backward passes use the weight matrices rounded to bfloat16
(round to nearest, ties to even); biases stay in float32.  The parameter vector
is [W1, b1, W2, b2, W3, b3], matrices row major (5122 values).
"""
from __future__ import annotations

import numpy as np

NIN, NH, NOUT = 12, 64, 2
SHAPES = [("W1", (NH, NIN)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("W3", (NOUT, NH)), ("b3", (NOUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(theta[o:o + n]).reshape(shp)
        o += n
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def bf16_round(a):
    """float32 -> nearest bfloat16 value (ties to even), returned as float32.

    A bfloat16 keeps the top 16 bits of the float32 pattern; rounding adds half
    of the dropped part's unit (0x7FFF) plus the kept part's lowest bit (so that
    exact halves go to the even neighbour), then truncates."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


def effective(theta, bf16=True):
    """Parameters as the forward pass sees them: float32, matrices in bf16.
    With bf16=False the parameters are used as given, in float64."""
    if not bf16:
        return {k: v.astype(np.float64) for k, v in unpack(np.asarray(theta, dtype=np.float64)).items()}
    p = unpack(np.asarray(theta, dtype=np.float32))
    for name in ("W1", "W2", "W3"):
        p[name] = bf16_round(p[name])
    return {k: v.astype(np.float64) for k, v in p.items()}


def init_params(seed):
    """He-uniform weights, zero biases, float32 (a seeded numpy draw)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shp in SHAPES:
        if name.startswith("W"):
            fan_in = shp[1]
            lim = np.sqrt(6.0 / fan_in)
            p[name] = rng.uniform(-lim, lim, size=shp)
        else:
            p[name] = np.zeros(shp)
    return pack(p).astype(np.float32)


def forward(theta, X, bf16=True):
    p = effective(theta, bf16)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ p["W3"].T + p["b3"]
    return y, (X, z1, h1, z2, h2)


def loss(theta, X, T, M, bf16=True):
    y, _ = forward(theta, X, bf16)
    T = np.asarray(T, dtype=np.float64)
    M = np.asarray(M, dtype=np.float64)
    per = M[:, 0] * 0.5 * (y[:, 0] - T[:, 0]) ** 2 + M[:, 1] * 0.5 * (y[:, 1] - T[:, 1]) ** 2
    return per.mean()


def grad(theta, X, T, M, bf16=True):
    """Mean loss and its gradient w.r.t. the parameter vector (the weights
    as used, i.e. the bf16-rounded ones), by backpropagation."""
    p = effective(theta, bf16)
    y, (X, z1, h1, z2, h2) = forward(theta, X, bf16)
    n = X.shape[0]
    T = np.asarray(T, dtype=np.float64)
    M = np.asarray(M, dtype=np.float64)
    dy = np.empty_like(y)
    dy[:, 0] = M[:, 0] * (y[:, 0] - T[:, 0])
    dy[:, 1] = M[:, 1] * (y[:, 1] - T[:, 1])
    dy /= n
    g = {}
    g["W3"] = dy.T @ h2
    g["b3"] = dy.sum(0)
    dh2 = dy @ p["W3"]
    dz2 = dh2 * (z2 > 0)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(0)
    dh1 = dz2 @ p["W2"]
    dz1 = dh1 * (z1 > 0)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(0)
    per = M[:, 0] * 0.5 * (y[:, 0] - T[:, 0]) ** 2 + M[:, 1] * 0.5 * (y[:, 1] - T[:, 1]) ** 2
    return per.mean(), pack(g)


def adam_step(theta, m, v, g, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, Algorithm 1) in float64; t counts from 1."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
