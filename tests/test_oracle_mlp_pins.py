"""Pins for the node-scorer oracle (oracle/mlp.py): backpropagation against
central finite differences, bfloat16 rounding against torch's conversion, and
closed-form special cases."""
import numpy as np
import pytest

from oracle import mlp


def _data(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, mlp.NIN))
    T = np.stack([rng.normal(size=n), (rng.uniform(size=n) < 0.5).astype(float)], 1)
    M = (rng.uniform(size=(n, 2)) < 0.8).astype(float)
    return X, T, M


def test_gradient_matches_finite_differences():
    theta = mlp.init_params(3).astype(np.float64)
    X, T, M = _data(17, 1)
    _, g = mlp.grad(theta, X, T, M, bf16=False)
    rng = np.random.default_rng(0)
    idx = np.concatenate([rng.choice(mlp.NPARAM, 60, replace=False), np.arange(mlp.NPARAM - 2, mlp.NPARAM)])
    h = 1e-6
    for i in idx:
        e = np.zeros(mlp.NPARAM); e[i] = h
        fd = (mlp.loss(theta + e, X, T, M, bf16=False) - mlp.loss(theta - e, X, T, M, bf16=False)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    a = np.concatenate([rng.normal(size=5000) * 10.0 ** rng.integers(-6, 6, size=5000),
                        np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -1 - 2 ** -8, 0.0, -0.0])]).astype(np.float32)
    ref = torch.from_numpy(a).to(torch.bfloat16).to(torch.float32).numpy()
    got = mlp.bf16_round(a)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))
    # ties to even: 1 + 2^-8 is halfway between 1 and 1 + 2^-7 -> 1; 1 + 3*2^-8 -> 1 + 2^-6
    assert mlp.bf16_round(np.float32(1 + 2 ** -8)) == 1.0
    assert mlp.bf16_round(np.float32(1 + 3 * 2 ** -8)) == np.float32(1 + 2 ** -6)


def test_special_cases():
    theta = np.zeros(mlp.NPARAM, np.float32)
    p = mlp.unpack(theta.copy())
    theta = mlp.pack({**p, "b3": np.array([0.25, -1.5])}).astype(np.float32)
    X, T, M = _data(5, 2)
    y, _ = mlp.forward(theta, X)
    assert np.all(y[:, 0] == 0.25) and np.all(y[:, 1] == -1.5)
    # loss with zero outputs: t^2 / 2 for each head; with outputs equal to the
    # targets (biases set to constant targets): zero
    z = np.zeros(mlp.NPARAM, np.float32)
    L = mlp.loss(z, X, T, np.ones_like(M))
    assert L == pytest.approx(np.mean(0.5 * T[:, 0] ** 2 + 0.5 * T[:, 1] ** 2), rel=1e-14)
    Tc = np.tile(np.array([[0.25, -1.5]]), (5, 1))
    assert mlp.loss(theta, X, Tc, np.ones_like(M)) == 0.0
    # a masked head contributes nothing
    assert mlp.loss(z, X, T, np.stack([np.ones(5), np.zeros(5)], 1)) == pytest.approx(np.mean(0.5 * T[:, 0] ** 2))
    # the first Adam step moves every parameter with a non-zero gradient by about lr against it
    g = np.array([3.0, -0.5, 0.0])
    th, m, v = mlp.adam_step(np.zeros(3), np.zeros(3), np.zeros(3), g, 1, lr=0.01)
    assert th[0] == pytest.approx(-0.01, rel=1e-6) and th[1] == pytest.approx(0.01, rel=1e-6) and th[2] == 0.0


def test_init_is_seeded_and_he_scaled():
    a, b = mlp.init_params(7), mlp.init_params(7)
    assert np.array_equal(a, b) and a.dtype == np.float32 and a.size == mlp.NPARAM == 5122
    W1 = mlp.unpack(a)["W1"]
    assert np.abs(W1).max() <= np.sqrt(6.0 / 12) + 1e-6


def test_forward_one_path_closed_form():
    """A single active path through the network (bf16-exact weights): input
    e_0 -> hidden unit 5 of layer 1 (weight 1) -> unit 7 of layer 2 (weight
    2) -> output 1 (weight 3) gives y = (0, 6); the weight W[i, j] maps unit j
    of the layer below to unit i (z = W h + b)."""
    p = mlp.unpack(np.zeros(mlp.NPARAM, np.float32).copy())
    p["W1"][5, 0] = 1.0
    p["W2"][7, 5] = 2.0
    p["W3"][1, 7] = 3.0
    theta = mlp.pack(p).astype(np.float32)
    x = np.zeros((2, mlp.NIN)); x[0, 0] = 1.0; x[1, 0] = -1.0
    y, _ = mlp.forward(theta, x)
    assert y.tolist() == [[0.0, 6.0], [0.0, 0.0]]   # the negative input is cut by the first ReLU


def test_adam_bias_correction_over_steps():
    """Adam with a constant gradient g: the bias-corrected moments are exactly
    g and g^2 at every step, so each step moves lr * g / (|g| + eps)."""
    g = np.array([2.0, -0.25])
    th, m, v = np.zeros(2), np.zeros(2), np.zeros(2)
    for t in range(1, 4):
        th, m, v = mlp.adam_step(th, m, v, g, t, lr=0.01)
    assert th == pytest.approx(-3 * 0.01 * g / (np.abs(g) + 1e-8), rel=1e-12)
