"""Pins of the FP64 MLP oracle: an explicit per-sample forward pass, central finite differences, Adam's first step."""
import numpy as np

from oracle import mlp


def _explicit_forward(theta, x):
    # one sample, written with plain loops from the layer definitions
    p = mlp.unpack(theta)
    h = list(x)
    for W, b, relu in ((p["W1"], p["b1"], True), (p["W2"], p["b2"], True), (p["W3"], p["b3"], False)):
        out = []
        for i in range(W.shape[0]):
            s = b[i]
            for j in range(W.shape[1]):
                s += W[i, j] * h[j]
            out.append(max(s, 0.0) if relu else s)
        h = out
    return np.array(h)


def test_parameter_count():
    assert mlp.NPARAM == 16 * 64 + 64 + 64 * 64 + 64 + 64 * 4 + 4 == 5508


def test_forward_matches_explicit_loops():
    rng = np.random.default_rng(0)
    theta = mlp.init(1)
    theta[1024:1088] = rng.uniform(-0.1, 0.1, 64)   # non-zero biases so every term matters
    theta[-4:] = rng.uniform(-1, 1, 4)
    X = rng.standard_normal((5, 16))
    out, _ = mlp.forward(theta, X)
    for i in range(5):
        assert np.allclose(out[i], _explicit_forward(theta, X[i]), rtol=1e-12, atol=1e-12)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(2)
    theta = mlp.init(3) + rng.uniform(-0.01, 0.01, mlp.NPARAM)
    X = rng.standard_normal((7, 16))
    T = rng.standard_normal((7, 4))
    L, g = mlp.grad(theta, X, T)
    assert abs(L - mlp.loss(theta, X, T)) <= 1e-15 * abs(L)
    h = 1e-6
    idx = rng.choice(mlp.NPARAM, 300, replace=False)
    idx = np.r_[idx, np.arange(mlp.NPARAM - 4, mlp.NPARAM), 1024, 5248]   # include biases of every layer
    for i in idx:
        e = np.zeros(mlp.NPARAM); e[i] = h
        fd = (mlp.loss(theta + e, X, T) - mlp.loss(theta - e, X, T)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(g[i])) + 1e-9, (i, fd, g[i])


def test_adam_first_step_is_signed_lr():
    # at t = 1 the bias-corrected moments are g and g^2, so each parameter moves by lr*g/(|g|+eps)
    rng = np.random.default_rng(4)
    theta = rng.standard_normal(mlp.NPARAM)
    g = rng.standard_normal(mlp.NPARAM)
    t1, m, v = mlp.adam_step(theta, np.zeros_like(theta), np.zeros_like(theta), g, 1, lr=1e-3)
    assert np.allclose(theta - t1, 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-10, atol=0)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_adam_decreases_loss():
    rng = np.random.default_rng(5)
    X = rng.standard_normal((64, 16))
    T = np.tanh(X[:, :4] + 0.5 * X[:, 4:8])
    theta = mlp.init(6)
    m = np.zeros_like(theta); v = np.zeros_like(theta)
    L0 = mlp.loss(theta, X, T)
    for t in range(1, 201):
        _, g = mlp.grad(theta, X, T)
        theta, m, v = mlp.adam_step(theta, m, v, g, t, lr=3e-3)
    assert mlp.loss(theta, X, T) < 0.2 * L0
