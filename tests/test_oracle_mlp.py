"""Pins of the numpy reference of the degree selector: the gradient against
central finite differences, softmax and loss identities, Adam's first step."""
import numpy as np

from oracle import mlp


def _data(seed, n=40):
    g = np.random.default_rng(seed)
    X = g.standard_normal((n, mlp.NF)) * 2 + 1
    y = g.integers(0, mlp.NC, n)
    return X, y


def test_gradient_matches_finite_differences():
    X, y = _data(1)
    p = mlp.init(3, X.mean(axis=0), X.std(axis=0))
    _, g = mlp.loss_and_grad(p, X, y)
    rng = np.random.default_rng(2)
    idx = rng.choice(np.arange(2 * mlp.NF, mlp.NPARAM), 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (mlp.loss_and_grad(p + e, X, y)[0] - mlp.loss_and_grad(p - e, X, y)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), i
    assert np.all(g[:2 * mlp.NF] == 0)


def test_uniform_logits_loss_is_log_classes():
    X, y = _data(4)
    d = mlp.unpack(mlp.init(5, X.mean(axis=0), X.std(axis=0)))
    d["W3"][:] = 0
    d["b3"][:] = 0
    loss, _ = mlp.loss_and_grad(mlp.pack(d), X, y)
    assert abs(loss - np.log(mlp.NC)) < 1e-14
    P = mlp.softmax(np.random.default_rng(0).standard_normal((7, mlp.NC)) * 30)
    assert np.allclose(P.sum(axis=1), 1.0)


def test_adam_first_step_is_lr_times_sign():
    p = np.zeros(mlp.NPARAM)
    g = np.random.default_rng(6).standard_normal(mlp.NPARAM)
    p2, m, v = mlp.adam_step(p, g, np.zeros_like(p), np.zeros_like(p), 1, 1e-3)
    exp = -1e-3 * g / (np.abs(g) + 1e-8)
    exp[:2 * mlp.NF] = 0
    assert np.allclose(p2, exp, rtol=1e-9, atol=1e-15)


def test_training_reduces_loss():
    X, y = _data(7, 200)
    y = (X[:, 0] > 1).astype(int) + 2 * (X[:, 1] > 1).astype(int)  # learnable labels
    p = mlp.init(8, X.mean(axis=0), X.std(axis=0))
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    l0 = mlp.loss_and_grad(p, X, y)[0]
    for t in range(1, 301):
        _, g = mlp.loss_and_grad(p, X, y)
        p, m, v = mlp.adam_step(p, g, m, v, t, 1e-2)
    assert mlp.loss_and_grad(p, X, y)[0] < 0.3 * l0
