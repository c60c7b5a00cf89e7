"""Pins of the surrogate's FP64 MLP reference: gradients against central
finite differences, a linear network against the closed-form least-squares
gradient, and one Adam step against its textbook first step (sign(g) * lr)."""
import numpy as np

from oracle import mlp


def _net(seed=0, sizes=(5, 7, 6, 2)):
    p = mlp.init(list(sizes), seed)
    # give every unit a nonzero bias so no relu sits exactly at its kink
    return [(W, np.random.default_rng(seed + 1).normal(0, 0.3, size=b.shape)) for W, b in p]


def test_gradients_match_central_differences():
    rng = np.random.default_rng(3)
    params = _net()
    x = rng.normal(size=(9, 5)); t = rng.normal(size=(9, 2))
    y, cache = mlp.forward(params, x)
    grads = mlp.backward(params, cache, y, t)
    h = 1e-6
    for li, (W, b) in enumerate(params):
        for arr, g in ((W, grads[li][0]), (b, grads[li][1])):
            flat = arr.reshape(-1); gf = g.reshape(-1)
            for idx in range(0, flat.size, max(1, flat.size // 7)):
                old = flat[idx]
                flat[idx] = old + h
                lp = mlp.loss(mlp.forward(params, x)[0], t)
                flat[idx] = old - h
                lm = mlp.loss(mlp.forward(params, x)[0], t)
                flat[idx] = old
                assert abs((lp - lm) / (2 * h) - gf[idx]) < 1e-6 * max(1.0, abs(gf[idx]))


def test_linear_layer_gradient_closed_form():
    rng = np.random.default_rng(5)
    W = rng.normal(size=(2, 4)); b = rng.normal(size=2)
    x = rng.normal(size=(11, 4)); t = rng.normal(size=(11, 2))
    y, cache = mlp.forward([(W, b)], x)
    (gW, gb), = mlp.backward([(W, b)], cache, y, t)
    # L = 1/(2B) ||X W^T + b - T||^2  =>  dL/dW = (X W^T + b - T)^T X / B
    R = x @ W.T + b - t
    assert np.allclose(gW, R.T @ x / 11, rtol=0, atol=1e-13)
    assert np.allclose(gb, R.sum(0) / 11, rtol=0, atol=1e-13)


def test_adam_first_step_is_signed_lr():
    params = _net()
    grads = [(np.full_like(W, 0.5), -np.ones_like(b)) for W, b in params]
    opt = mlp.Adam(params, lr=1e-2)
    new = opt.step(params, grads)
    for (W, b), (W1, b1) in zip(params, new):
        # m_hat = g, v_hat = g^2  ->  step = lr g / (|g| + eps)
        assert np.allclose(W1 - W, -1e-2 * 0.5 / (0.5 + 1e-8), rtol=0, atol=1e-15)
        assert np.allclose(b1 - b, 1e-2 / (1.0 + 1e-8), rtol=0, atol=1e-15)


def test_training_reduces_loss_on_a_learnable_map():
    rng = np.random.default_rng(7)
    x = rng.normal(size=(256, 5))
    t = np.stack([np.sin(x[:, 0]) + x[:, 1] ** 2, x[:, 2] * x[:, 3]], axis=1)
    params = mlp.init([5, 32, 32, 2], 1)
    opt = mlp.Adam(params, lr=3e-3)
    l0 = mlp.loss(mlp.forward(params, x)[0], t)
    for _ in range(300):
        y, cache = mlp.forward(params, x)
        params = opt.step(params, mlp.backward(params, cache, y, t))
    assert mlp.loss(mlp.forward(params, x)[0], t) < 0.1 * l0
