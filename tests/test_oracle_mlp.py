"""Pins for the FP64 MLP reference: a brute-force loop forward on a tiny
input, finite-difference gradients, and Adam's first step (a step of lr
against the sign of the gradient after bias correction)."""
import numpy as np

from oracle import mlp


def test_forward_matches_loops():
    rng = np.random.default_rng(0)
    p = mlp.init(1) + rng.normal(scale=0.05, size=mlp.n_params())
    x = rng.normal(size=(2, 16))
    y, _ = mlp.forward(p, x)
    layers = mlp.unpack(p)
    for r in range(2):
        h = list(x[r])
        for li, (W, b) in enumerate(layers):
            z = []
            for o in range(W.shape[0]):
                acc = b[o]
                for i in range(W.shape[1]):
                    acc += W[o, i] * h[i]
                z.append(acc)
            h = [max(v, 0.0) for v in z] if li < len(layers) - 1 else z
        assert np.allclose(y[r], h, rtol=1e-12, atol=1e-12)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(2)
    p = mlp.init(3) + rng.normal(scale=0.05, size=mlp.n_params())
    x = rng.normal(size=(7, 16))
    t = rng.normal(size=(7, 4))
    _, g = mlp.loss_and_grad(p, x, t)
    idx = rng.choice(mlp.n_params(), 60, replace=False)
    h = 1e-6
    for k in idx:
        e = np.zeros_like(p)
        e[k] = h
        fd = (mlp.loss_and_grad(p + e, x, t)[0] - mlp.loss_and_grad(p - e, x, t)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k])), (k, fd, g[k])


def test_adam_first_step_is_lr_times_sign():
    p = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -1e-3, 0.0])
    m = np.zeros(3)
    v = np.zeros(3)
    p1, m1, v1 = mlp.adam(p, g, m, v, 1, lr=0.01)
    # bias-corrected m/sqrt(v) = g/|g| (up to eps) on the first step
    assert np.allclose(p1[:2], p[:2] - 0.01 * np.sign(g[:2]), rtol=0, atol=1e-7)
    assert p1[2] == p[2]
    assert np.allclose(m1, 0.1 * g) and np.allclose(v1, 0.001 * g * g)
