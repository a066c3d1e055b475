"""Pins of the terminator network oracle: the analytic gradient equals central
finite differences of the loss (h = 1e-6), and one Adam step matches the
update written out for a scalar."""
import numpy as np

from oracle import mlp


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    p = mlp.init_params(1) + 0.05 * rng.standard_normal(mlp.n_params())
    x = rng.standard_normal((7, mlp.N_IN))
    t = rng.standard_normal((7, mlp.N_OUT))
    L, g = mlp.loss_and_grad(p, x, t)
    idx = rng.choice(p.size, size=60, replace=False)
    # include every parameter block
    sizes = np.cumsum([128 * 5, 128, 128 * 128, 128, 2 * 128, 2])
    idx = np.unique(np.concatenate([idx, sizes - 1, [0]]))
    h = 1e-6
    for k in idx:
        e = np.zeros_like(p)
        e[k] = h
        fd = (mlp.loss_and_grad(p + e, x, t)[0] - mlp.loss_and_grad(p - e, x, t)[0]) / (2 * h)
        assert abs(fd - g[k]) < 1e-7 * max(1.0, abs(g[k])), (k, fd, g[k])
    assert L > 0


def test_forward_agrees_with_loss():
    rng = np.random.default_rng(4)
    p = mlp.init_params(2)
    x = rng.standard_normal((5, mlp.N_IN))
    y = mlp.forward(p, x)
    L, _ = mlp.loss_and_grad(p, x, y)
    assert L == 0.0


def test_adam_scalar_update():
    p = np.array([1.0]); g = np.array([0.5]); m = np.zeros(1); v = np.zeros(1)
    p1, m1, v1 = mlp.adam_step(p, g, m, v, step=1, lr=0.1)
    # first step: m^ = g, v^ = g^2  =>  p - lr * g / (|g| + eps)
    assert abs(p1[0] - (1.0 - 0.1 * 0.5 / (0.5 + 1e-8))) < 1e-15
    assert abs(m1[0] - 0.05) < 1e-15 and abs(v1[0] - 0.00025) < 1e-15
