"""Pins of the warm-start MLP oracle: chain-rule gradients vs finite differences, Adam's closed-form first
step, and training that fits a smooth map."""
import numpy as np

import inputs
from oracle import mlp


def test_bf16_round():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, -3.14159, 0.0], dtype=np.float32)
    r = inputs.bf16_round(x)
    assert r[0] == 1.0 and r[2] == 1.0 + 2 ** -7
    assert r[1] in (1.0, 1.0 + 2 ** -7)                  # tie to even -> 1.0
    assert r[1] == 1.0
    assert abs(r[3] + 3.14159) < 2 ** -6 * 4 and r[4] == 0.0
    assert np.all(inputs.bf16_round(r) == r)              # idempotent


def test_gradient_matches_finite_differences():
    n_in, H, n_out = 2, 7, 3
    r = np.random.default_rng(0)
    p = r.standard_normal(H * n_in + H + H * H + H + n_out * H + n_out) * 0.5
    z = r.uniform(-1, 1, (5, n_in))
    t = r.standard_normal((5, n_out))
    _, g = mlp.loss_grad(p, z, t, n_in, H, n_out, round_weights=False)
    eps = 1e-6
    for k in r.choice(p.size, 25, replace=False):
        e = np.zeros_like(p); e[k] = eps
        fd = (mlp.loss_grad(p + e, z, t, n_in, H, n_out, False)[0] - mlp.loss_grad(p - e, z, t, n_in, H, n_out, False)[0]) / (2 * eps)
        assert np.isclose(g[k], fd, rtol=1e-6, atol=1e-9), k


def test_adam_first_step_closed_form():
    """At t = 1 the bias-corrected moments are g and g^2, so every parameter moves by lr * g / (|g| + eps)."""
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    p = np.ones(4)
    p1, m, v = mlp.adam_step(p, g, np.zeros(4), np.zeros(4), 1, 0.01)
    assert np.allclose(p1, 1.0 - 0.01 * g / (np.abs(g) + 1e-8))
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_training_fits_smooth_map():
    n_in, H, n_out = 2, 32, 3
    r = np.random.default_rng(1)
    mu = r.uniform(0.9, 1.1, (256, 2))
    x = np.stack([np.sin(3 * mu[:, 0]), mu[:, 0] * mu[:, 1], np.cos(2 * mu[:, 1])], 1)
    p0 = inputs.mlp_init(n_in, H, n_out)
    order = inputs.mlp_order(256, 60)
    p, losses, norm = mlp.train(p0, mu, x, 60, 32, 3e-3, order, n_in, H, n_out)
    assert losses[-1] < 0.05 * losses[0]
    pred = mlp.predict(p, norm, mu, n_in, H, n_out)
    assert np.sqrt(np.mean((pred - x) ** 2)) < 0.1 * x.std()
