"""Learned warm start: an MLP mu -> xh0 (FP64 reference of the training the library runs on the GPU).

Test infrastructure only (see ``oracle/__init__``).

The paper starts its SQP from RBF interpolants of snapshot latents (Sec. 7.2); the library replaces them by
a small MLP trained on solutions the SQP itself produces.  Model (flat parameter order W1, b1, W2, b2, W3, b3):
    a1 = tanh(W1 z + b1),  a2 = tanh(W2 a1 + b2),  y = W3 a2 + b3,
with input z = (mu - mu_c) / mu_s and output xh0 = out_mean + out_std * y (standardisation fixed from the
training set).  Loss: mean over samples and outputs of (y - t)^2, t = (xh* - out_mean) / out_std.
Gradients by the chain rule written out layer by layer; Adam (Kingma & Ba 2015): beta1 = 0.9,
beta2 = 0.999, eps = 1e-8, bias-corrected moments.  The forward/backward use the weights rounded to
bfloat16, as the GPU does; Adam updates FP32 master weights.
"""
from __future__ import annotations

import numpy as np

BETA1, BETA2, EPS = 0.9, 0.999, 1e-8


def unpack(p, n_in, H, n_out):
    o = 0
    shapes = [(H, n_in), (H,), (H, H), (H,), (n_out, H), (n_out,)]
    out = []
    for s in shapes:
        n = int(np.prod(s))
        out.append(np.asarray(p[o:o + n], dtype=np.float64).reshape(s))
        o += n
    return out


def bf16(a):
    import inputs
    return inputs.bf16_round(a).astype(np.float64)


def forward(p, z, n_in, H, n_out, round_weights=True):
    W1, b1, W2, b2, W3, b3 = unpack(p, n_in, H, n_out)
    if round_weights:
        W1, W2, W3 = bf16(W1), bf16(W2), bf16(W3)
    a1 = np.tanh(z @ W1.T + b1)
    a2 = np.tanh(a1 @ W2.T + b2)
    y = a2 @ W3.T + b3
    return y, (z, a1, a2, W1, W2, W3)


def loss_grad(p, z, t, n_in, H, n_out, round_weights=True):
    """(loss, gradient flat like p) of the mean squared error on one batch."""
    y, (z, a1, a2, W1, W2, W3) = forward(p, z, n_in, H, n_out, round_weights)
    nb = z.shape[0]
    L = float(np.mean((y - t) ** 2))
    dy = 2.0 * (y - t) / (nb * n_out)
    dW3 = dy.T @ a2
    db3 = dy.sum(0)
    dz2 = (dy @ W3) * (1.0 - a2 ** 2)
    dW2 = dz2.T @ a1
    db2 = dz2.sum(0)
    dz1 = (dz2 @ W2) * (1.0 - a1 ** 2)
    dW1 = dz1.T @ z
    db1 = dz1.sum(0)
    return L, np.concatenate([g.ravel() for g in (dW1, db1, dW2, db2, dW3, db3)])


def adam_step(p, g, m, v, t, lr):
    """One Adam update at step t (1-based); returns new (p, m, v)."""
    m = BETA1 * m + (1 - BETA1) * g
    v = BETA2 * v + (1 - BETA2) * g * g
    mh = m / (1 - BETA1 ** t)
    vh = v / (1 - BETA2 ** t)
    return p - lr * mh / (np.sqrt(vh) + EPS), m, v


def standardise(mu, x):
    """(mu_c, mu_s, out_mean, out_std) of a training set."""
    mu_c = 0.5 * (mu.max(0) + mu.min(0))
    mu_s = np.maximum(0.5 * (mu.max(0) - mu.min(0)), 1e-12)
    om = x.mean(0)
    os_ = np.maximum(x.std(0), 1e-8)
    return mu_c, mu_s, om, os_


def train(p0, mu, x, epochs, batch, lr, order, n_in, H, n_out):
    """Mini-batch Adam on the standardised data in the given per-epoch order; returns (p, losses)."""
    mu_c, mu_s, om, os_ = standardise(mu, x)
    z = (mu - mu_c) / mu_s
    t = (x - om) / os_
    p = np.asarray(p0, dtype=np.float64).copy()
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    step = 0
    losses = []
    for e in range(epochs):
        tot = 0.0
        nbat = 0
        for b0 in range(0, len(mu), batch):
            idx = order[e][b0:b0 + batch]
            L, g = loss_grad(p, z[idx], t[idx], n_in, H, n_out)
            step += 1
            p, m, v = adam_step(p, g, m, v, step, lr)
            tot += L
            nbat += 1
        losses.append(tot / nbat)
    return p, losses, (mu_c, mu_s, om, os_)


def predict(p, norm, mu, n_in, H, n_out):
    mu_c, mu_s, om, os_ = norm
    y, _ = forward(p, (mu - mu_c) / mu_s, n_in, H, n_out)
    return om + os_ * y
