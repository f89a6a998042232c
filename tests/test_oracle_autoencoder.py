"""Pins of the oracle's autoencoder training (Sec. 5.1, 7.2-7.3) against what the mathematics fixes:
finite-difference gradients of every parameter block, Adam's closed-form first step, the masks surviving
training, a linear autoencoder reaching the POD (Eckart-Young) bound, and decoders trained on FOM
snapshots giving a ROM whose SQP converges under the paper's stopping rule."""
import numpy as np
import pytest

import inputs
from oracle import setup
from oracle.autoencoder import PARAM_NAMES, MaskedAutoencoder, normalisation
from oracle.rom import relative_error


def tiny_ae(N=12, w=10, n=2, band=2, act="swish", key=(7, 0, 0)):
    dec = inputs.decoder(N, w, n, band, key, act=act)
    enc = inputs.encoder(N, w, n, inputs.transposed_mask(dec["cols"], w), key)
    return MaskedAutoencoder(enc, dec, act)


def test_transposed_mask_is_the_transpose():
    cols = inputs.band_mask(37, 16, 3)
    ct = inputs.transposed_mask(cols, 16)
    fwd = {(r, int(c)) for r in range(cols.shape[0]) for c in cols[r] if c >= 0}
    bwd = {(int(r), j) for j in range(16) for r in ct[j] if r >= 0}
    assert fwd == bwd
    for j in range(16):                                   # ascending, padding at the end
        v = ct[j][ct[j] >= 0]
        assert np.all(np.diff(v) > 0) and np.all(ct[j][len(v):] == -1)


@pytest.mark.parametrize("act", ["swish", "sigmoid"])
def test_gradient_matches_finite_differences(act):
    ae = tiny_ae(act=act)
    r = np.random.default_rng(1)
    Xt = r.uniform(-1, 1, (ae.N, 5))
    L, g = ae.loss_grad(Xt)
    h = 1e-6
    for k in PARAM_NAMES:
        P = ae.p[k]
        fd = np.zeros_like(P)
        mask = ae.Me1 if k == "We1" else ae.Md2 if k == "Wd2" else np.ones_like(P)
        for idx in np.ndindex(P.shape):
            if mask[idx] == 0:
                continue
            q = {kk: vv.copy() for kk, vv in ae.p.items()}
            q[k][idx] += h
            Lp = ae.loss(Xt, q)
            q[k][idx] -= 2 * h
            Lm = ae.loss(Xt, q)
            fd[idx] = (Lp - Lm) / (2 * h)
        np.testing.assert_allclose(g[k], fd, rtol=1e-5, atol=1e-7 * max(1.0, np.abs(fd).max()), err_msg=k)
        assert np.all(g[k][mask == 0] == 0.0)


def test_adam_first_step_closed_form():
    """After one step from zero moments, m_hat = g and v_hat = g^2: every parameter moves by
    -lr g / (|g| + eps)."""
    ae = tiny_ae()
    r = np.random.default_rng(2)
    X = r.uniform(0.2, 0.9, (6, ae.N))
    off, sc = normalisation(X)
    Xt = ((X - off) / sc).T
    p0 = {k: v.copy() for k, v in ae.p.items()}
    _, g = ae.loss_grad(Xt)
    lr = 1e-2
    ae.train(X, 1, 6, lr, np.arange(6)[None, :])
    for k in PARAM_NAMES:
        np.testing.assert_allclose(ae.p[k], p0[k] - lr * g[k] / (np.abs(g[k]) + 1e-8), rtol=1e-12, atol=1e-15)


def test_normalisation_maps_onto_unit_interval():
    X = np.random.default_rng(3).normal(size=(9, 7))
    off, sc = normalisation(X)
    Xt = (X - off) / sc
    assert np.allclose(Xt.max(axis=0), 1.0) and np.allclose(Xt.min(axis=0), -1.0)


def test_masks_survive_training():
    ae = tiny_ae()
    X = np.random.default_rng(4).uniform(0, 1, (16, ae.N))
    ae.train(X, 5, 4, 1e-2, inputs.ae_order(16, 5))
    assert np.all(ae.p["We1"][ae.Me1 == 0] == 0.0) and np.all(ae.p["Wd2"][ae.Md2 == 0] == 0.0)


def test_linear_autoencoder_reaches_the_pod_bound():
    """Identity activation and full masks make the autoencoder an affine map of rank <= n: its loss cannot go
    below the energy the best rank-n affine fit leaves, sum_{j > n} s_j^2 / n_snap of the centred snapshots
    (Eckart-Young; Sec. 3.3: POD minimises the same reconstruction error), and training reaches it."""
    N, w, n, ns = 8, 8, 2, 20
    full = np.tile(np.arange(w, dtype=np.int32), (N, 1))
    r = np.random.default_rng(5)
    dec = dict(N=N, w=w, n=n, W1=r.normal(size=(w, n)) / np.sqrt(n), b1=np.zeros(w), cols=full,
               vals=r.normal(size=(N, w)) / np.sqrt(w))
    enc = dict(cols=full.copy(), vals=r.normal(size=(w, N)) / np.sqrt(N), b1=np.zeros(w),
               W2=r.normal(size=(n, w)) / np.sqrt(w))
    ae = MaskedAutoencoder(enc, dec, "identity")
    # snapshots near a 2D affine subspace, plus small noise in the other directions
    basis = np.linalg.qr(r.normal(size=(N, N)))[0]
    coef = np.hstack([r.normal(size=(ns, n)) * [3.0, 2.0], 0.05 * r.normal(size=(ns, N - n))])
    X = 0.5 + 0.1 * coef @ basis.T
    off, sc = normalisation(X)
    Xt = (X - off) / sc
    s = np.linalg.svd(Xt - Xt.mean(axis=0), compute_uv=False)
    bound = np.sum(s[n:] ** 2) / ns
    ae.train(X, 3000, ns, 1e-2, np.tile(np.arange(ns), (3000, 1)))
    L = ae.loss(Xt.T)
    assert L >= bound * (1 - 1e-9)
    assert L <= 1.02 * bound


def test_trained_decoders_make_the_sqp_converge():
    """Decoders trained on FOM snapshots (12 x 12 grid of mu, Sec. 7.2) instead of random-init ones: the DD
    NM-ROM-HR SQP from xh0 = 0 meets the paper's stopping rule (||F|| < 1e-4 within 15 iterations, Sec. 7.1)
    at held-out mu, with a relative error against the FOM (Eq. relative_error) of the order the paper reports
    for its trained NM-ROM with HR (1e-3 .. 1e-2)."""
    wl = inputs.workload("c1")
    fom, dd, rom, raw = setup.build_trained(wl, n_side=12, epochs=300, batch=16, lr=3e-3)
    for ae in raw["autoencoders"]:
        assert ae.losses[-1] < 0.05 * ae.losses[0]
    for m in inputs.mu_batch(3, seed=99):
        res = rom.solve(m)
        assert res.status == 0 and res.iters < 15
        xf, _ = fom.newton(m, x0=fom.exact_state(m))
        err = relative_error([(xf[sd.interior], xf[sd.interface]) for sd in dd.subs], rom.states(res.x))
        assert err < 3e-2
