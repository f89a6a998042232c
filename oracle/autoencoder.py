"""Offline training of the sparse-masked shallow autoencoders (Sec. 3.4 "Nonlinear-manifold ROM", Sec. 5.1,
Sec. 7.2-7.3), FP64.

Test infrastructure only (see ``oracle/__init__``).

For one subdomain and one kind of state (interior or interface), with snapshots x_l of that state:

    normalisation   xt = (x - offset) / scale,  offset = (max+min)/2, scale = (max-min)/2 over the
                    training snapshots, so every component lies in [-1, 1] (Sec. 7.3)
    encoder         h(xt)  = We2 sigma(We1 xt + be1)           (Eq. autoencoder_architecture a / c)
    decoder         gt(xh) = Wd2 sigma(Wd1 xh + bd1)           (Eq. autoencoder_architecture b / d)
    de-normalised   g(xh)  = offset + scale o gt(xh)            (the ROM's decoder, Sec. 7.3)
    loss            L = (1/n_b) sum_{l in batch} || xt_l - gt(h(xt_l)) ||_2^2
                                                                (Eq. autoencoder_AbsMSE_loss on the normalised
                                                                 snapshots)

Wd2 (N x w) carries the three-band mask, We1 (w x N) its transpose (Sec. 5.1, Sec. 7.3); Wd1, bd1, be1, We2
are dense.  The parameters are trained by mini-batch Adam (Sec. 7.3).  The mask is held as a dense 0/1
matrix here and every product is a plain dense matrix product with the mask applied to the weights and to
their gradients: slow, and meant to be read against the equations.

Readings (the paper leaves these open or fixes them only for its own runs):
* the loss sums the squared error over the components of a snapshot and averages over the snapshots of a
  batch (Eq. autoencoder_AbsMSE_loss, restricted to the batch); the epoch loss is the mean of its batch losses;
* Adam with beta = (0.9, 0.999), eps = 1e-8 and a constant learning rate; the paper's learning-rate decay on
  plateau and early stopping are left out (a fixed number of epochs);
* the sample order of each epoch is an input (a seeded permutation), and so are the initial weights.
"""
from __future__ import annotations

import numpy as np

from .decoders import activation


def _dense(cols, vals, n_rows, n_cols):
    W = np.zeros((n_rows, n_cols))
    M = np.zeros((n_rows, n_cols))
    cols = np.asarray(cols)
    for r in range(n_rows):
        m = cols[r] >= 0
        W[r, cols[r][m]] = np.asarray(vals)[r][m]
        M[r, cols[r][m]] = 1.0
    return W, M


def normalisation(X):
    """(offset, scale) of Sec. 7.3 over snapshots X (n_snap x N); a constant component gets scale 1."""
    X = np.asarray(X, dtype=np.float64)
    hi, lo = X.max(axis=0), X.min(axis=0)
    scale = 0.5 * (hi - lo)
    return 0.5 * (hi + lo), np.where(scale > 0.0, scale, 1.0)


PARAM_NAMES = ("We1", "be1", "We2", "Wd1", "bd1", "Wd2")


class MaskedAutoencoder:
    """enc: dict of ``inputs.encoder`` (cols/vals on the transposed mask, b1, W2); dec: dict of
    ``inputs.decoder`` (W1, b1, cols/vals of the band mask; its scale/offset are replaced by the
    normalisation of the training snapshots)."""

    def __init__(self, enc: dict, dec: dict, act: str = "swish"):
        self.N, self.w, self.n = dec["N"], dec["w"], dec["n"]
        self.act = act
        self.sigma, self.dsigma = activation(act)
        We1, self.Me1 = _dense(enc["cols"], enc["vals"], self.w, self.N)
        Wd2, self.Md2 = _dense(dec["cols"], dec["vals"], self.N, self.w)
        self.p = {"We1": We1, "be1": np.array(enc["b1"], dtype=np.float64),
                  "We2": np.array(enc["W2"], dtype=np.float64), "Wd1": np.array(dec["W1"], dtype=np.float64),
                  "bd1": np.array(dec["b1"], dtype=np.float64), "Wd2": Wd2}
        self.dec_cols = np.asarray(dec["cols"])
        self.enc_cols = np.asarray(enc["cols"])
        self.offset = np.zeros(self.N)
        self.scale = np.ones(self.N)

    # -- forward and the chain rule --------------------------------------------------------------------
    def forward(self, Xt, p=None):
        """Xt: normalised snapshots, one per column (N x n_b).  Returns the intermediate quantities."""
        p = self.p if p is None else p
        z1 = p["We1"] @ Xt + p["be1"][:, None]
        a1 = self.sigma(z1)
        lat = p["We2"] @ a1                                   # h(xt)
        z2 = p["Wd1"] @ lat + p["bd1"][:, None]
        a2 = self.sigma(z2)
        Y = p["Wd2"] @ a2                                     # gt(h(xt))
        return z1, a1, lat, z2, a2, Y

    def loss_grad(self, Xt, p=None):
        """L of the batch Xt (N x n_b) and dL/dp for every parameter (masked weights: the gradient on the
        mask only)."""
        p = self.p if p is None else p
        nb = Xt.shape[1]
        z1, a1, lat, z2, a2, Y = self.forward(Xt, p)
        E = Y - Xt
        L = float(np.sum(E * E)) / nb
        dY = 2.0 * E / nb                                      # dL/dY
        g = {}
        g["Wd2"] = (dY @ a2.T) * self.Md2
        dz2 = (p["Wd2"].T @ dY) * self.dsigma(z2)
        g["Wd1"] = dz2 @ lat.T
        g["bd1"] = dz2.sum(axis=1)
        dlat = p["Wd1"].T @ dz2
        g["We2"] = dlat @ a1.T
        dz1 = (p["We2"].T @ dlat) * self.dsigma(z1)
        g["We1"] = (dz1 @ Xt.T) * self.Me1
        g["be1"] = dz1.sum(axis=1)
        return L, g

    def loss(self, Xt, p=None):
        Y = self.forward(Xt, p)[-1]
        return float(np.sum((Y - Xt) ** 2)) / Xt.shape[1]

    # -- training -----------------------------------------------------------------------------------------
    def train(self, X, epochs, batch, lr, order, beta1=0.9, beta2=0.999, eps=1e-8):
        """Mini-batch Adam on the snapshots X (n_snap x N, un-normalised); order: epochs x n_snap sample
        order.  Sets the normalisation from X first.  Returns the epoch losses."""
        X = np.asarray(X, dtype=np.float64)
        self.offset, self.scale = normalisation(X)
        Xt = ((X - self.offset) / self.scale).T                # N x n_snap
        m = {k: np.zeros_like(v) for k, v in self.p.items()}
        v = {k: np.zeros_like(v) for k, v in self.p.items()}
        t = 0
        losses = []
        n = X.shape[0]
        for e in range(epochs):
            acc, nbatch = 0.0, 0
            for b0 in range(0, n, batch):
                idx = order[e][b0:b0 + batch]
                L, g = self.loss_grad(Xt[:, idx])
                t += 1
                for k in self.p:
                    m[k] = beta1 * m[k] + (1.0 - beta1) * g[k]
                    v[k] = beta2 * v[k] + (1.0 - beta2) * g[k] ** 2
                    mh = m[k] / (1.0 - beta1 ** t)
                    vh = v[k] / (1.0 - beta2 ** t)
                    self.p[k] = self.p[k] - lr * mh / (np.sqrt(vh) + eps)
                acc += L
                nbatch += 1
            losses.append(acc / nbatch)
        return np.array(losses)

    # -- the trained maps -----------------------------------------------------------------------------------
    def encode(self, X):
        """h applied to un-normalised states X (n x N) -> latent coordinates (n x n_lat)."""
        Xt = ((np.asarray(X, dtype=np.float64) - self.offset) / self.scale).T
        return self.forward(Xt)[2].T

    def decoder_spec(self) -> dict:
        """The trained decoder with its de-normalisation, in the ELL form the ROM loads
        (g = offset + scale o Wd2 sigma(Wd1 xh + bd1))."""
        cols = self.dec_cols
        vals = np.zeros(cols.shape)
        for r in range(self.N):
            m = cols[r] >= 0
            vals[r][m] = self.p["Wd2"][r, cols[r][m]]
        return dict(N=self.N, w=self.w, n=self.n, act=self.act, W1=self.p["Wd1"].copy(), b1=self.p["bd1"].copy(),
                    cols=cols.copy(), vals=vals, offset=self.offset.copy(), scale=self.scale.copy())
