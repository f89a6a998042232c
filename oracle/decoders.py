"""Decoders (Sec. 3.3, 3.4, 5.1, 5.4), FP64.

Test infrastructure only (see ``oracle/__init__``).

* ``MaskedDecoder``: g(x) = offset + scale o (W2 sigma(W1 x + b1))   (Eq. autoencoder_architecture
  (b)/(d), followed by the de-normalisation layer of Sec. 7.3); W2 is the sparse masked output
  layer, held here as a dense N x w matrix with explicit zeros.
  Jacobian dg/dx = diag(scale) W2 diag(sigma'(W1 x + b1)) W1.
* ``subnet``: the HR subnet of Sec. 5.4 (Eq. subnet) for an output index set I_o.
* ``LinearDecoder``: the LS-ROM map g(x) = Phi x + x_ref with constant Jacobian Phi (Sec. 3.3).
* ``pod_basis``: thin SVD + energy criterion, Eq. (energy_criterion).
"""
from __future__ import annotations

import numpy as np


def activation(name: str):
    """(sigma, sigma') for swish z/(1+e^-z) (Sec. 7.5), sigmoid, identity."""
    if name == "swish":
        def f(z):
            return z / (1.0 + np.exp(-z))

        def df(z):
            s = 1.0 / (1.0 + np.exp(-z))
            return s + z * s * (1.0 - s)
        return f, df
    if name == "sigmoid":
        def f(z):
            return 1.0 / (1.0 + np.exp(-z))

        def df(z):
            s = 1.0 / (1.0 + np.exp(-z))
            return s * (1.0 - s)
        return f, df
    if name == "identity":
        return (lambda z: z), (lambda z: np.ones_like(z))
    raise KeyError(name)


class MaskedDecoder:
    def __init__(self, spec: dict):
        self.N, self.w, self.n = spec["N"], spec["w"], spec["n"]
        self.W1 = np.asarray(spec["W1"], dtype=np.float64)
        self.b1 = np.asarray(spec["b1"], dtype=np.float64)
        W2 = np.zeros((self.N, self.w))
        cols, vals = np.asarray(spec["cols"]), np.asarray(spec["vals"])
        for r in range(self.N):
            m = cols[r] >= 0
            W2[r, cols[r][m]] = vals[r][m]
        self.W2 = W2
        self.scale = np.asarray(spec["scale"], dtype=np.float64)
        self.offset = np.asarray(spec["offset"], dtype=np.float64)
        self.act_name = spec.get("act", "swish")
        self.sigma, self.dsigma = activation(self.act_name)

    def value(self, x):
        z = self.W1 @ x + self.b1
        return self.offset + self.scale * (self.W2 @ self.sigma(z))

    def jacobian(self, x):
        z = self.W1 @ x + self.b1
        return (self.scale[:, None] * self.W2) @ (self.dsigma(z)[:, None] * self.W1)

    def value_jacobian(self, x):
        return self.value(x), self.jacobian(x)

    def value_jacobian_rows(self, x, rows):
        """Values and Jacobian rows at the outputs `rows` only."""
        z = self.W1 @ x + self.b1
        W2 = self.W2[rows]
        g = self.offset[rows] + self.scale[rows] * (W2 @ self.sigma(z))
        J = (self.scale[rows][:, None] * W2) @ (self.dsigma(z)[:, None] * self.W1)
        return g, J


class EllDecoder:
    """The same decoder g(x) = offset + scale o (W2 sigma(W1 x + b1)) (Sec. 5.1, Eq.
    autoencoder_architecture b/d) with W2 kept in its ELL form (mask columns and values per output row),
    for decoders whose dense W2 does not fit in memory.  Row r: g_r = offset_r + scale_r sum_k val_rk
    sigma(z_{c_rk}), dg_r/dx = scale_r sum_k val_rk sigma'(z_{c_rk}) W1[c_rk, :]."""

    def __init__(self, spec: dict):
        self.N, self.w, self.n = spec["N"], spec["w"], spec["n"]
        self.W1 = np.asarray(spec["W1"], dtype=np.float64)
        self.b1 = np.asarray(spec["b1"], dtype=np.float64)
        cols = np.asarray(spec["cols"], dtype=np.int64)
        self.valid = cols >= 0
        self.cols = np.where(self.valid, cols, 0)
        self.vals = np.where(self.valid, np.asarray(spec["vals"], dtype=np.float64), 0.0)
        self.scale = np.asarray(spec["scale"], dtype=np.float64)
        self.offset = np.asarray(spec["offset"], dtype=np.float64)
        self.act_name = spec.get("act", "swish")
        self.sigma, self.dsigma = activation(self.act_name)

    def value_jacobian_rows(self, x, rows):
        z = self.W1 @ x + self.b1
        c, v = self.cols[rows], self.vals[rows]
        g = self.offset[rows] + self.scale[rows] * (v * self.sigma(z)[c]).sum(axis=1)
        P = self.dsigma(z)[:, None] * self.W1                   # w x n: sigma'(z_c) W1[c, :]
        J = self.scale[rows][:, None] * np.einsum("rk,rkn->rn", v, P[c])
        return g, J

    def value(self, x):
        z = self.W1 @ x + self.b1
        return self.offset + self.scale * (self.vals * self.sigma(z)[self.cols]).sum(axis=1)

    def value_jacobian(self, x):
        return self.value_jacobian_rows(x, np.arange(self.N))


class Subnet:
    """g~(x) = W2~ sigma(W1~ x + b1~) over the hidden set I_h (Eq. subnet), de-normalised on I_o."""

    def __init__(self, dec: MaskedDecoder, I_o):
        I_o = np.sort(np.asarray(I_o, dtype=np.int64))
        I_h = np.flatnonzero((dec.W2[I_o] != 0.0).any(axis=0))     # ascending
        self.I_o, self.I_h = I_o, I_h
        self.W2 = dec.W2[np.ix_(I_o, I_h)]
        self.W1 = dec.W1[I_h]
        self.b1 = dec.b1[I_h]
        self.scale, self.offset = dec.scale[I_o], dec.offset[I_o]
        self.sigma, self.dsigma = dec.sigma, dec.dsigma

    def value(self, x):
        return self.offset + self.scale * (self.W2 @ self.sigma(self.W1 @ x + self.b1))

    def jacobian(self, x):
        z = self.W1 @ x + self.b1
        return (self.scale[:, None] * self.W2) @ (self.dsigma(z)[:, None] * self.W1)


def subnet(dec: MaskedDecoder, I_o) -> Subnet:
    return Subnet(dec, I_o)


class LinearDecoder:
    """LS-ROM map g(x) = Phi x + x_ref (Sec. 3.3); x_ref = 0 in the paper."""

    def __init__(self, Phi, x_ref=None):
        self.Phi = np.asarray(Phi, dtype=np.float64)
        self.N, self.n = self.Phi.shape
        self.x_ref = np.zeros(self.N) if x_ref is None else np.asarray(x_ref, dtype=np.float64)

    def value(self, x):
        return self.Phi @ x + self.x_ref

    def jacobian(self, x):
        return self.Phi

    def value_jacobian(self, x):
        return self.value(x), self.Phi

    def value_jacobian_rows(self, x, rows):
        return self.Phi[rows] @ x + self.x_ref[rows], self.Phi[rows]


class IdentityDecoder(LinearDecoder):
    """g(x) = x: turns the ROM machinery back into the DD FOM (Sec. 4.1)."""

    def __init__(self, N):
        super().__init__(np.eye(N))


def pod_basis(X, nu_tol: float):
    """POD basis of the snapshot matrix X (N x n_mu): thin SVD, smallest n with
    sum_{j<=n} s_j^2 >= (1 - nu_tol) sum_j s_j^2  (Eq. energy_criterion).  Returns (Phi, s)."""
    U, s, _ = np.linalg.svd(X, full_matrices=False)
    e = np.cumsum(s ** 2)
    n = int(np.searchsorted(e, (1.0 - nu_tol) * e[-1] * (1 - 1e-15)) + 1)
    return U[:, :n], s
