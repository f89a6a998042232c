"""Gappy-POD hyper-reduction (Sec. 3.1 Eq. dd_lspg_NLP, Sec. 5.3 and its greedy-sampling remark), FP64.

Test infrastructure only (see ``oracle/__init__``).

For subdomain i with residual rows P_i^r (N_i^r of them):

    residual snapshots   r(x_k; mu) at every Newton iterate x_k of the FOM solves (Sec. 5.3 remark: the
                         iteration history of Newton's method), restricted to the subdomain's rows
    residual basis       Phi_i^r: POD of those snapshots (thin SVD, Eq. energy_criterion), n_i^r columns
    row sampling         Z_i: N_i^B rows chosen greedily from Phi_i^r (below)
    HR operator          B_i = (Z_i Phi_i^r)^+ Z_i   (Moore-Penrose pseudoinverse; n_i^r x N_i^r)

so that the ROM objective 1/2 sum_i ||B_i r_i||^2 uses the sampled residual rows Z_i r_i mapped onto the
coefficients of their least-squares fit in the residual basis.

Readings (the paper defers the greedy algorithm to Carlberg et al. 2013, Algo. 3, and fixes no sizes):
* residual snapshots come from Newton started at x = 0 (the oracle FOM's default start), every iterate
  above the final (converged) one;
* n_i^r = the energy criterion with tolerance ``nu_tol``, capped at ``max_nr``;
* greedy sampling, one row per step: step k < n_r picks the row where basis vector k is worst reproduced
  by the least-squares fit of basis vectors 0..k-1 on the rows picked so far (at k = 0: the largest entry of
  vector 0), which makes Z Phi square and invertible after n_r steps; a step k >= n_r picks the row i with the
  largest leverage phi_i^T (Phi_S^T Phi_S)^{-1} phi_i against the picked rows S (phi_i: row i of Phi), the row
  whose addition most increases det(Phi_S^T Phi_S) and so most steadies the least-squares fit.  Rows already
  picked are excluded, ties go to the smaller row index; the rows are returned sorted.
"""
from __future__ import annotations

import numpy as np

from .burgers import Burgers
from .decoders import pod_basis


def residual_snapshots(fom: Burgers, mus) -> np.ndarray:
    """Residual vectors of every Newton iterate of the FOM solves at the rows of mus, except the converged
    last one (n_snap x 2N)."""
    out = []
    for m in np.asarray(mus, dtype=np.float64).reshape(-1, 2):
        rs = []
        fom.newton(m, residuals=rs)
        out.extend(rs[:-1])
    return np.array(out)


def residual_basis(snap_rows: np.ndarray, nu_tol: float = 1e-8, max_nr: int | None = None) -> np.ndarray:
    """POD basis (N_r x n_r) of residual snapshots restricted to one subdomain's rows (n_snap x N_r)."""
    Phi, _ = pod_basis(np.asarray(snap_rows, dtype=np.float64).T, nu_tol)
    if max_nr is not None:
        Phi = Phi[:, :max_nr]
    return Phi


def _fit_error(Phi: np.ndarray, picked: list, cols: int, target: int) -> np.ndarray:
    """Phi[:, target] minus its least-squares fit by Phi[:, :cols] on the picked rows (whole column)."""
    v = Phi[:, target]
    if not picked or cols == 0:
        return v.copy()
    A = Phi[picked, :cols]
    c = np.linalg.lstsq(A, v[picked], rcond=None)[0]
    return v - Phi[:, :cols] @ c


def greedy_rows(Phi: np.ndarray, n_s: int) -> np.ndarray:
    """n_s sample rows for the residual basis Phi (N_r x n_r), n_r <= n_s <= N_r; sorted local row ids."""
    N, n_r = Phi.shape
    assert n_r <= n_s <= N
    picked: list = []
    for k in range(n_s):
        if k < n_r:
            a = np.abs(_fit_error(Phi, picked, k, k))
        else:
            G = Phi[picked].T @ Phi[picked]
            a = np.einsum("ij,ij->i", Phi, np.linalg.solve(G, Phi.T).T)
        a[picked] = -1.0
        picked.append(int(np.argmax(a)))
    return np.sort(np.array(picked, dtype=np.int64))


def gappy_projector(Phi: np.ndarray, rows) -> np.ndarray:
    """(Z Phi)^+ for the sampled rows (n_r x N_B, columns in the order of rows): B_i = this times Z_i."""
    return np.linalg.pinv(Phi[np.asarray(rows)])


def gappy_hr(fom: Burgers, dd, snaps: np.ndarray, n_samples, nu_tol: float = 1e-8, max_nr=None):
    """Per subdomain: (sorted local residual-row ids Z_i, (Z_i Phi_i^r)^+) from residual snapshots (n_snap x 2N).
    n_samples: N_i^B per subdomain; max_nr: cap on n_i^r per subdomain (default N_i^B // 2)."""
    rows, projs = [], []
    for i, sd in enumerate(dd.subs):
        ns = int(n_samples[i])
        cap = ns // 2 if max_nr is None else int(max_nr)
        Phi = residual_basis(snaps[:, sd.res_rows], nu_tol, cap)
        z = greedy_rows(Phi, ns)
        rows.append(z)
        projs.append(gappy_projector(Phi, z))
    return rows, projs
