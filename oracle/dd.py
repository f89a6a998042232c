"""Algebraic domain decomposition of the FOM (Sec. 2), FP64 / integer bookkeeping.

Test infrastructure only (see ``oracle/__init__``).

Readings (the paper states the construction for a generic 5-point stencil, Fig. 1-2):
* subdomains are boxes of grid nodes cut at node breakpoints xb, yb; subdomain
  s = sy*kx + sx (x fastest, as in Fig. 2);
* residual sampling P_i^r takes both residual components (u and v rows) of the nodes a
  subdomain owns; rows in ascending global index (all u rows, then all v rows);
* the variables entering subdomain i's residuals ("dependency set") are u and v at the
  owned nodes and at their in-grid 5-point neighbours;
* interface states of i: dependency variables that also enter another subdomain's
  residuals; interior states: the rest (they only enter subdomain i);
* ports group interface variables by the set P(j) of subdomains sharing them; for each
  shared variable the |P(j)|-1 non-redundant conditions x_{s_1} = x_{s_2}, ...,
  x_{s_{m-1}} = x_{s_m} (ascending subdomain order) give rows of (A_1 .. A_n) with +1 on
  the lower and -1 on the higher subdomain; rows ordered by global variable, then by the
  position in that chain.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp


@dataclass
class Subdomain:
    index: int
    nodes: np.ndarray        # owned node ids, ascending
    res_rows: np.ndarray     # global residual rows (P_i^r), ascending
    interior: np.ndarray     # global variable ids of x_i^Omega (P_i^Omega), ascending
    interface: np.ndarray    # global variable ids of x_i^Gamma (P_i^Gamma), ascending


@dataclass
class Decomposition:
    nx: int
    ny: int
    subs: list
    A: list                  # A_i, sparse N_A x N_i^Gamma
    ports: dict              # tuple(P(j)) -> number of variables N_j^p
    row_var: np.ndarray      # global variable of each constraint row
    row_pair: np.ndarray     # (lower subdomain, higher subdomain) of each constraint row

    @property
    def N_A(self) -> int:
        return self.row_var.size

    @property
    def n_sub(self) -> int:
        return len(self.subs)


def _neighbours(p, nx, ny):
    i, j = p % nx, p // nx
    out = [p]
    if i > 0:
        out.append(p - 1)
    if i < nx - 1:
        out.append(p + 1)
    if j > 0:
        out.append(p - nx)
    if j < ny - 1:
        out.append(p + nx)
    return out


def decompose(nx: int, ny: int, xb, yb) -> Decomposition:
    N = nx * ny
    kx, ky = len(xb) - 1, len(yb) - 1
    n = kx * ky
    owned = []
    for sy in range(ky):
        for sx in range(kx):
            ii, jj = np.meshgrid(np.arange(xb[sx], xb[sx + 1]), np.arange(yb[sy], yb[sy + 1]))
            owned.append(np.sort((jj * nx + ii).ravel()))
    # dependency node sets (owned nodes and their in-grid 5-point neighbours) and, for every node, the
    # subdomains whose residuals it enters, in ascending order (a node enters at most 3 of them)
    dep = []
    cnt = np.zeros(N, dtype=np.int64)
    enters = np.full((N, 5), -1, dtype=np.int64)
    for s in range(n):
        p = owned[s]
        i, j = p % nx, p // nx
        d = np.unique(np.concatenate([p, p[i > 0] - 1, p[i < nx - 1] + 1, p[j > 0] - nx, p[j < ny - 1] + nx]))
        dep.append(d)
        enters[d, cnt[d]] = s
        cnt[d] += 1
    subs = []
    for s in range(n):
        shared = cnt[dep[s]] > 1
        inter_nodes = dep[s][~shared]
        face_nodes = dep[s][shared]
        subs.append(Subdomain(
            index=s, nodes=owned[s],
            res_rows=np.concatenate([owned[s], N + owned[s]]),
            interior=np.concatenate([inter_nodes, N + inter_nodes]),
            interface=np.concatenate([face_nodes, N + face_nodes])))
    # compatibility rows, by global variable then chain position: for each shared variable with sorted
    # sharing set S, the rows x_{S0} - x_{S1}, x_{S1} - x_{S2}, ...
    q = np.flatnonzero(cnt > 1)
    var = np.concatenate([q, N + q])
    node = var % N
    npair = cnt[node] - 1
    row_var = np.repeat(var, npair)
    k = np.arange(row_var.size) - np.repeat(np.cumsum(npair) - npair, npair)
    lo = enters[node.repeat(npair), k]
    hi = enters[node.repeat(npair), k + 1]
    r = row_var.size
    rows = np.arange(r)
    A = []
    for s in range(n):
        iface = subs[s].interface
        ml, mh = lo == s, hi == s
        rr = np.concatenate([rows[ml], rows[mh]])
        cc = np.concatenate([np.searchsorted(iface, row_var[ml]), np.searchsorted(iface, row_var[mh])])
        vv = np.concatenate([np.ones(ml.sum()), -np.ones(mh.sum())])
        A.append(sp.csr_matrix((vv, (rr, cc)), shape=(r, iface.size)))
    ports: dict = {}
    keys, counts = np.unique(enters[q, :], axis=0, return_counts=True)
    for key, c in zip(keys, counts):
        ports[tuple(int(v) for v in key if v >= 0)] = 2 * int(c)     # u and v of each shared node
    return Decomposition(nx, ny, subs, A, ports, row_var.astype(np.int64),
                         np.stack([lo, hi], 1).astype(np.int64).reshape(-1, 2))


def restrict(dd: Decomposition, x: np.ndarray):
    """(P_i^Omega x, P_i^Gamma x) for every subdomain."""
    return [(x[sd.interior], x[sd.interface]) for sd in dd.subs]
