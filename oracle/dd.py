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
    owner = np.empty(N, dtype=np.int64)
    owned = []
    for sy in range(ky):
        for sx in range(kx):
            s = sy * kx + sx
            ii, jj = np.meshgrid(np.arange(xb[sx], xb[sx + 1]), np.arange(yb[sy], yb[sy + 1]))
            nodes = np.sort((jj * nx + ii).ravel())
            owner[nodes] = s
            owned.append(nodes)
    n = kx * ky
    # dependency node sets and, for every node, the subdomains whose residuals it enters
    dep = []
    enters = [set() for _ in range(N)]
    for s in range(n):
        d = set()
        for p in owned[s]:
            d.update(_neighbours(int(p), nx, ny))
        dep.append(np.array(sorted(d), dtype=np.int64))
        for q in d:
            enters[q].add(s)
    subs = []
    for s in range(n):
        shared = np.array([len(enters[q]) > 1 for q in dep[s]])
        inter_nodes = dep[s][~shared]
        face_nodes = dep[s][shared]
        subs.append(Subdomain(
            index=s, nodes=owned[s],
            res_rows=np.concatenate([owned[s], N + owned[s]]),
            interior=np.concatenate([inter_nodes, N + inter_nodes]),
            interface=np.concatenate([face_nodes, N + face_nodes])))
    # compatibility rows, by global variable then chain position
    loc = [dict(zip(sd.interface.tolist(), range(sd.interface.size))) for sd in subs]
    rows, cols_sub, cols_loc, vals, row_var, row_pair = [], [], [], [], [], []
    ports: dict = {}
    r = 0
    for var in range(2 * N):
        S = sorted(enters[var % N])
        if len(S) < 2:
            continue
        ports[tuple(S)] = ports.get(tuple(S), 0) + 1
        for k in range(len(S) - 1):
            lo, hi = S[k], S[k + 1]
            rows += [r, r]
            cols_sub += [lo, hi]
            cols_loc += [loc[lo][var], loc[hi][var]]
            vals += [1.0, -1.0]
            row_var.append(var)
            row_pair.append((lo, hi))
            r += 1
    rows = np.array(rows, dtype=np.int64)
    cols_sub = np.array(cols_sub, dtype=np.int64)
    cols_loc = np.array(cols_loc, dtype=np.int64)
    vals = np.array(vals)
    A = []
    for s in range(n):
        m = cols_sub == s
        A.append(sp.csr_matrix((vals[m], (rows[m], cols_loc[m])), shape=(r, subs[s].interface.size)))
    return Decomposition(nx, ny, subs, A, ports, np.array(row_var, dtype=np.int64),
                         np.array(row_pair, dtype=np.int64).reshape(-1, 2))


def restrict(dd: Decomposition, x: np.ndarray):
    """(P_i^Omega x, P_i^Gamma x) for every subdomain."""
    return [(x[sd.interior], x[sd.interface]) for sd in dd.subs]
