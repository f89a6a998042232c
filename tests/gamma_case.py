"""A workload whose subdomain 0 is singular in its interface block (test helper, no method arithmetic).

Subdomain 0's collocation rows are chosen so that no 5-point stencil touches one of its interface states: the
row's node and its in-grid neighbours are all interior states of subdomain 0.  Then R_0 = Z_0 dr/dx dg/dxh has
zero interface columns, H_0 = R_0^T R_0 is singular in its Gamma block while positive definite on its Omega
block, and the KKT system stays solvable through the constraint (Lemma 1 needs H_i PD on null(E_i) only).  The
other subdomains keep the seeded draw."""
import numpy as np

import inputs
from oracle.dd import decompose


def gamma_singular_workload(name="tiny16x16_2x2", n_nodes=8):
    wl = inputs.workload(name)
    dd = decompose(wl.nx, wl.ny, wl.xb, wl.yb)
    N = wl.nx * wl.ny
    sd = dd.subs[0]
    interior = set(int(v) for v in sd.interior if v < N)
    rows = []
    for k, p in enumerate(sd.nodes):
        i, j = int(p) % wl.nx, int(p) // wl.nx
        nb = [p] + ([p - 1] if i > 0 else []) + ([p + 1] if i < wl.nx - 1 else []) + \
             ([p - wl.nx] if j > 0 else []) + ([p + wl.nx] if j < wl.ny - 1 else [])
        if all(int(q) in interior for q in nb):
            rows.append(k)
    rows = rows[:n_nodes]
    n_owned = len(sd.nodes)
    hr = inputs.hr_sets(wl)
    hr[0] = np.array(sorted(rows + [n_owned + k for k in rows]), dtype=np.int64)
    wl.hr_override = hr
    return wl
