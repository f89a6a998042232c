"""Strong ROM-port constraint (SRPC) formulation (Sec. 3.2, Eq. dd_lspg_NLP_rom_port; Sec. 5.2, Eq.
interface_decoder_rom_port_blocks), FP64 / integer bookkeeping.

Test infrastructure only (see ``oracle/__init__``).

Ports: the interface variables of the FOM grouped by the set P(j) of subdomains sharing them (Sec. 2), each
port's variables x_j^p in ascending global order.  Each port j gets one decoder g_j^p: R^{n_j^p} -> R^{N_j^p}
with n_j^p = max(min(N_j^p - 1, n~), 1) (Sec. 7.5).  Subdomain i's reduced interface variable is the
concatenation of the port latents of its ports Q(i) (ascending port order), x^_j^p = P^_i^j x^_i^G, and

    g_i^G(x^_i^G) = sum_{j in Q(i)} (P_i^j)^T g_j^p(P^_i^j x^_i^G)           (Eq. gamma_map_port)

which is one shallow decoder whose W1 and W2 are block-diagonal over the ports (Eq.
interface_decoder_rom_port_blocks).  The constraints are linear, sum_i A^_i x^_i^G = 0 (Eq.
rom_strong_constraint): for every port j with sharing set s_0 < ... < s_{m-1} and every latent component c of the
port, the rows x^_{s_k}[c] - x^_{s_{k+1}}[c], k = 0..m-2; rows ordered by port, then component, then k (the
FOM's A_i orders by variable, then chain position; this is the same rule on the port latents).
"""
from __future__ import annotations

import numpy as np

from .dd import Decomposition


def ports(dd: Decomposition):
    """[(P(j) as a sorted tuple, global variable ids of port j, ascending)] in ascending order of P(j)."""
    N = dd.nx * dd.ny
    owners: dict = {}
    for sd in dd.subs:
        for v in sd.interface:
            owners.setdefault(int(v), []).append(sd.index)
    groups: dict = {}
    for v, subs in owners.items():
        groups.setdefault(tuple(sorted(subs)), []).append(v)
    out = []
    for key in sorted(groups):
        vs = np.array(sorted(groups[key]), dtype=np.int64)
        out.append((key, vs))
    assert sum(len(v) for _, v in out) == len({v for sd in dd.subs for v in sd.interface})
    assert all(len(k) >= 2 for k, _ in out) and N > 0
    return out


def port_latent_sizes(port_list, n_tilde: int):
    """n_j^p = max(min(N_j^p - 1, n~), 1) (Sec. 7.5)."""
    return [max(min(len(v) - 1, n_tilde), 1) for _, v in port_list]


def subdomain_ports(dd: Decomposition, port_list, n_p):
    """Per subdomain: Q(i) as [(port j, offset of x^_j^p in x^_i^G)], and n_i^G = sum of its ports' n_j^p."""
    Q, n_gamma = [], []
    for sd in dd.subs:
        q, off = [], 0
        for j, (key, _) in enumerate(port_list):
            if sd.index in key:
                q.append((j, off))
                off += n_p[j]
        Q.append(q)
        n_gamma.append(off)
    return Q, n_gamma


def rom_port_constraints(dd: Decomposition, port_list, n_p, Q, n_gamma):
    """A^_i (n_A x n_i^G) for every subdomain, entries in {-1, 0, 1} (Eq. rom_strong_constraint)."""
    n_A = sum((len(key) - 1) * n_p[j] for j, (key, _) in enumerate(port_list))
    A = [np.zeros((n_A, g)) for g in n_gamma]
    offs = [{j: o for j, o in q} for q in Q]
    row = 0
    for j, (key, _) in enumerate(port_list):
        for c in range(n_p[j]):
            for k in range(len(key) - 1):
                lo, hi = key[k], key[k + 1]
                A[lo][row, offs[lo][j] + c] = 1.0
                A[hi][row, offs[hi][j] + c] = -1.0
                row += 1
    return A


def interface_decoder(sd, port_list, port_decs, q):
    """g_i^G of subdomain sd assembled from the port decoders of its ports q = [(j, latent offset)] (Eq.
    interface_decoder_rom_port_blocks): hidden units and latents of the ports stacked in port order, W1 and W2
    block-diagonal; every interface row takes the row of its port's decoder.  Returns a decoder spec (ELL W2)."""
    hid_off, lat_off = {}, {}
    w = n = 0
    for j, o in q:
        hid_off[j] = w
        lat_off[j] = o
        w += port_decs[j]["w"]
        n += port_decs[j]["n"]
    W1 = np.zeros((w, n))
    b1 = np.zeros(w)
    for j, _ in q:
        d = port_decs[j]
        W1[hid_off[j]:hid_off[j] + d["w"], lat_off[j]:lat_off[j] + d["n"]] = d["W1"]
        b1[hid_off[j]:hid_off[j] + d["w"]] = d["b1"]
    K = max(np.asarray(port_decs[j]["cols"]).shape[1] for j, _ in q)
    N = sd.interface.size
    cols = np.full((N, K), -1, dtype=np.int32)
    vals = np.zeros((N, K))
    scale = np.ones(N)
    offset = np.zeros(N)
    for j, _ in q:
        d = port_decs[j]
        pos = np.searchsorted(sd.interface, port_list[j][1])          # rows of port j in x_i^G (P_i^j)
        dc = np.asarray(d["cols"])
        kk = dc.shape[1]
        cols[pos, :kk] = np.where(dc >= 0, dc + hid_off[j], -1)
        vals[pos, :kk] = np.where(dc >= 0, np.asarray(d["vals"]), 0.0)
        scale[pos] = d["scale"]
        offset[pos] = d["offset"]
    acts = {port_decs[j].get("act", "sigmoid") for j, _ in q}
    assert len(acts) == 1
    return dict(N=N, w=w, n=n, act=acts.pop(), W1=W1, b1=b1, cols=cols, vals=vals, scale=scale, offset=offset)
