"""Pins of the oracle's algebraic DD (Sec. 2) against what the paper prints and against
Theorem 1.  The printed numbers live in tests/golden/paper_setup_numbers.txt."""
import os

import numpy as np
import pytest

import inputs
from oracle.burgers import Burgers
from oracle.dd import decompose, restrict
from oracle.decoders import IdentityDecoder
from oracle.rom import DDROM, CONVERGED

GOLD = {}
with open(os.path.join(os.path.dirname(__file__), "golden", "paper_setup_numbers.txt")) as f:
    for line in f:
        line = line.split("#")[0].strip()
        if line:
            k, v = (t.strip() for t in line.split("="))
            GOLD[k] = float(v)


def sig4(x):
    return float(f"{x:.3e}")


def ae_params(N, n, nnz_band=5, shift=5):
    """Parameters of one sparse autoencoder of Sec. 5.1 (encoder + decoder), width = shift*N:
    decoder W1 (w x n) + b1 (w) + masked W2; encoder masked W1 + b1 (w) + W2 (n x w)."""
    w = shift * N
    nnz = int((inputs.band_mask(N, w, nnz_band) >= 0).sum())
    return 2 * (w * n + w + nnz), w, nnz


@pytest.fixture(scope="module")
def layouts():
    out = {}
    for kx, ky in ((1, 1), (2, 1), (2, 2), (4, 2), (8, 2)):
        out[(kx, ky)] = decompose(480, 24, inputs.equal_breaks(480, kx), inputs.equal_breaks(24, ky))
    return out


def test_table_nn_params(layouts):
    """Table NN_params: (n^O, n^G) = (6, 3), n = 9 single domain.  "Max # subdomain params" is the
    largest single autoencoder (the interior one); "Total" sums every autoencoder of every subdomain."""
    res = {}
    for (kx, ky), dd in layouts.items():
        if kx * ky == 1:
            p = ae_params(2 * 480 * 24, 9)[0]
            per = [p]
        else:
            per = [ae_params(sd.interior.size, 6)[0] for sd in dd.subs] + \
                  [ae_params(sd.interface.size, 3)[0] for sd in dd.subs]
        res[(kx, ky)] = (max(per), sum(per))
        tag = f"{kx}x{ky}"
        assert sig4(max(per)) == GOLD[f"nnparams_{tag}_max"], (tag, max(per))
        assert sig4(sum(per)) == GOLD[f"nnparams_{tag}_total"], (tag, sum(per))
    base = res[(1, 1)][0]
    for tag, key in (("2x1", (2, 1)), ("2x2", (2, 2)), ("4x2", (4, 2)), ("8x2", (8, 2))):
        red = 100.0 * (1.0 - res[key][0] / base)
        assert round(red, 1) == GOLD[f"nnparams_reduction_{tag}"]
    # the exact counts behind the rounded table
    assert res[(1, 1)][0] == 2995100 and res[(2, 2)] == (525700, 2384080)


def test_sec75_sizes(layouts):
    """Sec. 7.5, 2x2 subdomains: N^G = 1006, N^O = 5258 (printed 5238, see golden note), DoF 25056,
    widths 5N, mask nnz and sparsity."""
    dd = layouts[(2, 2)]
    for sd in dd.subs:
        assert sd.interface.size == GOLD["interface_size_2x2"]
        assert sd.interior.size == GOLD["interior_size_2x2"]
    assert sum(sd.interior.size + sd.interface.size for sd in dd.subs) == GOLD["dof_2x2"]
    _, wO, nnzO = ae_params(5258, 8)
    _, wG, nnzG = ae_params(1006, 4)
    assert (wO, wG) == (GOLD["width_interior_2x2"], GOLD["width_interface_2x2"])
    assert (nnzO, nnzG) == (GOLD["mask_nnz_interior_2x2"], GOLD["mask_nnz_interface_2x2"])
    assert round(100 * (1 - nnzO / (5258 * wO)), 2) == GOLD["sparsity_interior_pct"]
    assert round(100 * (1 - nnzG / (1006 * wG)), 2) == GOLD["sparsity_interface_pct"]


def test_dense_vs_sparse_encoder_counts():
    """Table dense_vs_sparse_encoder: 240x12 single domain (FOM 5760), ROM size 4."""
    N, n = 2 * 240 * 12, 4
    assert N == GOLD["fom_size_240x12"]
    wd = 3 * N
    dense = wd * N + wd + n * wd                  # dense W1 + b1 + W2
    ws = 5 * N
    nnz = int((inputs.band_mask(N, ws, 5) >= 0).sum())
    sparse = nnz + ws + n * ws
    assert wd == GOLD["dense_encoder_width"] and ws == GOLD["sparse_encoder_width"]
    assert float(f"{dense:.2e}") == GOLD["dense_encoder_params"]
    assert float(f"{sparse:.1e}") == GOLD["sparse_encoder_params"]


def test_fig2_ports():
    """Fig. 2: a 2x2 layout has the four edge ports {1,2},{2,4},{3,4},{1,3} and a shared region at
    the cross point.  With the 5-point stencil no variable enters all four residuals: the cross
    region splits into four ports of three subdomains, one node (u and v) each."""
    dd = decompose(12, 10, [0, 6, 12], [0, 5, 10])
    edges = {(0, 1), (1, 3), (2, 3), (0, 2)}
    triples = {(0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)}
    assert set(dd.ports) == edges | triples
    assert all(dd.ports[t] == 2 for t in triples)
    assert dd.ports[(0, 1)] == 2 * 2 * (5 - 1)      # two node columns of height 5 minus the corner nodes
    # N_A = sum_j (|P(j)| - 1) N_j^p
    assert dd.N_A == sum((len(P) - 1) * n for P, n in dd.ports.items())


@pytest.mark.parametrize("nx,ny,xb,yb", [(12, 10, [0, 6, 12], [0, 5, 10]),
                                          (13, 9, [0, 3, 8, 13], [0, 4, 9]),
                                          (10, 10, [0, 10], [0, 2, 5, 10])])
def test_compatibility_matrix_properties(nx, ny, xb, yb):
    dd = decompose(nx, ny, xb, yb)
    A = np.hstack([a.toarray() for a in dd.A])
    # each row is one equality x_s = x_t: exactly one +1 and one -1
    assert np.all((A == 1).sum(axis=1) == 1) and np.all((A == -1).sum(axis=1) == 1)
    assert np.linalg.matrix_rank(A) == dd.N_A                  # full row rank (Sec. 2)
    x = np.random.default_rng(0).standard_normal(2 * nx * ny)
    parts = restrict(dd, x)
    assert np.allclose(sum(a @ g for a, (_, g) in zip(dd.A, parts)), 0.0)
    # residual rows partition the FOM rows; interiors are disjoint
    rows = np.concatenate([sd.res_rows for sd in dd.subs])
    assert np.array_equal(np.sort(rows), np.arange(2 * nx * ny))
    inter = np.concatenate([sd.interior for sd in dd.subs])
    assert np.unique(inter).size == inter.size
    # interior states enter only their own subdomain's residuals; interface states enter another one
    fom = Burgers(nx, ny)
    J = abs(fom.jacobian(np.random.default_rng(1).standard_normal(2 * nx * ny), (1.0, 1.0))).toarray() > 0
    for i, sd in enumerate(dd.subs):
        others = np.concatenate([s.res_rows for s in dd.subs if s.index != i])
        assert not J[np.ix_(others, sd.interior)].any()
        assert J[np.ix_(others, sd.interface)].any(axis=0).all()
        assert set(np.flatnonzero(J[sd.res_rows].any(axis=0))) == set(sd.interior) | set(sd.interface)


def test_theorem1_dd_fom_equals_fom():
    """Theorem 1: with identity maps, B_i = I and C = I (strong constraints) the SQP solution of the
    DD FOM Eq. (fom_dd_nlp) is the monolithic FOM solution, constraints vanish, and the
    Gauss-Newton SQP converges quadratically (zero residual, Theorem 4 with eta_k -> 0)."""
    nx, ny = 8, 6
    fom = Burgers(nx, ny)
    dd = decompose(nx, ny, [0, 4, 8], [0, 3, 6])
    rom = DDROM(fom, dd, [IdentityDecoder(sd.interior.size) for sd in dd.subs],
                [IdentityDecoder(sd.interface.size) for sd in dd.subs], None, np.eye(dd.N_A))
    mu = (1.02, 0.93)
    xf, _ = fom.newton(mu)
    res = rom.solve(mu, tol=1e-11, max_iter=30)
    assert res.status == CONVERGED
    x = np.concatenate([np.concatenate([xf[sd.interior], xf[sd.interface]]) for sd in dd.subs])
    assert np.allclose(res.x, x, atol=1e-10)
    assert np.allclose(rom.full_state(res.x), xf, atol=1e-10)
    ev = rom.evaluate(res.x, res.lam, mu)
    assert np.linalg.norm(ev.Atil) < 1e-11
    h = [p for p in res.phi_hist if p > 1e-9]
    for k in range(1, len(h) - 1):                    # quadratic once close
        if h[k] < 1e-2:
            assert h[k + 1] <= 50.0 * h[k] ** 2
