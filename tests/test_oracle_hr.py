"""Pins of the oracle's gappy-POD hyper-reduction (Sec. 3.1 Eq. dd_lspg_NLP with B_i = (Z_i Phi_i^r)^+ Z_i;
Sec. 5.3 greedy remark): residual snapshots, the greedy row sampling and the gappy ROM, against closed forms,
special cases that reduce to collocation or to vanilla LSPG, invariances and finite differences."""
import numpy as np
import pytest

import inputs
from oracle import setup
from oracle.burgers import Burgers
from oracle.dd import decompose
from oracle.decoders import MaskedDecoder
from oracle.hr import gappy_hr, gappy_projector, greedy_rows, residual_basis, residual_snapshots
from oracle.rom import DDROM


def test_greedy_picks_the_rows_of_unit_basis_vectors():
    """Phi = columns e_5, e_2, e_9: each step's fit error is the next unit vector, so the rows are 5, 2, 9."""
    Phi = np.eye(12)[:, [5, 2, 9]]
    assert list(greedy_rows(Phi, 3)) == [2, 5, 9]


def test_greedy_first_row_is_largest_entry_and_rows_distinct():
    r = np.random.default_rng(0)
    Phi = np.linalg.qr(r.standard_normal((60, 5)))[0]
    rows = greedy_rows(Phi, 17)
    assert len(set(rows)) == 17 and np.all(np.diff(rows) > 0)
    assert int(np.argmax(np.abs(Phi[:, 0]))) in rows
    # with the basis' own rows, Z Phi has full column rank
    assert np.linalg.matrix_rank(Phi[rows]) == 5


def test_greedy_is_equivariant_under_row_permutation_and_column_scaling():
    r = np.random.default_rng(1)
    Phi = r.standard_normal((40, 4))
    rows = greedy_rows(Phi, 9)
    perm = r.permutation(40)                      # row i of Phi becomes row inv[i] of Phi[perm]
    inv = np.argsort(perm)
    assert sorted(inv[rows]) == list(greedy_rows(Phi[perm], 9))
    scaled = Phi * np.array([-3.0, 0.5, 7.0, -0.25])
    assert list(greedy_rows(scaled, 9)) == list(rows)


def test_gappy_reconstruction_is_exact_on_the_basis_span():
    """Phi (Z Phi)^+ Z r = r for r in span(Phi) once Z Phi has full column rank; with every row sampled and Phi
    orthonormal, (Z Phi)^+ = Phi^T."""
    r = np.random.default_rng(2)
    Phi = np.linalg.qr(r.standard_normal((50, 6)))[0]
    rows = greedy_rows(Phi, 10)
    P = gappy_projector(Phi, rows)
    v = Phi @ r.standard_normal(6)
    assert np.allclose(Phi @ (P @ v[rows]), v, rtol=0, atol=1e-12)
    assert np.allclose(gappy_projector(Phi, np.arange(50)), Phi.T, atol=1e-13)


def test_residual_snapshots_follow_newtons_history():
    """Newton from 0 on the 12 x 10 grid: one snapshot per iterate but the converged last one; the first is
    r(0); every snapshot is the FOM residual of an iterate (norms falling); POD of them spans them."""
    fom = Burgers(12, 10, 0.1)
    mus = inputs.mu_batch(2, seed=4)
    S = residual_snapshots(fom, mus)
    rs = []
    _, hist = fom.newton(mus[0], residuals=rs)
    assert len(rs) == len(hist)
    n0 = len(rs) - 1
    assert np.allclose(S[0], fom.residual(np.zeros(2 * fom.N), mus[0]), rtol=0, atol=1e-14)
    assert np.all(np.diff(np.linalg.norm(S[:n0], axis=1)) < 0)
    Phi = residual_basis(S, nu_tol=1e-12)        # energy criterion: the discarded energy is below 1e-12
    assert np.linalg.norm(S.T - Phi @ (Phi.T @ S.T)) <= 1e-6 * np.linalg.norm(S)


def _tiny(hr_proj=None, hr=None):
    wl = inputs.workload("tiny12x10_2x2")
    fom = Burgers(wl.nx, wl.ny, wl.nu)
    dd = decompose(wl.nx, wl.ny, wl.xb, wl.yb)
    raw = setup.build(wl)[3]
    return wl, fom, dd, DDROM(fom, dd, [MaskedDecoder(d) for d in raw["dec_o"]],
                              [MaskedDecoder(d) for d in raw["dec_g"]], raw["hr"] if hr is None else hr,
                              raw["C"], hr_proj=hr_proj), raw


def test_gappy_with_identity_projector_is_collocation():
    """(Z Phi)^+ = I (Phi = Z^T: the basis of unit vectors at the sampled rows) gives B_i = Z_i."""
    wl, fom, dd, col, raw = _tiny()
    eye = [np.eye(len(h)) for h in raw["hr"]]
    _, _, _, gap, _ = _tiny(hr_proj=eye)
    mu = inputs.mu_batch(1)[0]
    x = 0.2 * np.random.default_rng(3).standard_normal(col.n_D)
    lam = np.random.default_rng(4).standard_normal(col.n_C)
    a, b = col.evaluate(x, lam, mu), gap.evaluate(x, lam, mu)
    for i in range(len(a.H)):
        assert np.allclose(a.H[i], b.H[i], rtol=1e-14, atol=0) and np.allclose(a.rho[i], b.rho[i], rtol=1e-14, atol=0)


def test_gappy_objective_gradient_matches_finite_differences():
    """rho_i's R_i^T r_i part is the gradient of 1/2 ||B_i r_i||^2 with B_i = (Z_i Phi_i^r)^+ Z_i (a residual
    basis from the Newton history, 10 sampled rows): central differences of the objective."""
    wl, fom, dd, col, raw = _tiny()
    S = residual_snapshots(fom, inputs.snapshot_mu(2))
    rows, projs = gappy_hr(fom, dd, S, [10] * wl.n_sub)
    _, _, _, gap, _ = _tiny(hr_proj=projs, hr=rows)
    mu = inputs.mu_batch(1)[0]
    x = 0.2 * np.random.default_rng(5).standard_normal(gap.n_D)
    lam = np.zeros(gap.n_C)
    ev = gap.evaluate(x, lam, mu)

    def obj(xx):
        e = gap.evaluate(xx, lam, mu)
        return 0.5 * sum(float(np.sum((projs[i] @ e.r[i]) ** 2)) for i in range(wl.n_sub))

    g = np.concatenate(ev.grad)
    eps = 1e-6
    for k in range(gap.n_D):
        d = np.zeros(gap.n_D)
        d[k] = eps
        fd = (obj(x + d) - obj(x - d)) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k]))
    for i in range(wl.n_sub):
        Rb = projs[i] @ ev.R[i]
        assert np.allclose(ev.H[i], Rb.T @ Rb, rtol=1e-13, atol=0)


def test_gappy_sampling_all_rows_with_full_basis_is_vanilla_lspg():
    """Every residual row sampled and Phi^r orthonormal and complete (n_r = N_r): B_i = Phi^T, an orthogonal map,
    so ||B_i r_i|| = ||r_i||: H_i and the gradient equal those of B_i = I."""
    wl = inputs.workload("tiny12x10_2x2")
    fom = Burgers(wl.nx, wl.ny, wl.nu)
    dd = decompose(wl.nx, wl.ny, wl.xb, wl.yb)
    raw = setup.build(wl)[3]
    r = np.random.default_rng(6)
    projs, rows = [], []
    for sd in dd.subs:
        n = sd.res_rows.size
        Phi = np.linalg.qr(r.standard_normal((n, n)))[0]
        rows.append(np.arange(n))
        projs.append(gappy_projector(Phi, np.arange(n)))
    decs = ([MaskedDecoder(d) for d in raw["dec_o"]], [MaskedDecoder(d) for d in raw["dec_g"]])
    full = DDROM(fom, dd, *decs, None, raw["C"])
    gap = DDROM(fom, dd, *decs, rows, raw["C"], hr_proj=projs)
    mu = inputs.mu_batch(1)[0]
    x = 0.2 * r.standard_normal(full.n_D)
    lam = r.standard_normal(full.n_C)
    a, b = full.evaluate(x, lam, mu), gap.evaluate(x, lam, mu)
    for i in range(wl.n_sub):
        assert np.allclose(a.H[i], b.H[i], rtol=1e-10, atol=1e-10 * np.abs(a.H[i]).max())
        assert np.allclose(a.rho[i], b.rho[i], rtol=1e-10, atol=1e-10 * np.abs(a.rho[i]).max())
