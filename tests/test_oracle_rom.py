"""Pins of the oracle's decoders (Sec. 3.3, 5.1, 5.4) and of the WFPC ROM + SQP (Sec. 3.1, 4)
against finite differences, Lemma 2, library routines and closed forms."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.special as ssp
import scipy.optimize as so

import inputs
from oracle import setup
from oracle.burgers import Burgers
from oracle.dd import decompose
from oracle.decoders import EllDecoder, LinearDecoder, MaskedDecoder, activation, pod_basis, subnet
from oracle.rom import CONVERGED, MAX_ITER, DDROM, relative_error


def _dec(N=40, w=24, n=3, act="swish", seed=0):
    off = np.linspace(-0.2, 0.3, N)
    sc = np.linspace(0.05, 0.1, N)
    return MaskedDecoder(inputs.decoder(N, w, n, 4, (99, seed), off, sc, act=act))


@pytest.mark.parametrize("act", ["swish", "sigmoid", "identity"])
def test_decoder_jacobian_fd(act):
    d = _dec(act=act)
    x = np.random.default_rng(0).standard_normal(3)
    J = d.jacobian(x)
    eps = 1e-6
    for k in range(3):
        e = np.zeros(3); e[k] = eps
        fd = (d.value(x + e) - d.value(x - e)) / (2 * eps)
        assert np.allclose(J[:, k], fd, rtol=1e-7, atol=1e-10)


def test_swish_closed_form():
    f, df = activation("swish")
    assert f(0.0) == 0.0 and df(0.0) == 0.5
    z = np.linspace(-6, 6, 13)
    assert np.allclose(f(z), z * ssp.expit(z))
    assert np.allclose(df(z), (f(z + 1e-6) - f(z - 1e-6)) / 2e-6, atol=1e-8)


def test_subnet_matches_full_decoder():
    """Eq. (subnet): restricted to I_o, the subnet reproduces the full decoder and its Jacobian."""
    d = _dec(N=60, w=300)
    I_o = np.array([3, 7, 8, 20, 41, 59])
    sn = subnet(d, I_o)
    assert np.all(np.diff(sn.I_h) > 0)
    assert set(sn.I_h) == set(np.flatnonzero(d.W2[I_o].any(axis=0)))
    x = np.random.default_rng(1).standard_normal(3)
    assert np.allclose(sn.value(x), d.value(x)[I_o], rtol=1e-14, atol=1e-15)
    assert np.allclose(sn.jacobian(x), d.jacobian(x)[I_o], rtol=1e-14, atol=1e-15)
    assert sn.I_h.size < d.w


def test_band_mask_structure():
    """Sec. 7.3: three bands of b contiguous columns, band shift per row, separation b*shift."""
    N, b = 20, 3
    w = 5 * N
    m = inputs.band_mask(N, w, b)
    for r in (6, 10, 13):
        c = 5 * r
        assert list(m[r]) == list(range(c - 15, c - 12)) + list(range(c, c + 3)) + list(range(c + 15, c + 18))
    assert list(m[0][:3]) == [0, 1, 2] and m[0][6] == -1       # left band clipped at the start
    assert (m >= 0).sum() == 9 * N - 2 * 3 * 3                 # 3 clipped rows at each end


def test_pod_energy_criterion():
    r = np.random.default_rng(2)
    X = r.standard_normal((50, 8)) @ np.diag([10, 5, 2, 1, 0.5, 0.1, 0.01, 0.001]) @ r.standard_normal((8, 12))
    Phi, s = pod_basis(X, 1e-3)
    n = Phi.shape[1]
    e = s ** 2
    assert e[:n].sum() >= (1 - 1e-3) * e.sum() and e[:n - 1].sum() < (1 - 1e-3) * e.sum()
    assert np.allclose(Phi.T @ Phi, np.eye(n))
    err = np.linalg.norm(X - Phi @ (Phi.T @ X)) ** 2      # Eckart-Young: the discarded energy
    assert np.isclose(err, e[n:].sum(), rtol=1e-8)


@pytest.fixture(scope="module")
def tiny():
    wl = inputs.workload("tiny12x10_2x2")
    fom, dd, rom, raw = setup.build(wl)
    return wl, fom, dd, rom, raw


def test_whole_evaluation_fd(tiny):
    """R_i = d(Z_i r_i)/dxh_i, D_i = d Atil/dxh_i^G and grad = R_i^T r_i = d(1/2||Z r||^2)/dxh, by FD."""
    wl, fom, dd, rom, raw = tiny
    mu = inputs.mu_batch(1)[0]
    r = np.random.default_rng(3)
    x = 0.3 * r.standard_normal(rom.n_D)
    lam = r.standard_normal(rom.n_C)
    ev = rom.evaluate(x, lam, mu)
    eps = 1e-6
    for i in range(dd.n_sub):
        a = rom.off[i]
        for k in range(rom.n_i[i]):
            e = np.zeros(rom.n_D); e[a + k] = eps
            ep, em = rom.evaluate(x + e, lam, mu), rom.evaluate(x - e, lam, mu)
            assert np.allclose(ev.R[i][:, k], (ep.r[i] - em.r[i]) / (2 * eps), rtol=1e-6, atol=1e-7)
            obj = lambda E: 0.5 * sum(np.sum(q ** 2) for q in E.r)
            assert np.isclose(ev.grad[i][k], (obj(ep) - obj(em)) / (2 * eps), rtol=1e-6, atol=1e-7)
            if k >= rom.nO[i]:
                fd = (ep.Atil - em.Atil) / (2 * eps)
                assert np.allclose(ev.D[i][:, k - rom.nO[i]], fd, rtol=1e-6, atol=1e-8)
        assert np.allclose(ev.H[i], ev.R[i].T @ ev.R[i])
        assert np.allclose(ev.rho[i][rom.nO[i]:], ev.grad[i][rom.nO[i]:] + ev.D[i].T @ lam)


def test_lemma2_kkt_step_is_qp_solution(tiny):
    """Lemma 2: the KKT step solves the QP Eq. (dd_lspg_NLP_general_QP); its multiplier is lambda + s^lambda.
    Independent route: null-space method (particular solution + basis of null(E))."""
    wl, fom, dd, rom, raw = tiny
    mu = inputs.mu_batch(2)[1]
    r = np.random.default_rng(4)
    x = 0.2 * r.standard_normal(rom.n_D)
    lam = r.standard_normal(rom.n_C)
    ev = rom.evaluate(x, lam, mu)
    s, sl = rom.kkt_step(ev)
    Rb = sla.block_diag(*ev.R)                    # stacked Z R (objective Jacobian)
    rb = np.concatenate(ev.r)
    E = np.hstack([np.hstack([np.zeros((rom.n_C, rom.nO[i])), ev.D[i]]) for i in range(dd.n_sub)])
    sp_ = np.linalg.lstsq(E, -ev.Atil, rcond=None)[0]
    Z = sla.null_space(E)
    y = np.linalg.lstsq(Rb @ Z, -(rb + Rb @ sp_), rcond=None)[0]
    s_qp = sp_ + Z @ y
    assert np.allclose(s, s_qp, rtol=1e-8, atol=1e-10)
    mult = np.linalg.lstsq(E.T, -Rb.T @ (rb + Rb @ s_qp), rcond=None)[0]
    assert np.allclose(lam + sl, mult, rtol=1e-7, atol=1e-9)


def test_lambda_ls(tiny):
    wl, fom, dd, rom, raw = tiny
    mu = inputs.mu_batch(1)[0]
    ev = rom.evaluate(np.zeros(rom.n_D), np.zeros(rom.n_C), mu)
    lam = rom.lambda_ls(ev)
    M = np.vstack([D.T for D in ev.D])
    b = -np.concatenate([g[rom.nO[i]:] for i, g in enumerate(ev.grad)])
    assert np.allclose(M.T @ (M @ lam - b), 0.0, atol=1e-9 * np.abs(M.T @ b).max())
    ev2 = rom.evaluate(np.zeros(rom.n_D), lam, mu)
    g2 = np.concatenate([ev2.rho[i][rom.nO[i]:] for i in range(dd.n_sub)])
    assert np.linalg.norm(g2) <= np.linalg.norm(b) + 1e-12      # the LS multiplier can only reduce it


def test_identity_activation_equals_ls_rom(tiny):
    """A decoder with identity activation is affine; an independently coded linear decoder
    Phi xh + x_ref (Sec. 3.3, LS-ROM) with Phi = diag(scale) W2 W1 gives the same ROM."""
    wl, fom, dd, _, raw = tiny
    C = raw["C"]
    decs = setup.inputs.decoders_for(wl, [s.interior for s in dd.subs], [s.interface for s in dd.subs], act="identity")
    mO, mG = [MaskedDecoder(d) for d in decs[0]], [MaskedDecoder(d) for d in decs[1]]
    lin = lambda m: LinearDecoder(m.scale[:, None] * (m.W2 @ m.W1), m.offset + m.scale * (m.W2 @ m.b1))
    nm = DDROM(fom, dd, mO, mG, raw["hr"], C)
    ls = DDROM(fom, dd, [lin(m) for m in mO], [lin(m) for m in mG], raw["hr"], C)
    mu = inputs.mu_batch(1)[0]
    a = nm.solve(mu, max_iter=6, tol=0.0)
    b = ls.solve(mu, max_iter=6, tol=0.0)
    assert np.allclose(a.x, b.x, rtol=1e-10, atol=1e-12) and np.allclose(a.lam, b.lam, rtol=1e-9, atol=1e-11)


def test_single_domain_is_gauss_newton():
    """n_Omega = 1 (Eq. monolithic_nmrom): no constraints; the SQP reduces to Gauss-Newton and
    its limit matches scipy's least_squares on min ||Z r(g(xh))||^2."""
    nx, ny = 10, 8
    fom = Burgers(nx, ny)
    dd = decompose(nx, ny, [0, nx], [0, ny])
    sd = dd.subs[0]
    assert sd.interface.size == 0 and dd.N_A == 0
    off, sc = inputs.denormalisation(sd.interior, nx, ny)
    dO = MaskedDecoder(inputs.decoder(sd.interior.size, 20, 3, 4, (7, 0), off, sc))
    dG = LinearDecoder(np.zeros((0, 0)))
    hr = [inputs.hr_rows(sd.res_rows.size, 60, 0)]
    rom = DDROM(fom, dd, [dO], [dG], hr, np.zeros((0, 0)))
    mu = (1.0, 1.05)
    res = rom.solve(mu, tol=1e-10, max_iter=60)
    rows = sd.res_rows[hr[0]]

    def fun(xh):
        x = np.zeros(2 * fom.N); x[sd.interior] = dO.value(xh)
        return fom.residual(x, mu)[rows]
    ref = so.least_squares(fun, np.zeros(3), xtol=1e-15, ftol=1e-15, gtol=1e-15, method="lm")
    assert np.allclose(res.x, ref.x, rtol=1e-6, atol=1e-8)


def test_ls_rom_converges_and_constraints_vanish():
    """An LS-ROM (POD of FOM snapshots, Sec. 3.3) with HR: the SQP drives F = [rho; Atil] to zero,
    so the weak interface constraints vanish at convergence; the ROM error vs the FOM is small."""
    nx, ny = 16, 16
    fom = Burgers(nx, ny)
    dd = decompose(nx, ny, [0, 8, 16], [0, 8, 16])
    g = np.linspace(0.9, 1.1, 4)
    snaps = np.stack([fom.newton((a, l))[0] for a in g for l in g], axis=1)
    mean = snaps.mean(axis=1)
    dO, dG = [], []
    for sd in dd.subs:
        PO, _ = pod_basis(snaps[sd.interior] - mean[sd.interior, None], 1e-10)
        PG, _ = pod_basis(snaps[sd.interface] - mean[sd.interface, None], 1e-10)
        dO.append(LinearDecoder(PO[:, :4], mean[sd.interior]))
        dG.append(LinearDecoder(PG[:, :2], mean[sd.interface]))
    hr = [inputs.hr_rows(sd.res_rows.size, 60, i) for i, sd in enumerate(dd.subs)]
    C = inputs.test_matrix(4, dd.N_A)
    rom = DDROM(fom, dd, dO, dG, hr, C)
    mu = (0.95, 1.07)
    res = rom.solve(mu, tol=1e-10, max_iter=40)
    assert res.status == CONVERGED
    ev = rom.evaluate(res.x, res.lam, mu)
    assert np.linalg.norm(ev.Atil) < 1e-10
    xf, _ = fom.newton(mu)
    err = relative_error([(xf[sd.interior], xf[sd.interface]) for sd in dd.subs], rom.states(res.x))
    assert err < 1e-3


def test_random_decoder_sqp_monotone_and_bounded(tiny):
    """Armijo acceptance makes the merit decrease at every accepted step; max_iter always ends it."""
    wl, fom, dd, rom, raw = tiny
    mu = inputs.mu_batch(1)[0]
    res = rom.solve(mu, tol=0.0, max_iter=7)
    assert res.status == MAX_ITER and res.iters == 7
    for k, a in enumerate(res.alpha_hist):
        assert res.phi_hist[k + 1] ** 2 <= (1 - 2e-4 * a) * res.phi_hist[k] ** 2 or a <= 0.5 ** 20
    res0 = rom.solve(mu, tol=0.0, max_iter=3, max_bt=0)
    assert all(a == 1.0 for a in res0.alpha_hist)


def test_relative_error_formula():
    r = np.random.default_rng(5)
    ref = [(r.standard_normal(5), r.standard_normal(3)), (r.standard_normal(4), r.standard_normal(2))]
    assert relative_error(ref, ref) == 0.0
    scaled = [(1.1 * a, 1.1 * b) for a, b in ref]
    assert np.isclose(relative_error(ref, scaled), 0.1)


# ---- the row-restricted and ELL forms the large workloads need, pinned against the plain forms ----

def test_residual_and_jacobian_rows_match_full():
    """Burgers.residual_rows / jacobian_rows are exactly the picked rows of the full residual and
    Jacobian (same operators, restricted before the products)."""
    fom = Burgers(9, 7, 0.1)
    r = np.random.default_rng(5)
    x = r.standard_normal(2 * fom.N)
    mu = (1.03, 0.95)
    rows = np.sort(r.choice(2 * fom.N, size=40, replace=False))
    assert np.allclose(fom.residual_rows(x, mu, rows), fom.residual(x, mu)[rows], rtol=0, atol=1e-13)
    J = fom.jacobian(x, mu)[rows].toarray()
    assert np.allclose(fom.jacobian_rows(x, mu, rows).toarray(), J, rtol=0, atol=1e-13)
    with pytest.raises(ValueError):
        fom.residual_rows(x, mu, rows[::-1])


def test_ell_decoder_matches_dense_decoder():
    """EllDecoder (W2 kept as mask columns and values) against MaskedDecoder (dense W2): values and
    Jacobian rows at any output subset, for a three-band mask with clipped rows."""
    spec = inputs.decoder(37, 48, 5, 4, (91, 1), offset=np.linspace(-1, 1, 37), scale=np.linspace(0.5, 2, 37))
    dense, ell = MaskedDecoder(spec), EllDecoder(spec)
    x = np.random.default_rng(6).standard_normal(5)
    g, J = dense.value_jacobian(x)
    g2, J2 = ell.value_jacobian(x)
    assert np.allclose(g2, g, rtol=1e-14, atol=1e-14) and np.allclose(J2, J, rtol=1e-13, atol=1e-14)
    assert np.allclose(ell.value(x), g, rtol=1e-14, atol=1e-14)
    rows = np.array([0, 3, 17, 36])
    g3, J3 = ell.value_jacobian_rows(x, rows)
    g4, J4 = dense.value_jacobian_rows(x, rows)
    assert np.allclose(g3, g[rows], rtol=1e-14, atol=1e-14) and np.allclose(J3, J[rows], rtol=1e-13, atol=1e-14)
    assert np.allclose(g4, g[rows], rtol=1e-14, atol=1e-14) and np.allclose(J4, J[rows], rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("name", ["c1", "tiny12x10_2x2", "tiny13x9_3x2"])
def test_restricted_evaluation_matches_dense(name):
    """DDROM.evaluate (collocation rows and touched outputs only, sparse C A_i) equals the plain
    whole-state evaluation, for dense and for ELL decoders."""
    wl = inputs.workload(name)
    fom, dd, rom, raw = setup.build(wl)
    fom2, dd2, rom_ell, _ = setup.build(wl, ell=True)
    r = np.random.default_rng(7)
    x = 0.3 * r.standard_normal(rom.n_D)
    lam = r.standard_normal(rom.n_C)
    mu = inputs.mu_batch(1)[0]
    a, b, c = rom.evaluate_dense(x, lam, mu), rom.evaluate(x, lam, mu), rom_ell.evaluate(x, lam, mu)
    for e in (b, c):
        assert np.allclose(e.F, a.F, rtol=1e-12, atol=1e-12)
        for i in range(dd.n_sub):
            assert np.allclose(e.H[i], a.H[i], rtol=1e-12, atol=1e-12)
            assert np.allclose(e.D[i], a.D[i], rtol=1e-12, atol=1e-12)
            assert np.allclose(e.r[i], a.r[i], rtol=1e-12, atol=1e-12)


def test_gamma_singular_case_premise():
    """The case of tests/gamma_case.py: subdomain 0's collocation rows touch no interface state, so R_0 has
    zero interface columns and H_0 is singular in its Gamma block but PD on its Omega block; the KKT matrix of
    Eq. (sqp_system) is still nonsingular (Lemma 1: H_i PD on null(E_i)), and the oracle's SQP runs."""
    from gamma_case import gamma_singular_workload
    wl = gamma_singular_workload()
    fom, dd, rom, raw = setup.build(wl)
    mu = inputs.mu_batch(1)[0]
    ev = rom.evaluate(np.zeros(rom.n_D), np.zeros(rom.n_C), mu)
    nO = rom.nO[0]
    H0 = ev.H[0]
    assert np.abs(ev.R[0][:, nO:]).max() == 0.0
    assert np.abs(H0[nO:, :]).max() == 0.0 and np.abs(H0[:, nO:]).max() == 0.0
    assert np.linalg.eigvalsh(H0[:nO, :nO]).min() > 0.0
    K = rom.kkt_matrix(ev)
    assert np.linalg.cond(K) < 1e12
    res = rom.solve(mu, tol=0.0, max_iter=3)
    assert np.all(np.isfinite(res.x)) and np.all(np.isfinite(res.lam)) and res.iters == 3
