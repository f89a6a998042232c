"""Pins of the oracle's SRPC formulation (Sec. 3.2, Eq. dd_lspg_NLP_rom_port; Sec. 5.2, Eq.
interface_decoder_rom_port_blocks) against what the paper fixes: the ports partition the interface variables,
the constraint matrix has full row rank with a null space of dimension sum_i n_i^G - n_A (Theorem
dd_lspg_NLP_rom_port_solution i), the assembled interface decoders reproduce the port decoders port by port,
and -- the point of the formulation -- strong FOM-port compatibility sum_i A_i g_i^G(xh_i^G) = 0 holds at every
point of that null space; an SRPC SQP solve is feasible after its first full step."""
import numpy as np
import pytest

import inputs
from oracle.decoders import MaskedDecoder
from srpc_case import srpc_case, srpc_rom


@pytest.mark.parametrize("name", ["tiny12x10_2x2", "tiny13x9_3x2", "c1"])
def test_ports_partition_the_interface(name):
    wl, dd, pl, n_p, Q, n_gamma, Ah, _, _ = srpc_case(name)
    for sd in dd.subs:
        mine = np.concatenate([vs for key, vs in pl if sd.index in key])
        assert np.array_equal(np.sort(mine), sd.interface)
    assert all(1 <= n <= len(vs) - 1 or len(vs) == 1 for n, (_, vs) in zip(n_p, pl))
    assert n_gamma == [sum(n_p[j] for j, _ in q) for q in Q]


@pytest.mark.parametrize("name", ["tiny12x10_2x2", "tiny13x9_3x2", "c1"])
def test_constraint_rank_and_null_space(name):
    wl, dd, pl, n_p, Q, n_gamma, Ah, _, _ = srpc_case(name)
    M = np.hstack(Ah)
    n_A = sum((len(k) - 1) * n_p[j] for j, (k, _) in enumerate(pl))
    assert M.shape == (n_A, sum(n_gamma))
    assert set(np.unique(M)) <= {-1.0, 0.0, 1.0}
    assert np.linalg.matrix_rank(M) == n_A
    assert M.shape[1] - n_A >= 1
    # every row is one port latent equal across two neighbouring subdomains of the port
    assert np.all((M != 0).sum(axis=1) == 2) and np.all(M.sum(axis=1) == 0)


@pytest.mark.parametrize("name", ["tiny12x10_2x2", "tiny13x9_3x2"])
def test_assembled_decoder_reproduces_port_decoders(name):
    wl, dd, pl, n_p, Q, n_gamma, Ah, port_decs, dec_g = srpc_case(name)
    r = np.random.default_rng(0)
    for i, sd in enumerate(dd.subs):
        g = MaskedDecoder(dec_g[i])
        x = r.standard_normal(n_gamma[i])
        val, J = g.value_jacobian(x)
        for j, o in Q[i]:
            pd = MaskedDecoder(port_decs[j])
            pos = np.searchsorted(sd.interface, pl[j][1])
            xj = x[o:o + n_p[j]]
            assert np.allclose(val[pos], pd.value(xj), rtol=1e-14, atol=1e-15)
            Jj = np.zeros((len(pos), n_gamma[i]))
            Jj[:, o:o + n_p[j]] = pd.jacobian(xj)
            assert np.allclose(J[pos], Jj, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("name", ["tiny12x10_2x2", "tiny13x9_3x2", "c1"])
def test_strong_compatibility_on_the_null_space(name):
    """sum_i A^_i xh_i^G = 0  implies  sum_i A_i g_i^G(xh_i^G) = 0 (Sec. 3.2); off the null space it fails."""
    wl, dd, pl, n_p, Q, n_gamma, Ah, _, dec_g = srpc_case(name)
    M = np.hstack(Ah)
    _, sv, Vt = np.linalg.svd(M)
    Z = Vt[M.shape[0]:].T                                     # orthonormal null-space basis
    r = np.random.default_rng(1)
    xg = Z @ r.standard_normal(Z.shape[1])
    off = np.concatenate([[0], np.cumsum(n_gamma)]).astype(int)
    decs = [MaskedDecoder(d) for d in dec_g]
    jump = sum(dd.A[i] @ decs[i].value(xg[off[i]:off[i + 1]]) for i in range(dd.n_sub))
    scale = max(np.abs(decs[i].value(xg[off[i]:off[i + 1]])).max() for i in range(dd.n_sub))
    assert np.max(np.abs(jump)) <= 1e-14 * scale * 10
    bad = xg + 0.1 * r.standard_normal(xg.size)
    jump2 = sum(dd.A[i] @ decs[i].value(bad[off[i]:off[i + 1]]) for i in range(dd.n_sub))
    assert np.max(np.abs(jump2)) > 1e-6 * scale


@pytest.mark.parametrize("name", ["tiny12x10_2x2", "tiny13x9_3x2"])
def test_srpc_solve_is_feasible_after_the_first_step(name):
    """The constraints are linear: from x^ = 0 (feasible) the SQP step keeps A^ x^ = 0 to rounding whatever the
    step length, and D_i = A^_i at every evaluation."""
    wl, dd, rom, dec_o, port_decs, Ah, n_gamma = srpc_rom(name)
    mu = inputs.mu_batch(1, seed=3)[0]
    res = rom.solve(mu, tol=0.0, max_iter=1)
    off = np.concatenate([[0], np.cumsum(rom.n_i)]).astype(int)
    cons = sum(Ah[i] @ res.x[off[i] + rom.nO[i]:off[i + 1]] for i in range(len(Ah)))
    assert np.max(np.abs(cons)) <= 1e-12 * max(1.0, np.abs(res.x).max())
    ev = rom.evaluate(res.x, res.lam, mu)
    for i in range(len(Ah)):
        assert np.array_equal(ev.D[i], Ah[i])
    assert np.max(np.abs(ev.Atil)) <= 1e-12 * max(1.0, np.abs(res.x).max())
