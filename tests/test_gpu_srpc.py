"""The SRPC formulation on the GPU (Sec. 3.2, Eq. dd_lspg_NLP_rom_port; Sec. 5.2, Eq.
interface_decoder_rom_port_blocks) against the oracle's SRPC ROM on the same seeded port decoders.

The library builds the ports, A^_i and the assembled interface decoders itself (ddnm_set_srpc,
ddnm_load_port_decoder; the host test checks the bookkeeping against the oracle exactly); here the evaluation
(H_i, D_i = A^_i exactly, Atil = sum_i A^_i xh_i^G, rho_i, the collocated residuals) is compared per block and
element (1e-9 FP64, 2e-5 mixed), then a few SQP iterations (1e-6 / 1e-4; counts, status and flags exactly).
Every residual row is collocated (B_i = I), as in the oracle's pins: with sampled rows a small corner port can
be seen by no row, and its latent is then fixed by nothing.  The solutions satisfy the linear constraints to
rounding, and through them strong compatibility of the decoded interface states (sum_i A_i g_i^G = 0)."""
import numpy as np
import pytest

import inputs
import parity
from srpc_case import srpc_rom

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)
lib = pytest.importorskip("paper_2305_15163_gb300")

FP64, MIXED = 0, 1
TOL = {FP64: 1e-6, MIXED: 1e-4}
TOL_EVAL = {FP64: 1e-9, MIXED: 2e-5}


def srpc_solver(name, n_tilde, prec):
    wl, dd, rom, dec_o, port_decs, Ah, n_gamma = srpc_rom(name, n_tilde)
    wl.hr_override = [np.arange(n) for n in wl.residual_rows()]
    s = lib.Solver(wl, precision=prec, n_gamma=n_gamma, n_c=Ah[0].shape[0])
    s.load_srpc(n_tilde, dec_o, port_decs)
    return wl, dd, rom, s, Ah


CASES = [("tiny12x10_2x2", 2, FP64), ("tiny12x10_2x2", 4, MIXED), ("c1", 3, FP64), ("c1", 1, MIXED),
         ("tiny13x9_3x2", 1, FP64)]


@pytest.mark.parametrize("name,n_tilde,prec", CASES)
def test_srpc_evaluation_matches_oracle(name, n_tilde, prec):
    wl, dd, rom, s, Ah = srpc_solver(name, n_tilde, prec)
    B = 3
    r = np.random.default_rng(21)
    mu = inputs.mu_batch(B, seed=61)
    x = 0.3 * r.standard_normal((B, rom.n_D))
    lam = r.standard_normal((B, rom.n_C))
    H, D, A = s.linearize(mu, x, lam)
    F, rhr = s.residual(mu, x, lam)
    for b in range(B):
        ev = rom.evaluate(x[b], lam[b], mu[b])
        parity.evaluation(rom, ev, TOL_EVAL[prec], H=H[b], A=A[b], F=F[b], rhr=rhr[b],
                          what=f"SRPC {name} n~={n_tilde} instance {b}")
        for i, d in enumerate(parity.split(D[b], [rom.n_C * g for g in rom.nG])):
            assert np.array_equal(d.reshape(rom.n_C, rom.nG[i]), Ah[i]), f"instance {b}: D_{i} is not A^_{i}"
    s.close()


@pytest.mark.parametrize("name,n_tilde,prec,K", [("tiny12x10_2x2", 2, FP64, 4), ("tiny12x10_2x2", 4, FP64, 6),
                                                 ("c1", 3, FP64, 5), ("tiny13x9_3x2", 1, FP64, 3)])
def test_srpc_iterations_match_oracle(name, n_tilde, prec, K):
    """FP64 only: the corner ports' latents (one node, two outputs) give H_i pivots of 1e-5 to 1e-9 of the
    block's largest diagonal entry, at or below the mixed path's rank test, so the mixed path takes their
    directions as singular where the oracle solves for them; its evaluation is compared above."""
    wl, dd, rom, s, Ah = srpc_solver(name, n_tilde, prec)
    mu = inputs.mu_batch(4, seed=17)
    s.options(tol=0.0, max_iter=K)
    x, lam, st = s.solve(mu)
    off = np.concatenate([[0], np.cumsum(rom.n_i)]).astype(int)
    for b in range(len(mu)):
        ref = rom.solve(mu[b], tol=0.0, max_iter=K)
        parity.solve_result(rom, x[b], lam[b], st[b], ref, TOL[prec], f"SRPC {name} n~={n_tilde} K={K} instance {b}")
        # from the feasible start xh = 0 every full or damped step keeps sum_i A^_i xh_i^G = 0 to the rounding of
        # the KKT solves, and the decoded interface states then agree across the subdomains sharing them
        # (Sec. 3.2); off the null space they disagree by O(0.1) (the oracle's pin)
        xg = [x[b][off[i] + rom.nO[i]:off[i + 1]] for i in range(dd.n_sub)]
        cons = sum(Ah[i] @ xg[i] for i in range(dd.n_sub))
        assert np.max(np.abs(cons)) <= 1e-10 * max(1.0, np.abs(x[b]).max())
        vals = [rom.dG[i].value(xg[i]) for i in range(dd.n_sub)]
        jump = sum(dd.A[i] @ vals[i] for i in range(dd.n_sub))
        assert np.max(np.abs(jump)) <= 1e-9 * max(np.abs(v).max() for v in vals)
    s.close()
