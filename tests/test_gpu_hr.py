"""Gappy-POD hyper-reduction on the GPU (Sec. 3.1 Eq. dd_lspg_NLP with B_i = (Z_i Phi_i^r)^+ Z_i; Sec. 5.3
greedy remark) against the oracle's gappy ROM, and the FOM residual entry point that collects the residual
snapshots.

The sample rows and projectors come from the oracle (residual snapshots of its Newton history, its POD and
greedy selection; ddnm_hr_select is checked against it on the host) and are given to both sides: the GPU
evaluation's blocks per subdomain and element (1e-9 FP64, 2e-5 mixed), and a few SQP iterations (1e-6 / 1e-4,
integer results exactly)."""
import numpy as np
import pytest

import inputs
import parity
from oracle import setup
from oracle.burgers import Burgers
from oracle.dd import decompose
from oracle.decoders import MaskedDecoder
from oracle.hr import gappy_hr, residual_snapshots
from oracle.rom import DDROM

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)
lib = pytest.importorskip("paper_2305_15163_gb300")

FP64, MIXED = 0, 1
TOL = {FP64: 1e-6, MIXED: 1e-4}
TOL_EVAL = {FP64: 1e-9, MIXED: 2e-5}


def gappy_case(name, prec, side=3, nr=6):
    wl = inputs.workload(name)
    fom = Burgers(wl.nx, wl.ny, wl.nu)
    dd = decompose(wl.nx, wl.ny, wl.xb, wl.yb)
    S = residual_snapshots(fom, inputs.snapshot_mu(side))
    n_s = [len(h) for h in inputs.hr_sets(wl)]
    rows, projs = gappy_hr(fom, dd, S, n_s, nu_tol=1e-14, max_nr=nr)
    wl.hr_override = rows
    raw = setup.build(wl)[3]
    rom = DDROM(fom, dd, [MaskedDecoder(d) for d in raw["dec_o"]], [MaskedDecoder(d) for d in raw["dec_g"]], rows,
                raw["C"], hr_proj=projs)
    s = lib.Solver(wl, precision=prec)
    s.load(raw["dec_o"], raw["dec_g"], raw["C"])
    for i, p in enumerate(projs):
        lib.ddnm_set_hr_projection(s.ctx, i, p)
    return wl, fom, rom, s


@pytest.mark.parametrize("name,prec", [("c1", FP64), ("c1", MIXED), ("tiny13x9_3x2", FP64), ("tiny13x9_3x2", MIXED)])
def test_gappy_evaluation_matches_oracle(name, prec):
    wl, fom, rom, s = gappy_case(name, prec)
    B = 3
    r = np.random.default_rng(11)
    mu = inputs.mu_batch(B, seed=78)
    x = 0.3 * r.standard_normal((B, rom.n_D))
    lam = r.standard_normal((B, rom.n_C))
    H, D, A = s.linearize(mu, x, lam)
    F, rhr = s.residual(mu, x, lam)
    for b in range(B):
        ev = rom.evaluate(x[b], lam[b], mu[b])
        parity.evaluation(rom, ev, TOL_EVAL[prec], H=H[b], D=D[b], A=A[b], F=F[b], rhr=rhr[b],
                          what=f"gappy {name} instance {b}")
    s.close()


@pytest.mark.parametrize("name,prec,K", [("c1", FP64, 4), ("c1", MIXED, 2), ("tiny13x9_3x2", FP64, 3)])
def test_gappy_iterations_match_oracle(name, prec, K):
    wl, fom, rom, s = gappy_case(name, prec)
    mu = inputs.mu_batch(3, seed=5)
    s.options(tol=0.0, max_iter=K)
    x, lam, st = s.solve(mu)
    for b in range(3):
        ref = rom.solve(mu[b], tol=0.0, max_iter=K)
        parity.solve_result(rom, x[b], lam[b], st[b], ref, TOL[prec], f"gappy {name} K={K} instance {b}")
    # back to collocation: the projector cleared, the evaluation equals the plain collocated one
    for i in range(wl.n_sub):
        lib.ddnm_set_hr_projection(s.ctx, i, None)
    col = DDROM(rom.fom, rom.dd, rom.dO, rom.dG, [np.searchsorted(sd.res_rows, rr) for sd, rr in
                                                    zip(rom.dd.subs, rom.rows)], rom.C)
    H, _, _ = s.linearize(mu, np.zeros((3, rom.n_D)))
    for b in range(3):
        ev = col.evaluate(np.zeros(rom.n_D), np.zeros(rom.n_C), mu[b])
        parity.evaluation(col, ev, 1e-9 if prec == FP64 else 2e-5, H=H[b], what=f"collocation again {b}")
    s.close()


@pytest.mark.parametrize("name", ["tiny12x10_2x2", "c2"])
def test_fom_residual_matches_oracle(name):
    """ddnm_fom_residual against the oracle's Eq. (burgers_discretized) residual at perturbed exact states, per
    component block and element (1e-11 of the block's largest entry), host and device memory."""
    wl = inputs.workload(name)
    fom = Burgers(wl.nx, wl.ny, wl.nu)
    s = lib.Solver(wl)
    mu = inputs.mu_batch(3, seed=8)
    r = np.random.default_rng(3)
    X = np.array([fom.exact_state(m) for m in mu]) + 1e-2 * r.standard_normal((3, 2 * fom.N))
    Rg = lib.ddnm_fom_residual(s.ctx, mu, X)
    dev = torch.device("cuda:0")
    Rd = torch.zeros((3, 2 * fom.N), dtype=torch.float64, device=dev)
    lib.ddnm_fom_residual(s.ctx, torch.from_numpy(mu).to(dev), torch.from_numpy(X).to(dev), Rd)
    torch.cuda.synchronize()
    assert np.array_equal(Rd.cpu().numpy(), Rg)
    N = fom.N
    for b in range(3):
        ref = fom.residual(X[b], mu[b])
        parity.close(Rg[b][:N], ref[:N], 1e-11, f"{name} r_u {b}")
        parity.close(Rg[b][N:], ref[N:], 1e-11, f"{name} r_v {b}")
    s.close()
