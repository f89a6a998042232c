"""The 1024x1024 grid, 8x8 subdomains, latent (8, 4), width 1024, 2% collocation rows, n_C = 128 workload at
its full size.  The oracle cannot solve 1024 instances in a test, so the checks are sampled: one evaluation of a
few instances block by block, and the whole 1024-instance batch solved in the launch plan the benchmark uses
for the full 15 SQP iterations, with 16 seeded instances compared element by element against the oracle's
solves (run in a process pool on the host cores), in the mixed and the FP64 path."""
import numpy as np
import pytest

import inputs
import parity
from oracle import setup

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)
lib = pytest.importorskip("paper_2305_15163_gb300")

FP64, MIXED = 0, 1
TOL = {FP64: 1e-6, MIXED: 1e-4}
TOL_EVAL = {FP64: 1e-9, MIXED: 2e-5}
K = 15
N_SAMPLE = 16


@pytest.fixture(scope="module")
def large():
    wl = inputs.workload("c5")
    mu = inputs.mu_batch(wl.batch)
    pick = np.sort(np.random.default_rng(55).choice(wl.batch, N_SAMPLE, replace=False))
    # oracle solves in a spawn pool (a forked pool after CUDA initialisation could hang)
    refs = parity.oracle_solves("c5", mu[pick], tol=0.0, max_iter=K)
    fom, dd, rom, raw = setup.build(wl)
    solvers = {}
    for prec in (MIXED, FP64):
        s = lib.Solver(wl, precision=prec)
        s.load(raw["dec_o"], raw["dec_g"], raw["C"])
        solvers[prec] = s
    yield wl, rom, solvers, mu, pick, refs
    for s in solvers.values():
        s.close()


@pytest.mark.parametrize("prec", [MIXED, FP64])
def test_one_evaluation_sampled(large, prec):
    wl, rom, solvers, _, _, _ = large
    s = solvers[prec]
    B = 3
    r = np.random.default_rng(12)
    mu = inputs.mu_batch(B, seed=91)
    x = 0.3 * r.standard_normal((B, rom.n_D))
    lam = r.standard_normal((B, rom.n_C))
    H, D, A = s.linearize(mu, x, lam)
    F, rhr = s.residual(mu, x, lam)
    for b in (0, B - 1):
        ev = rom.evaluate(x[b], lam[b], mu[b])
        parity.evaluation(rom, ev, TOL_EVAL[prec], H=H[b], D=D[b], A=A[b], F=F[b], rhr=rhr[b],
                          what=f"c5 instance {b}")


@pytest.mark.parametrize("prec", [MIXED, FP64])
def test_full_batch_solve_sampled(large, prec):
    """All 1024 instances in one batched solve (graph-resident loop, autotuned plan as in the benchmark),
    15 SQP iterations; 16 seeded instances against the oracle element by element, and the whole batch
    reproducible bit for bit."""
    wl, rom, solvers, mu, pick, refs = large
    s = solvers[prec]
    lib.ddnm_autotune(s.ctx, mu, max_iter=1, reps=1)
    s.options(tol=0.0, max_iter=K)
    x, lam, st = s.solve(mu)
    assert np.all(st["iters"] == K) and np.all(np.isfinite(st["merit"]))
    for b, ref in zip(pick, refs):
        parity.solve_result(rom, x[b], lam[b], st[b], ref, TOL[prec], f"c5 prec {prec} instance {b}")
    x2, lam2, st2 = s.solve(mu)
    assert np.array_equal(x, x2) and np.array_equal(lam, lam2)
    s.options()
