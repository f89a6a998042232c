"""The 1024x1024 grid, 8x8 subdomains, latent (8, 4), width 1024, 2% collocation rows, n_C = 128 workload at
its full size.  The oracle cannot solve 1024 instances, so the checks are sampled: one evaluation of a few
instances block by block, and the whole 1024-instance batch solved in the launch plan the benchmark uses,
with sampled instances compared one by one against the oracle's solve from the same start (2 SQP
iterations), in the mixed and the FP64 path."""
import numpy as np
import pytest

import inputs
from oracle import setup

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)
lib = pytest.importorskip("paper_2305_15163_gb300")

FP64, MIXED = 0, 1
TOL = {FP64: 1e-6, MIXED: 1e-4}
TOL_EVAL = {FP64: 1e-9, MIXED: 2e-5}


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def large():
    wl = inputs.workload("c5")
    fom, dd, rom, raw = setup.build(wl)
    solvers = {}
    for prec in (MIXED, FP64):
        s = lib.Solver(wl, precision=prec)
        s.load(raw["dec_o"], raw["dec_g"], raw["C"])
        solvers[prec] = s
    yield wl, rom, solvers
    for s in solvers.values():
        s.close()


@pytest.mark.parametrize("prec", [MIXED, FP64])
def test_one_evaluation_sampled(large, prec):
    wl, rom, solvers = large
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
        assert rel(F[b], ev.F) < TOL_EVAL[prec]
        assert rel(H[b], np.concatenate([h.ravel() for h in ev.H])) < TOL_EVAL[prec]
        assert rel(D[b], np.concatenate([d.ravel() for d in ev.D])) < TOL_EVAL[prec]
        assert rel(A[b], ev.Atil) < TOL_EVAL[prec]
        assert rel(rhr[b], np.concatenate(ev.r)) < TOL_EVAL[prec]


def test_full_batch_solve_sampled(large):
    """All 1024 instances in one batched solve (graph-resident loop, autotuned plan as in the benchmark),
    2 SQP iterations; instances 0 and 1023 against the oracle in both precisions, and the whole batch
    reproducible bit for bit."""
    wl, rom, solvers = large
    mu = inputs.mu_batch(wl.batch)
    K = 2
    refs = {b: rom.solve(mu[b], tol=0.0, max_iter=K) for b in (0, wl.batch - 1)}
    for prec, s in solvers.items():
        lib.ddnm_autotune(s.ctx, mu, max_iter=1, reps=1)
        s.options(tol=0.0, max_iter=K)
        x, lam, st = s.solve(mu)
        assert np.all(st["iters"] == K) and np.all(np.isfinite(st["merit"]))
        for b, ref in refs.items():
            assert st[b]["n_evals"] == ref.n_evals
            assert rel(x[b], ref.x) < TOL[prec] and rel(lam[b], ref.lam) < TOL[prec]
            assert abs(st[b]["merit"] - ref.phi) <= TOL[prec] * ref.phi
        x2, lam2, st2 = s.solve(mu)
        assert np.array_equal(x, x2) and np.array_equal(lam, lam2)
        s.options()
