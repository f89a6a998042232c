"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the same seeded inputs.

Tolerances (relative, in the 2-norm over the compared quantity):
* FP64 path: 1e-6 on latent coordinates, multipliers and reconstructed state (1e-9 on one
  evaluation's blocks, where only rounding order differs);
* mixed path (FP32 evaluation, FP64 KKT): 1e-4 -- one evaluation carries ~1e-6 relative
  FP32 rounding, which the Gauss-Newton steps of a few iterations amplify by at most ~10^2.
Integer work (sizes, index maps, iteration and evaluation counts) must match exactly.
"""
import numpy as np
import pytest

import inputs
from oracle import setup

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)
lib = pytest.importorskip("paper_2305_15163_gb300")

_CACHE = {}


def case(name, precision):
    key = (name, precision)
    if key not in _CACHE:
        wl = inputs.workload(name)
        fom, dd, rom, raw = setup.build(wl)
        s = lib.Solver(wl, precision=precision)
        s.load(raw["dec_o"], raw["dec_g"], raw["C"])
        _CACHE[key] = (wl, fom, dd, rom, raw, s)
    return _CACHE[key]


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


FP64, MIXED = 0, 1
TOL = {FP64: 1e-6, MIXED: 1e-4}
TOL_EVAL = {FP64: 1e-9, MIXED: 2e-5}

EVAL_CASES = [("c1", FP64), ("c1", MIXED), ("tiny12x10_2x2", FP64), ("tiny12x10_2x2", MIXED),
              ("tiny13x9_3x2", FP64), ("tiny13x9_3x2", MIXED), ("c2", MIXED), ("c2", FP64), ("c3", MIXED)]


@pytest.mark.parametrize("name,prec", EVAL_CASES)
def test_one_evaluation(name, prec):
    """H_i, D_i, Atil, F = [rho; Atil] and the collocated residuals at a random (xh, lambda)."""
    wl, fom, dd, rom, raw, s = case(name, prec)
    B = 3
    r = np.random.default_rng(10)
    mu = inputs.mu_batch(B, seed=77)
    x = 0.3 * r.standard_normal((B, rom.n_D))
    lam = r.standard_normal((B, rom.n_C))
    H, D, A = s.linearize(mu, x, lam)
    F, rhr = s.residual(mu, x, lam)
    for b in range(B):
        ev = rom.evaluate(x[b], lam[b], mu[b])
        assert rel(H[b], np.concatenate([h.ravel() for h in ev.H])) < TOL_EVAL[prec]
        assert rel(D[b], np.concatenate([d.ravel() for d in ev.D])) < TOL_EVAL[prec]
        assert rel(A[b], ev.Atil) < TOL_EVAL[prec]
        assert rel(F[b], ev.F) < TOL_EVAL[prec]
        assert rel(rhr[b], np.concatenate(ev.r)) < TOL_EVAL[prec]


@pytest.mark.parametrize("name,prec,K", [("c1", FP64, 1), ("c1", FP64, 2), ("c1", FP64, 3), ("c1", FP64, 15),
                                         ("tiny12x10_2x2", FP64, 6), ("tiny13x9_3x2", FP64, 4),
                                         ("c1", MIXED, 1), ("c1", MIXED, 3), ("tiny12x10_2x2", MIXED, 3),
                                         ("c3", MIXED, 2)])
def test_fixed_iterations(name, prec, K):
    """K SQP iterations (tol = 0): same iterates, same line-search decisions, same counts."""
    wl, fom, dd, rom, raw, s = case(name, prec)
    mu = inputs.mu_batch(3)
    s.options(tol=0.0, max_iter=K)
    x, lam, st = s.solve(mu)
    for b in range(3):
        ref = rom.solve(mu[b], tol=0.0, max_iter=K)
        assert st[b]["iters"] == K and st[b]["status"] == lib.DDNM_MAX_ITER
        assert st[b]["n_evals"] == ref.n_evals
        assert rel(x[b], ref.x) < TOL[prec] and rel(lam[b], ref.lam) < TOL[prec]
        assert abs(st[b]["merit"] - ref.phi) <= TOL[prec] * ref.phi
        assert st[b]["alpha_last"] == ref.alpha_hist[-1]


def test_default_options_c1_fp64():
    """The paper's stopping rule (||F|| < 1e-4 or 15 iterations) on the 32x32 FP64 workload."""
    wl, fom, dd, rom, raw, s = case("c1", FP64)
    s.options()
    mu = inputs.mu_batch(4)
    x, lam, st, state = s.solve(mu, state=True)
    for b in range(4):
        ref = rom.solve(mu[b])
        assert st[b]["status"] == ref.status and st[b]["iters"] == ref.iters
        assert rel(x[b], ref.x) < TOL[FP64] and rel(lam[b], ref.lam) < TOL[FP64]
        assert rel(state[b], rom.full_state(ref.x)) < TOL[FP64]


def test_given_multiplier_start_and_x0():
    wl, fom, dd, rom, raw, s = case("tiny12x10_2x2", FP64)
    s.options(tol=0.0, max_iter=2)
    r = np.random.default_rng(3)
    mu = inputs.mu_batch(2)
    x0 = 0.2 * r.standard_normal((2, rom.n_D))
    l0 = r.standard_normal((2, rom.n_C))
    x, lam, st = s.solve(mu, x0=x0, lam0=l0)
    for b in range(2):
        ref = rom.solve(mu[b], x0=x0[b], lam0=l0[b], tol=0.0, max_iter=2)
        assert rel(x[b], ref.x) < TOL[FP64] and rel(lam[b], ref.lam) < TOL[FP64]
        assert st[b]["n_evals"] == ref.n_evals


def test_c2_full_launch_sampled():
    """The 128x128 4x4 workload as the benchmark launches it (64 instances, mixed path,
    paper's stopping rule); instances 0 and 41 re-solved by the oracle."""
    wl, fom, dd, rom, raw, s = case("c2", MIXED)
    s.options()
    mu = inputs.mu_batch(wl.batch)
    x, lam, st = s.solve(mu)
    assert np.all((st["status"] == lib.DDNM_MAX_ITER) | (st["status"] == lib.DDNM_CONVERGED))
    for b in (0, 41):
        ref = rom.solve(mu[b])
        assert st[b]["iters"] == ref.iters and st[b]["status"] == ref.status
        assert rel(x[b], ref.x) < TOL[MIXED] and rel(lam[b], ref.lam) < TOL[MIXED]


def test_reconstruction_and_full_residual():
    wl, fom, dd, rom, raw, s = case("tiny12x10_2x2", FP64)
    r = np.random.default_rng(5)
    mu = inputs.mu_batch(2)
    x = 0.3 * r.standard_normal((2, rom.n_D))
    F, rhr, rfull = s.residual(mu, x, None, full=True)
    for b in range(2):
        st = rom.full_state(x[b])
        assert rel(rfull[b], fom.residual(st, mu[b])) < 1e-10


def test_device_memory_path_matches_host():
    wl, fom, dd, rom, raw, s = case("tiny12x10_2x2", MIXED)
    s.options(tol=0.0, max_iter=3)
    mu = inputs.mu_batch(5)
    x, lam, st = s.solve(mu)
    dev = torch.device("cuda:0")
    mu_d = torch.from_numpy(mu).to(dev)
    x_d = torch.zeros((5, rom.n_D), dtype=torch.float64, device=dev)
    l_d = torch.zeros((5, rom.n_C), dtype=torch.float64, device=dev)
    st_d = torch.zeros(5 * 32, dtype=torch.uint8, device=dev)
    lib.ddnm_solve_batch(s.ctx, 5, mu_d, None, None, x_d, l_d, None, st_d)
    torch.cuda.synchronize()
    assert np.array_equal(x_d.cpu().numpy(), x) and np.array_equal(l_d.cpu().numpy(), lam)
    st2 = np.frombuffer(st_d.cpu().numpy().tobytes(), dtype=lib.STATS_DTYPE)
    assert np.array_equal(st2["n_evals"], st["n_evals"])


def test_non_pd_hessian_reports_kkt_fail():
    """W1 = 0 makes every decoder constant: R_i = 0, H_i = 0 is not PD (Lemma 1 fails)."""
    wl = inputs.workload("tiny12x10_2x2")
    fom, dd, rom, raw = setup.build(wl)
    s = lib.Solver(wl, precision=FP64)
    dec_o = [dict(d, W1=np.zeros_like(d["W1"])) for d in raw["dec_o"]]
    s.load(dec_o, raw["dec_g"], raw["C"])
    x, lam, st = s.solve(inputs.mu_batch(2))
    assert np.all(st["status"] == lib.DDNM_KKT_FAIL)
    s.close()


def test_nan_weights_end_with_a_status_not_a_hang():
    wl = inputs.workload("tiny12x10_2x2")
    fom, dd, rom, raw = setup.build(wl)
    s = lib.Solver(wl, precision=MIXED)
    dec_g = [dict(d, scale=np.full_like(d["scale"], np.nan)) for d in raw["dec_g"]]
    s.load(raw["dec_o"], dec_g, raw["C"])
    x, lam, st = s.solve(inputs.mu_batch(3))
    assert np.all(np.isin(st["status"], [lib.DDNM_NONFINITE, lib.DDNM_KKT_FAIL]))
    s.close()


def test_batch_sizes_ragged():
    """B = 1 and an odd B give the same per-instance results as a larger batch."""
    wl, fom, dd, rom, raw, s = case("tiny13x9_3x2", MIXED)
    s.options(tol=0.0, max_iter=2)
    mu = inputs.mu_batch(7)
    x7, l7, st7 = s.solve(mu)
    x1, l1, st1 = s.solve(mu[3:4])
    assert np.array_equal(x1[0], x7[3]) and np.array_equal(l1[0], l7[3])


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_gamma_singular_block_matches_oracle(prec):
    """Subdomain 0 singular in its interface block (collocation rows that touch no interface state, see
    tests/gamma_case.py): its factorisation stops after the Omega columns, the KKT step keeps its interface
    steps as unknowns of the second Schur level, and 3 SQP iterations match the oracle's dense KKT solves."""
    from gamma_case import gamma_singular_workload
    wl = gamma_singular_workload()
    fom, dd, rom, raw = setup.build(wl)
    s = lib.Solver(wl, precision=prec)
    s.load(raw["dec_o"], raw["dec_g"], raw["C"])
    mu = inputs.mu_batch(3)
    s.options(tol=0.0, max_iter=3)
    x, lam, st = s.solve(mu)
    for b in range(3):
        ref = rom.solve(mu[b], tol=0.0, max_iter=3)
        assert st[b]["status"] == lib.DDNM_MAX_ITER and st[b]["n_evals"] == ref.n_evals
        assert rel(x[b], ref.x) < TOL[prec] and rel(lam[b], ref.lam) < TOL[prec]
    s.close()
