"""Launch plan of the batched solve: the graph-resident SQP loop (one CUDA graph launch with a device-side
while loop per instance group), the persistent evaluation and the constraint-slice size change how the work
is scheduled, never what is computed.  Every such plan gives bit-identical iterates, multipliers and
per-instance statistics to the host-driven loop.  Where D_i is formed (inside the evaluation or in the
batched GEMM) changes its summation order only: both match the oracle.  The autotuner returns a valid plan
and the solve under it still matches the oracle."""
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
HOST = dict(graph=0, chains=1, con_split=512, eval_persist=0, eval_groups=1)
PLANS = [dict(graph=1, chains=1, con_split=512, eval_persist=0),
         dict(graph=1, chains=3, con_split=1024, eval_persist=2, eval_groups=0),
         dict(graph=1, chains=16, con_split=2048, eval_persist=1),
         dict(graph=1, chains=64, con_split=512, eval_persist=0),
         dict(graph=1, chains=4, con_split=512, eval_persist=4, eval_groups=0),
         dict(graph=0, chains=1, con_split=2048, eval_persist=3),
         dict(graph=0, chains=1, con_split=512, eval_persist=0, eval_groups=0)]
TOL = {FP64: 1e-6, MIXED: 1e-4}


def solver(name, prec):
    wl = inputs.workload(name)
    s = lib.Solver(wl, precision=prec)
    dec_o, dec_g = inputs.decoders_for(wl, [d["interior"] for d in s.subs], [d["interface"] for d in s.subs])
    s.load(dec_o, dec_g, inputs.test_matrix(wl.n_c(), s.sizes.N_A))
    return wl, s


def same(a, b):
    xa, la, sa = a
    xb, lb, sb = b
    assert np.array_equal(xa, xb) and np.array_equal(la, lb)
    for f in ("iters", "status", "flags", "n_evals", "merit", "alpha_last"):
        assert np.array_equal(sa[f], sb[f]), f


@pytest.mark.parametrize("d_gemm,atil", [(0, 0), (1, 0), (0, 1)])
@pytest.mark.parametrize("name,prec,B", [("c2", MIXED, 13), ("c2", FP64, 5), ("c3", MIXED, 7), ("c1", FP64, 1),
                                         ("tiny13x9_3x2", MIXED, 4), ("c2", MIXED, 40)])
def test_plans_are_bit_identical(name, prec, B, d_gemm, atil):
    """Every launch plan gives the same bits (the double-float Atil of the mixed path too: its summation order
    does not depend on the instance tiles, whose size follows the instance group's)."""
    wl, s = solver(name, prec)
    mu = inputs.mu_batch(B, seed=31)
    s.options(tol=0.0, max_iter=4)
    lib.ddnm_set_tune(s.ctx, **HOST, d_gemm=d_gemm, atil=atil)
    ref = s.solve(mu)
    for plan in PLANS:
        lib.ddnm_set_tune(s.ctx, **plan, d_gemm=d_gemm, atil=atil)
        same(s.solve(mu), ref)
        same(s.solve(mu), ref)                 # replay of the captured graph
    s.options()
    lib.ddnm_set_tune(s.ctx, **HOST, d_gemm=d_gemm, atil=atil)
    ref = s.solve(mu)                          # stopping rule active: groups finish at different passes
    lib.ddnm_set_tune(s.ctx, graph=1, chains=min(B, 5), con_split=1024, eval_persist=2, d_gemm=d_gemm, atil=atil)
    same(s.solve(mu), ref)
    s.close()


@pytest.mark.parametrize("name,B", [("c2", 70), ("c3", 19), ("tiny13x9_3x2", 5), ("c5", 67)])
def test_tensor_core_d_gemm_matches_fp32_gemm(name, B):
    """D_i = Q_i P_G on the tensor cores (d_gemm = 2: tcgen05 kind::tf32 with hi + lo operand splits, FP32
    accumulation) against the FP32-pipe GEMM (d_gemm = 1), block by block at 1e-5 of the block's largest
    entry (both carry FP32 rounding of sums over up to 1024 hidden units, in different orders; the split
    operands add about 2^-21 per product); H_i and Atil, which do not depend on D_i, are bit-identical, and
    F = [rho; Atil] agrees at 1e-5 per block.  Batches of 70 and 67
    instances cover a full tile of 64 and a ragged one."""
    wl, s = solver(name, MIXED)
    r = np.random.default_rng(6)
    mu = inputs.mu_batch(B, seed=43)
    x = 0.3 * r.standard_normal((B, s.sizes.n_D))
    lam = r.standard_normal((B, s.sizes.n_C))
    out = {}
    for d in (1, 2):
        lib.ddnm_set_tune(s.ctx, d_gemm=d)
        H, D, A = s.linearize(mu, x, lam)
        F, _ = s.residual(mu, x, lam)
        out[d] = (H, D, A, F)
    (H1, D1, A1, F1), (H2, D2, A2, F2) = out[1], out[2]
    assert np.array_equal(H1, H2) and np.array_equal(A1, A2)
    nC = s.sizes.n_C
    sizes_D = [nC * d["n_gamma"] for d in s.subs]
    sizes_F = [d["n_omega"] + d["n_gamma"] for d in s.subs] + [nC]
    for b in range(B):
        for i, (d1, d2) in enumerate(zip(parity.split(D1[b], sizes_D), parity.split(D2[b], sizes_D))):
            parity.close(d2, d1, 1e-5, f"{name} instance {b} D_{i}")
        for i, (f1, f2) in enumerate(zip(parity.split(F1[b], sizes_F), parity.split(F2[b], sizes_F))):
            parity.close(f2, f1, 1e-5, f"{name} instance {b} F block {i}")
    s.close()


@pytest.mark.parametrize("name,B", [("c2", 40), ("c3", 19), ("tiny13x9_3x2", 5), ("c5", 33)])
def test_double_float_atil_matches_fp64(name, B):
    """The mixed path's Atil = C jump on the FP32 pipe in double-float arithmetic (atil = 1) against the same
    product in FP64 (atil = 0) on the same FP32 interface outputs: within 1e-10 of the larger entries, per
    entry (the double-float sum carries about 2^-48 of sum_l |C_kl jump_l|, which the cancellation in C jump
    raises relative to |Atil| by about sqrt(N_A)).  The evaluation's other outputs are bit-identical."""
    wl, s = solver(name, MIXED)
    r = np.random.default_rng(5)
    mu = inputs.mu_batch(B, seed=41)
    x = 0.3 * r.standard_normal((B, s.sizes.n_D))
    lam = r.standard_normal((B, s.sizes.n_C))
    lib.ddnm_set_tune(s.ctx, atil=0)
    H0, D0, A0 = s.linearize(mu, x, lam)
    lib.ddnm_set_tune(s.ctx, atil=1)
    H1, D1, A1 = s.linearize(mu, x, lam)
    assert np.array_equal(H0, H1) and np.array_equal(D0, D1)
    for b in range(B):
        parity.close(A1[b], A0[b], 1e-10, f"{name} Atil instance {b}")
    s.close()


@pytest.mark.parametrize("name,prec", [("c1", FP64), ("c1", MIXED), ("tiny13x9_3x2", FP64), ("c3", MIXED)])
def test_both_d_forms_match_oracle(name, prec):
    """D_i inside the evaluation and D_i from the batched GEMM: both against the FP64 oracle (3 SQP
    iterations, same line-search decisions)."""
    wl = inputs.workload(name)
    fom, dd, rom, raw = setup.build(wl)
    s = lib.Solver(wl, precision=prec)
    s.load(raw["dec_o"], raw["dec_g"], raw["C"])
    mu = inputs.mu_batch(3)
    s.options(tol=0.0, max_iter=3)
    refs = [rom.solve(mu[b], tol=0.0, max_iter=3) for b in range(3)]
    for d_gemm in ((0, 1) if prec == FP64 else (0, 1, 2)):
        lib.ddnm_set_tune(s.ctx, graph=1, chains=2, d_gemm=d_gemm)
        x, lam, st = s.solve(mu)
        for b in range(3):
            parity.solve_result(rom, x[b], lam[b], st[b], refs[b], TOL[prec], f"d_gemm {d_gemm} instance {b}")
    s.close()


def test_graph_with_warm_start_and_starts():
    """The warm-start screening runs inside the graph (2B instances, then the selection); explicit starts
    x0 / lam0 skip it.  Both match the host-driven loop bit for bit."""
    wl, s = solver("c2", MIXED)
    nD, nC = s.sizes.n_D, s.sizes.n_C
    lib.ddnm_ws_init(s.ctx, 64, inputs.mlp_init(2, 64, nD))
    mu = inputs.mu_batch(64, seed=9)
    x_tr, _, _ = s.solve(mu)
    lib.ddnm_ws_train(s.ctx, mu, x_tr, 20, 32, 2e-3, inputs.mlp_order(64, 20))
    lib.ddnm_ws_enable(s.ctx, True)
    mu_te = inputs.mu_batch(11, seed=10)
    s.options(tol=0.0, max_iter=3)
    lib.ddnm_set_tune(s.ctx, **HOST)
    ref = s.solve(mu_te)
    lib.ddnm_set_tune(s.ctx, graph=1, chains=4, con_split=1024, eval_persist=2)
    same(s.solve(mu_te), ref)
    lib.ddnm_ws_enable(s.ctx, False)
    r = np.random.default_rng(2)
    x0, lam0 = 0.1 * r.standard_normal((11, nD)), r.standard_normal((11, nC))
    lib.ddnm_set_tune(s.ctx, **HOST)
    ref = s.solve(mu_te, x0=x0, lam0=lam0)
    lib.ddnm_set_tune(s.ctx, graph=1, chains=2, con_split=512, eval_persist=0)
    same(s.solve(mu_te, x0=x0, lam0=lam0), ref)
    s.close()


def test_launch_counts_of_graph_solve():
    """The graph's loop passes are read back: per pass and instance group one launch per width class,
    then the constraint (with the block factorisations) and KKT-step kernels (the step ends the pass with the
    loop control)."""
    wl, s = solver("c3", MIXED)
    mu = inputs.mu_batch(6, seed=3)
    s.options(tol=0.0, max_iter=2)
    lib.ddnm_timing_enable(s.ctx, True)
    lib.ddnm_timing_enable(s.ctx, False)           # counters reset, timing (host loop) off
    t0 = lib.ddnm_get_timing(s.ctx)
    lib.ddnm_set_tune(s.ctx, graph=1, chains=2, con_split=512, eval_persist=0)
    x, lam, st = s.solve(mu)
    t1 = lib.ddnm_get_timing(s.ctx)
    passes = t1["constraint_launches"] - t0["constraint_launches"]
    evals = t1["eval_launches"] - t0["eval_launches"]
    assert t1["step_launches"] - t0["step_launches"] == passes            # k_kkt
    assert evals % passes == 0 and evals // passes >= 1
    assert int(st["n_evals"].max()) <= passes <= 2 * (3 + 2 * 21)
    s.close()


def test_autotune_then_parity_with_oracle():
    wl = inputs.workload("c1")
    fom, dd, rom, raw = setup.build(wl)
    s = lib.Solver(wl, precision=FP64)
    s.load(raw["dec_o"], raw["dec_g"], raw["C"])
    mu = inputs.mu_batch(3)
    plan, ms = lib.ddnm_autotune(s.ctx, mu, max_iter=2, reps=2)
    assert plan["graph"] == 1 and 1 <= plan["chains"] <= 3 and plan["con_split"] in (512, 1024, 2048)
    assert plan["eval_persist"] in (0, 1, 2, 4) and plan["d_gemm"] in (0, 1) and plan["eval_groups"] in (0, 1)
    assert ms > 0
    assert lib.ddnm_get_tune(s.ctx) == plan
    s.options(tol=0.0, max_iter=3)
    x, lam, st = s.solve(mu)
    for b in range(3):
        res = rom.solve(mu[b], tol=0.0, max_iter=3)
        parity.solve_result(rom, x[b], lam[b], st[b], res, 1e-6, f"autotuned instance {b}")
    s.close()
