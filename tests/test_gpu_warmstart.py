"""Learned warm start on the GPU: the hand-written MLP forward/backward and Adam against the FP64 oracle,
and what the trained network gains over the default start on the 128x128 4x4 workload (the plain SQP
from xh0 = 0 is the judge)."""
import os
import tempfile

import numpy as np
import pytest

import inputs
import parity
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)
lib = pytest.importorskip("paper_2305_15163_gb300")

H = 256


def rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def c2():
    wl = inputs.workload("c2")
    s = lib.Solver(wl)
    dec_o, dec_g = inputs.decoders_for(wl, [d["interior"] for d in s.subs], [d["interface"] for d in s.subs])
    s.load(dec_o, dec_g, inputs.test_matrix(wl.n_c(), s.sizes.N_A))
    return wl, s


def test_gradient_parity_with_oracle(c2):
    """One batch: loss and the full gradient (backward kernels) against the FP64 chain rule on the same
    bfloat16 weights; FP32 accumulation bounds the difference at ~1e-5 relative."""
    wl, s = c2
    nD = s.sizes.n_D
    p0 = inputs.mlp_init(2, H, nD)
    lib.ddnm_ws_init(s.ctx, H, p0)
    r = np.random.default_rng(3)
    z = r.uniform(-1, 1, (48, 2)).astype(np.float32)
    t = r.standard_normal((48, nD)).astype(np.float32)
    loss, g = lib.ddnm_ws_loss_grad(s.ctx, z, t, lib.mlp_param_count(2, H, nD))
    L, g_ref = omlp.loss_grad(p0.astype(np.float64), z.astype(np.float64), t.astype(np.float64), 2, H, nD)
    assert abs(loss - L) <= 1e-5 * L
    assert rel(g, g_ref) < 1e-4
    # each parameter block separately, element by element (a transposed block would pass a norm test)
    for k, (gb, rb) in enumerate(zip(parity.split(g, [2 * H, H, H * H, H, nD * H, nD]),
                                     parity.split(g_ref, [2 * H, H, H * H, H, nD * H, nD]))):
        parity.close(gb, rb, 1e-4, f"gradient block {k}")


def test_training_trajectory_matches_oracle(c2):
    """A few epochs of mini-batch Adam: the GPU loss trajectory follows the FP64 oracle's."""
    wl, s = c2
    nD = s.sizes.n_D
    r = np.random.default_rng(4)
    mu = inputs.mu_batch(96, seed=41)
    x = np.tanh(((mu - 1.0) * 5) @ r.standard_normal((2, nD))) + 0.1 * r.standard_normal(nD)
    p0 = inputs.mlp_init(2, H, nD)
    order = inputs.mlp_order(96, 4)
    lib.ddnm_ws_init(s.ctx, H, p0)
    losses = lib.ddnm_ws_train(s.ctx, mu, x, 4, 32, 1e-3, order)
    _, ref, _ = omlp.train(p0, mu, x, 4, 32, 1e-3, order, 2, H, nD)
    assert np.allclose(losses, ref, rtol=2e-3)
    assert losses[-1] < losses[0]


def _solutions(s, mu, B=64):
    xs, sts = [], []
    for b0 in range(0, len(mu), B):
        x, lam, st = s.solve(mu[b0:b0 + B])
        xs.append(x)
        sts.append(st)
    return np.concatenate(xs), np.concatenate(sts)


def test_warm_start_beats_default_start(c2, tmp_path):
    """Trained on 512 SQP solutions of the workload (paper's stopping rule), judged on 128 held-out mu:
    from the learned start the SQP reaches the default start's final merit in fewer iterations."""
    wl, s = c2
    nD = s.sizes.n_D
    s.options()
    mu_tr = inputs.mu_batch(512, seed=101)
    x_tr, _ = _solutions(s, mu_tr)
    lib.ddnm_ws_init(s.ctx, H, inputs.mlp_init(2, H, nD))
    losses = lib.ddnm_ws_train(s.ctx, mu_tr, x_tr, 150, 64, 2e-3, inputs.mlp_order(512, 150))
    assert losses[-1] < 0.2 * losses[0]
    mu_te = inputs.mu_batch(128, seed=202)
    lib.ddnm_ws_enable(s.ctx, False)
    _, st_plain = _solutions(s, mu_te)
    phi_plain = st_plain["merit"]
    lib.ddnm_ws_enable(s.ctx, True)
    reach = np.full(128, 99)
    for K in (1, 2, 3, 4, 6, 8, 11, 15):
        s.options(tol=0.0, max_iter=K)
        _, st = _solutions(s, mu_te)
        newly = (st["merit"] <= phi_plain) & (reach == 99)
        reach[newly] = K
    s.options()
    _, st_ws = _solutions(s, mu_te)
    lib.ddnm_ws_enable(s.ctx, False)
    reached = reach < 99
    assert reached.mean() > 0.5                            # most instances reach the plain final merit
    assert np.median(reach[reached]) < 15                  # ... in fewer than the plain 15 iterations
    assert np.median(st_ws["merit"]) < np.median(phi_plain)
    # checkpoint round trip: same predictions after save / load
    path = str(tmp_path / "ws.bin")
    x0a = lib.ddnm_ws_predict(s.ctx, mu_te[:8], nD)
    lib.ddnm_ws_save(s.ctx, path)
    lib.ddnm_ws_load(s.ctx, path)
    x0b = lib.ddnm_ws_predict(s.ctx, mu_te[:8], nD)
    assert np.array_equal(x0a, x0b)


def test_non_finite_prediction_falls_back(c2):
    wl, s = c2
    nD = s.sizes.n_D
    lib.ddnm_ws_init(s.ctx, H, inputs.mlp_init(2, H, nD))
    lib.ddnm_ws_set_norm(s.ctx, [1.0, 1.0], [0.1, 0.1], np.zeros(nD), np.full(nD, 1e300))
    x0 = lib.ddnm_ws_predict(s.ctx, inputs.mu_batch(4), nD)
    assert np.all(x0 == 0.0)                               # non-finite rows replaced by the default start
    lib.ddnm_ws_enable(s.ctx, True)
    s.options(tol=0.0, max_iter=2)
    mu = inputs.mu_batch(4)
    x, lam, st = s.solve(mu)
    lib.ddnm_ws_enable(s.ctx, False)
    x_ref, lam_ref, st_ref = s.solve(mu)
    assert np.allclose(x, x_ref) and np.all(st["flags"] & lib.DDNM_FLAG_WS_FALLBACK)
    s.options()
