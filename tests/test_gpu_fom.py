"""The batched GPU FOM solve (ddnm_fom_solve: Newton with preconditioned BiCGSTAB on the steady Burgers system
of Sec. 7.1, Eq. burgers_discretized) against the oracle's sparse-LU Newton on the same grids and parameters.

Both stop at the FP64 rounding floor of the residual, so the two solutions agree to ~1e-12 of the state;
the test bound is 1e-9 per component block (u, v) and element.  At 1024 x 1024, where the oracle's LU would
take too long, the GPU solution is checked through the oracle's residual instead: r(x) at the returned state
must be at the rounding floor of r's own terms."""
import numpy as np
import pytest

import inputs
import parity
from oracle.burgers import Burgers

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)
lib = pytest.importorskip("paper_2305_15163_gb300")

TOL = 1e-9


def ctx_for(name):
    wl = inputs.workload(name)
    return wl, lib.Solver(wl)


def check_state(fom, x, ref, what):
    N = fom.N
    parity.close(x[:N], ref[:N], TOL, f"{what} u")
    parity.close(x[N:], ref[N:], TOL, f"{what} v")


@pytest.mark.parametrize("name,B", [("tiny12x10_2x2", 3), ("tiny13x9_3x2", 2), ("c1", 4), ("c2", 4)])
def test_fom_matches_oracle_newton(name, B):
    wl, s = ctx_for(name)
    fom = Burgers(wl.nx, wl.ny, wl.nu)
    mu = inputs.mu_batch(B, seed=17)
    x, st = lib.ddnm_fom_solve(s.ctx, mu)
    assert np.all(st["status"] == 0) and np.all(st["newton_iters"] >= 1)
    for b in range(B):
        ref, hist = fom.newton(mu[b], x0=fom.exact_state(mu[b]))
        check_state(fom, x[b], ref, f"{name} instance {b}")
        assert abs(st[b]["res0"] - hist[0]) <= 1e-9 * hist[0]
    s.close()


def test_fom_from_zero_start():
    """From x0 = 0 (far from the solution: the residual starts at the size of the boundary data's stencil
    terms) Newton takes more steps and reaches the same solution as the oracle's Newton from 0."""
    wl, s = ctx_for("c1")
    fom = Burgers(wl.nx, wl.ny, wl.nu)
    mu = inputs.mu_batch(2, seed=3)
    x, st = lib.ddnm_fom_solve(s.ctx, mu, x0=np.zeros((2, 2 * fom.N)))
    assert np.all(st["status"] == 0) and np.all(st["newton_iters"] >= 3)
    for b in range(2):
        ref, _ = fom.newton(mu[b])
        check_state(fom, x[b], ref, f"zero start instance {b}")
    s.close()


def test_fom_256_and_device_memory():
    """256 x 256 (the uneven workload's grid) against the oracle, the inputs and outputs in device memory."""
    wl, s = ctx_for("c3")
    fom = Burgers(wl.nx, wl.ny, wl.nu)
    mu = inputs.mu_batch(2, seed=23)
    dev = torch.device("cuda:0")
    mu_d = torch.from_numpy(mu).to(dev)
    x_d = torch.zeros((2, 2 * fom.N), dtype=torch.float64, device=dev)
    _, st = lib.ddnm_fom_solve(s.ctx, mu_d, x_out=x_d)
    torch.cuda.synchronize()
    x = x_d.cpu().numpy()
    assert np.all(st["status"] == 0)
    x_h, _ = lib.ddnm_fom_solve(s.ctx, mu)
    assert np.array_equal(x, x_h)
    for b in range(2):
        ref, _ = fom.newton(mu[b], x0=fom.exact_state(mu[b]))
        check_state(fom, x[b], ref, f"256x256 instance {b}")
    s.close()


def test_fom_1024_residual_at_rounding_floor():
    """The 1024 x 1024 grid: the oracle's residual r(x) at the GPU solution is at the rounding floor of the
    residual's terms (|r_k| <= 1e-11 times the largest stencil term), and it is far below the discretisation
    error (the exact solution at the nodes leaves a residual orders of magnitude larger)."""
    wl, s = ctx_for("c5")
    fom = Burgers(wl.nx, wl.ny, wl.nu)
    mu = inputs.mu_batch(2, seed=29)
    x, st = lib.ddnm_fom_solve(s.ctx, mu)
    assert np.all(st["status"] == 0)
    for b in range(2):
        r = fom.residual(x[b], mu[b])
        r_ex = fom.residual(fom.exact_state(mu[b]), mu[b])
        # largest stencil term: the diffusion coefficients 2 nu (1/h_x^2 + 1/h_y^2) times the largest state
        scale = 2.0 * fom.nu * (1.0 / fom.hx ** 2 + 1.0 / fom.hy ** 2) * np.abs(x[b]).max()
        assert np.abs(r).max() <= 1e-11 * scale
        assert np.linalg.norm(r) < 1e-4 * np.linalg.norm(r_ex)
        assert abs(st[b]["res"] - np.linalg.norm(r)) <= 1e-3 * np.linalg.norm(r_ex)
    s.close()
