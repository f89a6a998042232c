"""ddnm_residual_noalloc: the evaluation for callers that cannot allocate device memory (a memory
cap, a no-growth pool, or latency-critical code that must not allocate).  Its scratch is a static
device array shared by all calls; it is checked here against ddnm_residual on two calls in a row,
the second reusing the array that the first one filled.  Collected last (file name) so that a
run stopping at the first failure has already run every other test."""
import numpy as np
import pytest

import inputs
from oracle import setup

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)
lib = pytest.importorskip("paper_2305_15163_gb300")

TOL = {0: 1e-9, 1: 2e-5}     # the one-evaluation tolerances of the parity tests (FP64, mixed)


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("name,prec", [("c2", 1), ("tiny13x9_3x2", 0)])
def test_noalloc_matches_residual_two_calls(name, prec):
    wl = inputs.workload(name)
    fom, dd, rom, raw = setup.build(wl)
    s = lib.Solver(wl, precision=prec)
    s.load(raw["dec_o"], raw["dec_g"], raw["C"])
    nD, nC = s.sizes.n_D, s.sizes.n_C
    dev = torch.device("cuda:0")
    r = np.random.default_rng(21)
    B = 9
    calls = [(inputs.mu_batch(B, seed=5), 0.3 * r.standard_normal((B, nD)), r.standard_normal((B, nC))),
             (inputs.mu_batch(B, seed=6), 0.2 * r.standard_normal((B, nD)), None)]
    # one allocating call puts the tables on the device
    F_ref0, _ = s.residual(calls[0][0], calls[0][1], calls[0][2])
    refs = [F_ref0, s.residual(calls[1][0], calls[1][1], None)[0]]
    for (mu, x, lam), F_ref in zip(calls, refs):
        F_d = torch.full((B, nD + nC), float("nan"), dtype=torch.float64, device=dev)
        lib.ddnm_residual_noalloc(s.ctx, B, torch.from_numpy(mu).to(dev), torch.from_numpy(x).to(dev),
                                  None if lam is None else torch.from_numpy(lam).to(dev), F_d)
        torch.cuda.synchronize()
        F = F_d.cpu().numpy()
        for b in range(B):
            assert rel(F[b], F_ref[b]) < TOL[prec]
    s.close()


def test_noalloc_rejects_oversized_batch_and_missing_tables():
    wl = inputs.workload("c2")
    fom, dd, rom, raw = setup.build(wl)
    s = lib.Solver(wl)
    s.load(raw["dec_o"], raw["dec_g"], raw["C"])
    dev = torch.device("cuda:0")
    nD, nC = s.sizes.n_D, s.sizes.n_C
    big = 4096
    mu = torch.ones((big, 2), dtype=torch.float64, device=dev)
    x = torch.zeros((big, nD), dtype=torch.float64, device=dev)
    F = torch.zeros((big, nD + nC), dtype=torch.float64, device=dev)
    with pytest.raises(lib.DDNMError) as e:               # tables not uploaded yet
        lib.ddnm_residual_noalloc(s.ctx, 4, mu, x, None, F)
    assert e.value.code == lib.DDNM_E_STATE
    s.residual(inputs.mu_batch(1), np.zeros((1, nD)))
    with pytest.raises(lib.DDNMError) as e:               # beyond the 16 MiB static scratch
        lib.ddnm_residual_noalloc(s.ctx, big, mu, x, None, F)
    assert e.value.code == lib.DDNM_E_UNSUPPORTED and "16777216" in str(e.value)
    s.close()
