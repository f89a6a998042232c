"""ddnm_residual_noalloc: the evaluation for callers that cannot allocate device memory (a memory
cap, a no-growth pool, or latency-critical code that must not allocate).  Its scratch is a static
device array shared by all calls.  It is checked here against ddnm_residual and against the oracle on
two calls in a row, the second reusing the array that the first one filled, with D_i formed inside the
evaluation and by the batched GEMM (whose P_G also lives in the array), at a batch just under the array's
capacity, and with the device's free memory unchanged across the call.  Collected last (file name) so
that a run stopping at the first failure has already run every other test."""
import re

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

TOL = {0: 1e-9, 1: 2e-5}     # the one-evaluation tolerances of the parity tests (FP64, mixed)
DEV = torch.device("cuda:0")


def solver(name, prec, d_gemm):
    wl = inputs.workload(name)
    fom, dd, rom, raw = setup.build(wl)
    s = lib.Solver(wl, precision=prec)
    s.load(raw["dec_o"], raw["dec_g"], raw["C"])
    lib.ddnm_set_tune(s.ctx, d_gemm=d_gemm)
    return wl, rom, s


def noalloc(s, mu, x, lam):
    B = mu.shape[0]
    F_d = torch.full((B, s.sizes.n_D + s.sizes.n_C), float("nan"), dtype=torch.float64, device=DEV)
    args = [torch.from_numpy(mu).to(DEV), torch.from_numpy(x).to(DEV),
            None if lam is None else torch.from_numpy(lam).to(DEV)]
    torch.cuda.synchronize()
    alloc0, res0 = torch.cuda.memory_allocated(), torch.cuda.memory_reserved()
    free0 = torch.cuda.mem_get_info()[0]
    lib.ddnm_residual_noalloc(s.ctx, B, *args, F_d)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert torch.cuda.memory_allocated() == alloc0 and torch.cuda.memory_reserved() == res0
    return F_d.cpu().numpy(), free1 - free0


@pytest.mark.parametrize("d_gemm", [0, 1])
@pytest.mark.parametrize("name,prec", [("c2", 1), ("tiny13x9_3x2", 0)])
def test_noalloc_matches_residual_and_oracle_two_calls(name, prec, d_gemm):
    wl, rom, s = solver(name, prec, d_gemm)
    nD, nC = s.sizes.n_D, s.sizes.n_C
    r = np.random.default_rng(21)
    B = 9
    calls = [(inputs.mu_batch(B, seed=5), 0.3 * r.standard_normal((B, nD)), r.standard_normal((B, nC))),
             (inputs.mu_batch(B, seed=6), 0.2 * r.standard_normal((B, nD)), None)]
    # one allocating call puts the tables on the device
    refs = [s.residual(mu, x, lam)[0] for mu, x, lam in calls]
    freed = []
    for k, ((mu, x, lam), F_ref) in enumerate(zip(calls, refs)):
        F, dfree = noalloc(s, mu, x, lam)
        freed.append(dfree)
        for b in range(B):
            parity.close(F[b], F_ref[b], TOL[prec], f"call {k} instance {b} vs ddnm_residual")
            ev = rom.evaluate(x[b], np.zeros(nC) if lam is None else lam[b], mu[b])
            parity.evaluation(rom, ev, TOL[prec], F=F[b], what=f"call {k} instance {b} vs oracle")
    # the second call loads nothing new: the device's free memory does not move across it
    assert freed[1] == 0
    s.close()


def test_noalloc_batch_just_under_capacity():
    wl, rom, s = solver("c2", 1, -1)
    nD, nC = s.sizes.n_D, s.sizes.n_C
    s.residual(inputs.mu_batch(1), np.zeros((1, nD)))
    big = 4096
    with pytest.raises(lib.DDNMError) as e:
        lib.ddnm_residual_noalloc(s.ctx, big, torch.ones((big, 2), dtype=torch.float64, device=DEV),
                                  torch.zeros((big, nD), dtype=torch.float64, device=DEV), None,
                                  torch.zeros((big, nD + nC), dtype=torch.float64, device=DEV))
    cap = int(re.search(r"about (\d+) instances", str(e.value)).group(1))
    assert 16 < cap < big
    B = cap - 1
    r = np.random.default_rng(8)
    mu = inputs.mu_batch(B, seed=12)
    x = 0.3 * r.standard_normal((B, nD))
    lam = r.standard_normal((B, nC))
    F_ref = s.residual(mu, x, lam)[0]
    F, _ = noalloc(s, mu, x, lam)
    for b in range(B):
        parity.close(F[b], F_ref[b], TOL[1], f"B = {B} instance {b}")
    s.close()


def test_noalloc_rejects_bad_calls():
    wl, rom, s = solver("c2", 1, -1)
    nD, nC = s.sizes.n_D, s.sizes.n_C
    B = 4
    mu = torch.ones((B, 2), dtype=torch.float64, device=DEV)
    x = torch.zeros((B, nD), dtype=torch.float64, device=DEV)
    F = torch.zeros((B, nD + nC), dtype=torch.float64, device=DEV)
    with pytest.raises(lib.DDNMError) as e:               # tables not uploaded yet
        lib.ddnm_residual_noalloc(s.ctx, B, mu, x, None, F)
    assert e.value.code == lib.DDNM_E_STATE
    s.residual(inputs.mu_batch(1), np.zeros((1, nD)))
    big = 4096
    with pytest.raises(lib.DDNMError) as e:               # beyond the 16 MiB static scratch
        lib.ddnm_residual_noalloc(s.ctx, big, torch.ones((big, 2), dtype=torch.float64, device=DEV),
                                  torch.zeros((big, nD), dtype=torch.float64, device=DEV), None,
                                  torch.zeros((big, nD + nC), dtype=torch.float64, device=DEV))
    assert e.value.code == lib.DDNM_E_UNSUPPORTED and "16777216" in str(e.value)
    with pytest.raises(TypeError):                         # host arrays are refused by the binding
        lib.ddnm_residual_noalloc(s.ctx, B, np.ones((B, 2)), x, None, F)
    with pytest.raises(ValueError):                        # wrong dtype / shape
        lib.ddnm_residual_noalloc(s.ctx, B, mu.float(), x, None, F)
    with pytest.raises(ValueError):
        lib.ddnm_residual_noalloc(s.ctx, B, mu, x[:, :-1].contiguous(), None, F)
    # the C entry point itself refuses a host pointer before queueing any work
    host_mu = np.ones((B, 2))
    rc = lib._lib.ddnm_residual_noalloc(s.ctx, B, host_mu.ctypes.data, x.data_ptr(), None, F.data_ptr(),
                                        torch.cuda.current_stream().cuda_stream)
    assert rc == lib.DDNM_E_INVALID and "device memory" in lib.ddnm_last_error(s.ctx)
    s.close()
