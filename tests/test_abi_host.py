"""The C-ABI library loads, exports every declared symbol, and its host-side DD set-up
(index maps, constraint rows, sizes) matches the oracle bit for bit.  No GPU needed."""
import ctypes
import os
import re

import numpy as np
import pytest

import inputs
from oracle.dd import decompose

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
lib = pytest.importorskip("paper_2305_15163_gb300")


def test_exports_every_declared_symbol():
    with open(os.path.join(ROOT, "include", "ddnm.h")) as f:
        src = f.read()
    declared = set(re.findall(r"^\s*(?:int|void|const char\*)\s+(ddnm_\w+)\s*\(", src, re.M))
    assert {"ddnm_setup", "ddnm_load_decoders", "ddnm_solve_batch", "ddnm_residual"} <= declared
    so = ctypes.CDLL(lib.LIB_PATH)
    for name in declared:
        assert hasattr(so, name), name
    assert declared <= set(lib.EXPORTED)


@pytest.mark.parametrize("name", ["c1", "c2", "c3", "tiny12x10_2x2", "tiny13x9_3x2"])
def test_decomposition_matches_oracle(name):
    wl = inputs.workload(name)
    s = lib.Solver(wl)
    dd = decompose(wl.nx, wl.ny, wl.xb, wl.yb)
    assert s.sizes.n_sub == dd.n_sub and s.sizes.N_A == dd.N_A and s.sizes.N_x == 2 * wl.nx * wl.ny
    assert s.sizes.n_D == sum(wl.n_omega) + sum(wl.n_gamma) and s.sizes.n_C == wl.n_c()
    for i, sd in enumerate(dd.subs):
        info = s.subs[i]
        assert np.array_equal(info["interior"], sd.interior)
        assert np.array_equal(info["interface"], sd.interface)
        assert info["N_r"] == sd.res_rows.size and info["N_B"] == len(s.hr[i])
    var, lo, hi = lib.ddnm_get_constraints(s.ctx)
    assert np.array_equal(var, dd.row_var)
    assert np.array_equal(np.stack([lo, hi], 1), dd.row_pair)
    s.close()


def test_setup_rejects_bad_input():
    wl = inputs.workload("tiny12x10_2x2")
    hr = inputs.hr_sets(wl)
    args = dict(nx=12, ny=10, xb=[0, 6, 12], yb=[0, 5, 10], n_omega=[3] * 4, n_gamma=[2] * 4,
                hr_count=[len(h) for h in hr], hr_rows=np.concatenate(hr), n_c=4)
    ctx = lib.ddnm_setup(**args)
    lib.ddnm_destroy(ctx)
    bad = [dict(xb=[0, 6, 11]), dict(xb=[0, 12]  + [12]), dict(n_c=0), dict(n_c=1000),
           dict(n_omega=[0] * 4), dict(n_omega=[12] * 4, n_gamma=[5] * 4), dict(hr_count=[2] * 4),
           dict(hr_rows=np.concatenate([h[::-1] for h in hr])), dict(xb=[0, 12], yb=[0, 10])]
    for b in bad:
        a = dict(args)
        a.update(b)
        if "xb" in b and "yb" not in b and len(b["xb"]) == 3 and b["xb"][-1] == 12 and b["xb"][1] == 12:
            continue
        with pytest.raises(lib.DDNMError) as e:
            lib.ddnm_setup(**a)
        assert e.value.code in (lib.DDNM_E_INVALID, lib.DDNM_E_UNSUPPORTED)
        assert "ddnm_setup" in lib.ddnm_last_error(None)


def test_call_order_and_decoder_validation():
    wl = inputs.workload("tiny12x10_2x2")
    s = lib.Solver(wl)
    # solve before decoders / C are loaded: a state error, detected before any device work
    with pytest.raises(lib.DDNMError) as e:
        s.solve(inputs.mu_batch(1))
    assert e.value.code == lib.DDNM_E_STATE
    dd = decompose(wl.nx, wl.ny, wl.xb, wl.yb)
    dec_o, dec_g = inputs.decoders_for(wl, [x.interior for x in dd.subs], [x.interface for x in dd.subs])
    bad = dict(dec_o[0])
    bad["N"] = bad["N"] + 1
    with pytest.raises(lib.DDNMError) as e:
        lib.ddnm_load_decoders(s.ctx, 0, lib.DDNM_DECODER_INTERIOR, bad)
    assert e.value.code == lib.DDNM_E_INVALID
    bad = dict(dec_o[0])
    cols = bad["cols"].copy()
    cols[3, 0] = bad["w"]
    bad["cols"] = cols
    with pytest.raises(lib.DDNMError):
        lib.ddnm_load_decoders(s.ctx, 0, lib.DDNM_DECODER_INTERIOR, bad)
    with pytest.raises(lib.DDNMError):
        lib.ddnm_set_options(s.ctx, beta=1.5)
    s.close()


def test_launch_plan_validation():
    """ddnm_set_tune / ddnm_get_tune are host bookkeeping: defaults, a valid plan, and every bound."""
    wl = inputs.workload("tiny12x10_2x2")
    s = lib.Solver(wl)
    assert lib.ddnm_get_tune(s.ctx) == {"graph": 1, "chains": 1, "con_split": 512, "eval_persist": 0, "d_gemm": -1,
                                        "eval_groups": 1, "atil": -1}
    lib.ddnm_set_tune(s.ctx, graph=0, chains=64, con_split=2048, eval_persist=8, d_gemm=1, eval_groups=0, atil=1)
    assert lib.ddnm_get_tune(s.ctx) == {"graph": 0, "chains": 64, "con_split": 2048, "eval_persist": 8, "d_gemm": 1,
                                        "eval_groups": 0, "atil": 1}
    good = dict(graph=1, chains=2, con_split=1024, eval_persist=1, d_gemm=0, eval_groups=0, atil=0)
    for bad in (dict(graph=2), dict(graph=-1), dict(chains=0), dict(chains=65), dict(con_split=256),
                dict(con_split=768), dict(con_split=4096), dict(eval_persist=-1), dict(eval_persist=9),
                dict(d_gemm=3), dict(d_gemm=-2), dict(eval_groups=2), dict(eval_groups=-1), dict(atil=2),
                dict(atil=-2)):
        with pytest.raises(lib.DDNMError) as e:
            lib.ddnm_set_tune(s.ctx, **{**good, **bad})
        assert e.value.code == lib.DDNM_E_INVALID
    assert lib.ddnm_get_tune(s.ctx)["chains"] == 64      # a rejected plan leaves the old one
    s.close()
