"""ddnm_hr_select (host code of the library: residual POD basis, greedy sample rows, gappy projector; Sec. 3.1,
Sec. 5.3 greedy remark) against the oracle's gappy_hr on the same residual snapshots (the oracle's Newton
history).  The rows are integer results and must be identical; the projectors (Z Phi)^+ are compared through
P^T P, which does not depend on the sign or rotation of the basis vectors (the two sides compute the basis by
different routes), at 1e-9 of its largest entry.  No device is needed."""
import numpy as np
import pytest

import inputs
from oracle.burgers import Burgers
from oracle.dd import decompose
from oracle.hr import gappy_hr, residual_snapshots

lib = pytest.importorskip("paper_2305_15163_gb300")


@pytest.mark.parametrize("name,side,nr", [("tiny12x10_2x2", 2, 4), ("c1", 3, 8), ("tiny13x9_3x2", 2, 5)])
def test_library_selection_matches_oracle(name, side, nr):
    wl = inputs.workload(name)
    fom = Burgers(wl.nx, wl.ny, wl.nu)
    dd = decompose(wl.nx, wl.ny, wl.xb, wl.yb)
    S = residual_snapshots(fom, inputs.snapshot_mu(side))
    n_s = [len(h) for h in inputs.hr_sets(wl)]
    rows_o, proj_o = gappy_hr(fom, dd, S, n_s, nu_tol=1e-14, max_nr=nr)
    assert all(p.shape[0] == nr for p in proj_o)
    s = lib.Solver(wl)
    rows_l, proj_l = lib.ddnm_hr_select(s.ctx, S, [nr] * wl.n_sub, n_s)
    for i in range(wl.n_sub):
        assert np.array_equal(rows_l[i], rows_o[i]), f"subdomain {i} rows"
        Gl, Go = proj_l[i].T @ proj_l[i], proj_o[i].T @ proj_o[i]
        assert np.allclose(Gl, Go, rtol=0, atol=1e-9 * np.abs(Go).max()), f"subdomain {i} projector"
    s.close()


def test_selection_rejects_bad_sizes():
    wl = inputs.workload("tiny12x10_2x2")
    fom = Burgers(wl.nx, wl.ny, wl.nu)
    S = residual_snapshots(fom, inputs.snapshot_mu(2))
    s = lib.Solver(wl)
    n_s = [len(h) for h in inputs.hr_sets(wl)]
    for nr, ns in (([0] * 4, n_s), ([65] * 4, n_s), ([4] * 4, [3] * 4), ([4] * 4, [10 ** 6] * 4)):
        with pytest.raises(lib.DDNMError) as e:
            lib.ddnm_hr_select(s.ctx, S, nr, ns)
        assert e.value.code == lib.DDNM_E_INVALID
    s.close()
