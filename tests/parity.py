"""Element-wise parity checks and a process pool for oracle solves (test helpers, no method arithmetic).

Every comparison is per block (one subdomain's H_i, D_i, rho_i, Z_i r_i, xh_i; the multipliers; Atil; the
reconstructed state) and per element inside a block:

    |gpu - ref| <= tol * |ref| + tol * max|ref over the block|

so that an entry that is small next to the rest of its block is still checked against the block's own scale,
not against the norm of a long concatenated vector.

``oracle_solves`` runs oracle solves in a ``spawn`` process pool (a pool forked after the first CUDA call can
hang), one single-threaded worker per host core; each worker builds the oracle for the workload once.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np


def close(gpu, ref, tol, what=""):
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert gpu.shape == ref.shape, f"{what}: shape {gpu.shape} vs {ref.shape}"
    if ref.size == 0:
        return
    scale = float(np.max(np.abs(ref)))
    err = np.abs(gpu - ref)
    bound = tol * np.abs(ref) + tol * scale
    bad = ~(err <= bound)
    if bad.any():
        k = int(np.argmax(np.where(bad, err / np.maximum(bound, 1e-300), 0.0)))
        raise AssertionError(f"{what}: {int(bad.sum())} of {ref.size} entries outside tol {tol:g} "
                             f"(worst index {k}: gpu {gpu.flat[k]!r}, ref {ref.flat[k]!r}, block max {scale:.3e})")


def split(vec, sizes):
    """Cut a concatenated vector into consecutive blocks of the given sizes."""
    vec = np.asarray(vec)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(int)
    assert off[-1] == vec.size, f"blocks of {off[-1]} entries in a vector of {vec.size}"
    return [vec[off[k]:off[k + 1]] for k in range(len(sizes))]


def evaluation(rom, ev, tol, H=None, D=None, A=None, F=None, rhr=None, what=""):
    """One evaluation's outputs (GPU layout of ddnm_linearize / ddnm_residual) against the oracle's
    Evaluation ``ev``, subdomain by subdomain."""
    n_sub = len(rom.n_i)
    if H is not None:
        for i, h in enumerate(split(H, [n * n for n in rom.n_i])):
            close(h.reshape(rom.n_i[i], rom.n_i[i]), ev.H[i], tol, f"{what} H_{i}")
    if D is not None:
        for i, d in enumerate(split(D, [rom.n_C * g for g in rom.nG])):
            close(d.reshape(rom.n_C, rom.nG[i]), ev.D[i], tol, f"{what} D_{i}")
    if A is not None:
        close(A, ev.Atil, tol, f"{what} Atil")
    if F is not None:
        parts = split(F, list(rom.n_i) + [rom.n_C])
        for i in range(n_sub):
            close(parts[i], ev.rho[i], tol, f"{what} rho_{i}")
        close(parts[-1], ev.Atil, tol, f"{what} F[Atil]")
    if rhr is not None:
        for i, r in enumerate(split(rhr, [len(rr) for rr in ev.r])):
            close(r, ev.r[i], tol, f"{what} Z_{i} r_{i}")


def latent(rom, x, ref_x, tol, what=""):
    """xh per subdomain block (interior and interface coordinates as separate blocks)."""
    for i, (xi, ri) in enumerate(zip(split(x, rom.n_i), split(ref_x, rom.n_i))):
        close(xi[:rom.nO[i]], ri[:rom.nO[i]], tol, f"{what} xh_{i}^O")
        close(xi[rom.nO[i]:], ri[rom.nO[i]:], tol, f"{what} xh_{i}^G")


def solve_result(rom, x, lam, st, ref, tol, what="", alpha_exact=True, merit_atol=0.0):
    """A GPU solve of one instance against the oracle's SolveResult: iteration count, status, flags and
    evaluation count exactly; xh per block, lambda and the merit element-wise; the last step length
    exactly (both sides halve from 1 in binary).  merit_atol: an absolute floor on the merit comparison for
    solves that end below the stopping tolerance, where the merit is a sum of rounding remainders."""
    assert int(st["iters"]) == ref.iters, f"{what}: iters {int(st['iters'])} vs {ref.iters}"
    assert int(st["status"]) == ref.status, f"{what}: status {int(st['status'])} vs {ref.status}"
    assert int(st["n_evals"]) == ref.n_evals, f"{what}: n_evals {int(st['n_evals'])} vs {ref.n_evals}"
    assert int(st["flags"]) & 1 == ref.flags & 1, f"{what}: LS_FAIL flag {int(st['flags'])} vs {ref.flags}"
    latent(rom, x, ref.x, tol, what)
    close(lam, ref.lam, tol, f"{what} lambda")
    dm = abs(float(st["merit"]) - ref.phi)
    assert dm <= 2.0 * tol * abs(ref.phi) + merit_atol, f"{what} merit: gpu {float(st['merit'])!r}, ref {ref.phi!r}"
    if alpha_exact and ref.alpha_hist:
        assert float(st["alpha_last"]) == ref.alpha_hist[-1], f"{what}: alpha {float(st['alpha_last'])}"


def rom_from_raw(name, raw, builder=None):
    """The oracle's DDROM of a workload with the decoders, HR rows and test matrix of ``raw``."""
    import inputs
    from oracle.burgers import Burgers
    from oracle.dd import decompose
    from oracle.decoders import MaskedDecoder
    from oracle.rom import DDROM
    wl = builder() if builder is not None else inputs.workload(name)
    fom = Burgers(wl.nx, wl.ny, wl.nu)
    dd = decompose(wl.nx, wl.ny, wl.xb, wl.yb)
    return DDROM(fom, dd, [MaskedDecoder(d) for d in raw["dec_o"]], [MaskedDecoder(d) for d in raw["dec_g"]],
                 raw["hr"], raw["C"])


# ------------------------------------------------------------------ oracle solves in a spawn pool

_ROM = None


def _init(name, builder, raw=None):
    global _ROM
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    import inputs
    from oracle import setup
    wl = builder() if builder is not None else inputs.workload(name)
    _ROM = setup.build(wl)[2] if raw is None else rom_from_raw(name, raw, builder)


def _solve(job):
    mu, kw = job
    return _ROM.solve(mu, **kw)


_THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def _pool(workers, n_jobs, init=None, initargs=()):
    """A spawn pool of single-threaded workers.  The BLAS thread counts are set in this process's environment
    while the workers start (a worker imports numpy before its initializer runs, so setting them there is too
    late: every worker would start one BLAS thread per core)."""
    workers = max(1, min(workers or (os.cpu_count() or 1), 16, n_jobs))
    old = {k: os.environ.get(k) for k in _THREAD_VARS}
    os.environ.update({k: "1" for k in _THREAD_VARS})
    try:
        return mp.get_context("spawn").Pool(workers, initializer=init, initargs=initargs)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def oracle_solves(name, mu, workers=None, builder=None, raw=None, **kw):
    """rom.solve(mu[b], **kw) for every row of mu, in a spawn pool (builder: a picklable callable that
    returns the Workload, for cases that are not a named workload; raw: decoder specs, HR rows and C to use
    instead of the seeded random-init ones)."""
    mu = np.asarray(mu, dtype=np.float64).reshape(-1, 2)
    with _pool(workers, len(mu), _init, (name, builder, raw)) as pool:
        return pool.map(_solve, [(m, kw) for m in mu], chunksize=1)


def _fom_solve(job):
    name, m = job
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    import inputs
    from oracle.burgers import Burgers
    wl = inputs.workload(name)
    fom = Burgers(wl.nx, wl.ny, wl.nu)
    return fom.newton(m, x0=fom.exact_state(m))[0]


def oracle_fom(name, mu, workers=None):
    """The oracle's FOM solutions (Newton from the exact solution at the nodes) at every row of mu."""
    mu = np.asarray(mu, dtype=np.float64).reshape(-1, 2)
    with _pool(workers, len(mu)) as pool:
        return np.array(pool.map(_fom_solve, [(name, m) for m in mu], chunksize=1))


def _train_one(job):
    name, i, kind, Xs, epochs, batch, lr = job
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    import inputs
    from oracle import setup
    ae = setup.train_autoencoder(inputs.workload(name), i, kind, Xs, epochs, batch, lr)
    return ae.decoder_spec(), ae.losses


def oracle_trained(name, n_side, epochs, batch, lr, workers=None):
    """The workload with decoders the oracle trains (oracle.setup.train_autoencoders, one autoencoder per
    pool worker) on its own FOM snapshots at an n_side x n_side grid of mu: returns raw (dec_o, dec_g, hr,
    C, snapshots X, losses)."""
    import inputs
    from oracle.dd import decompose
    wl = inputs.workload(name)
    dd = decompose(wl.nx, wl.ny, wl.xb, wl.yb)
    X = oracle_fom(name, inputs.snapshot_mu(n_side), workers)
    jobs = [(name, i, kind, X[:, ids], epochs, batch, lr)
            for i, sd in enumerate(dd.subs) for kind, ids in ((0, sd.interior), (1, sd.interface))]
    with _pool(workers, len(jobs)) as pool:
        out = pool.map(_train_one, jobs, chunksize=1)
    dec_o = [out[2 * i][0] for i in range(wl.n_sub)]
    dec_g = [out[2 * i + 1][0] for i in range(wl.n_sub)]
    return dict(dec_o=dec_o, dec_g=dec_g, hr=inputs.hr_sets(wl),
                C=inputs.test_matrix(wl.n_c(), dd.N_A, inputs.SEED_C + wl.seed_offset), snapshots=X,
                losses=np.array([o[1] for o in out]).T)
