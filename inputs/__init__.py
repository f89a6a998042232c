"""Seeded synthetic inputs for the DD NM-ROM-HR solve.

This module is shared by the FP64 oracle (``oracle/``) and the CUDA path
(``paper_2305_15163_gb300``).  It holds *only* random draws and the fixed
workload tables; none of the method's arithmetic (residual, decoders,
constraints, SQP) lives here.  Everything the method derives from the grid
(interior/interface index sets, constraint rows, their counts) is computed
independently by each side and handed back here as plain sizes when a draw
needs them (e.g. the Gaussian test matrix needs ``N_A``).

Workloads follow the paper's 2D steady Burgers test (Sec. 7.1) on
``[-1,1]^2`` with ``mu = (a, lambda) in [0.9, 1.1]^2``:

* ``c1``  32x32 grid, 2x2 subdomains, latent (4,2), width 64, HR 15 %, B = 1, FP64
* ``c2``  128x128 grid, 4x4 subdomains, latent (6,3), width 256, HR 5 %, B = 64
* ``c3``  256x256 grid, 3x5 uneven subdomains (Dirichlet widths), latent 4..10,
          width 128..512, HR 2..8 %, B = 256
* ``c5``  1024x1024 grid, 8x8 subdomains, latent (8,4), width 1024, HR 2 %, B = 1024

Decoders are random-init sparse-masked shallow networks (Sec. 5.1, Eq.
``autoencoder_architecture``) with the three-band mask of Sec. 7.3 and the
de-normalisation layer of Sec. 7.3 (snapshot min/max).  Trained weights are
not available, so the de-normalisation statistics are taken from the closed
form exact solution (Eq. ``burgers_pde_exact_solution``) sampled on a 4x4
grid of ``mu`` -- the continuum stand-in for the paper's FOM snapshots.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_GRID, SEED_HR, SEED_C, SEED_DEC, SEED_MU, SEED_MLP = 0, 1, 2, 3, 4, 5
MU_LO, MU_HI = 0.9, 1.1

# stream tags, so that each draw has its own independent generator
_TAG = {"grid": 11, "hr": 12, "C": 13, "dec": 14, "mu": 15, "mlp": 16, "lat": 17, "enc": 18, "ae": 19}


def rng(kind: str, *key: int) -> np.random.Generator:
    """Independent PCG64 stream for one purpose (platform independent)."""
    return np.random.default_rng(np.random.SeedSequence([_TAG[kind], *[int(k) for k in key]]))


@dataclass
class Workload:
    """Shape of one synthetic workload (no derived DD quantities)."""

    name: str
    nx: int
    ny: int
    kx: int
    ky: int
    xb: list[int]                 # kx+1 node breakpoints in [0, nx]
    yb: list[int]                 # ky+1 node breakpoints in [0, ny]
    n_omega: list[int]            # per subdomain interior latent dim
    n_gamma: list[int]            # per subdomain interface latent dim
    width: list[int]              # per subdomain decoder width (both decoders)
    hr_frac: list[float]          # per subdomain fraction of residual rows sampled
    band: int = 8                 # nonzeros per band of the decoder mask
    batch: int = 1                # number of mu instances in one launch
    nu: float = 0.1
    mixed: bool = True            # FP32 evaluation / FP64 KKT when True
    seed_offset: int = 0
    extras: dict = field(default_factory=dict)

    @property
    def n_sub(self) -> int:
        return self.kx * self.ky

    def owned_counts(self) -> list[int]:
        """Owned node count of each subdomain (x fastest subdomain order)."""
        return [(self.xb[sx + 1] - self.xb[sx]) * (self.yb[sy + 1] - self.yb[sy])
                for sy in range(self.ky) for sx in range(self.kx)]

    def residual_rows(self) -> list[int]:
        return [2 * c for c in self.owned_counts()]

    def hr_counts(self) -> list[int]:
        return [int(math.ceil(f * nr - 1e-12)) for f, nr in zip(self.hr_frac, self.residual_rows())]

    def n_c(self) -> int:
        return int(math.ceil(0.5 * sum(self.n_gamma)))


def equal_breaks(n: int, k: int) -> list[int]:
    return [(n * s) // k for s in range(k + 1)]


def dirichlet_breaks(n: int, k: int, min_width: int, r: np.random.Generator) -> list[int]:
    """Uneven split of n nodes into k pieces, each at least min_width wide."""
    w = r.dirichlet(np.ones(k))
    free = n - k * min_width
    widths = [min_width + int(round(wi * free)) for wi in w[:-1]]
    widths.append(n - sum(widths))
    if widths[-1] < min_width:            # rounding pushed the last piece too small
        deficit = min_width - widths[-1]
        j = int(np.argmax(widths[:-1]))
        widths[j] -= deficit
        widths[-1] += deficit
    b = [0]
    for wd in widths:
        b.append(b[-1] + wd)
    return b


def workload(name: str) -> Workload:
    """The seeded synthetic workloads (see module docstring)."""
    if name == "c1":
        return Workload("c1", 32, 32, 2, 2, equal_breaks(32, 2), equal_breaks(32, 2),
                        [4] * 4, [2] * 4, [64] * 4, [0.15] * 4, band=8, batch=1, mixed=False)
    if name == "c2":
        return Workload("c2", 128, 128, 4, 4, equal_breaks(128, 4), equal_breaks(128, 4),
                        [6] * 16, [3] * 16, [256] * 16, [0.05] * 16, band=8, batch=64)
    if name == "c3":
        r = rng("grid", SEED_GRID)
        xb = dirichlet_breaks(256, 3, 8, r)
        yb = dirichlet_breaks(256, 5, 8, r)
        n = 15
        rl = rng("lat", SEED_GRID)
        lat = [int(v) for v in rl.integers(4, 11, size=n)]
        wid = [32 * int(v) for v in rl.integers(4, 17, size=n)]
        frac = [float(v) for v in rl.uniform(0.02, 0.08, size=n)]
        return Workload("c3", 256, 256, 3, 5, xb, yb, lat, [int(math.ceil(l / 2)) for l in lat],
                        wid, frac, band=8, batch=256)
    if name == "c5":
        return Workload("c5", 1024, 1024, 8, 8, equal_breaks(1024, 8), equal_breaks(1024, 8),
                        [8] * 64, [4] * 64, [1024] * 64, [0.02] * 64, band=8, batch=1024)
    if name.startswith("tiny"):
        # small cases for tests: tiny<nx>x<ny>_<kx>x<ky>
        g, s = name[4:].split("_")
        nx, ny = (int(v) for v in g.split("x"))
        kx, ky = (int(v) for v in s.split("x"))
        k = kx * ky
        return Workload(name, nx, ny, kx, ky, equal_breaks(nx, kx), equal_breaks(ny, ky),
                        [3] * k, [2] * k, [24] * k, [0.4] * k, band=4, batch=2, mixed=False)
    raise KeyError(name)


# ----------------------------------------------------------------------------- draws

def mu_batch(B: int, seed: int = SEED_MU) -> np.ndarray:
    """B parameter instances mu = (a, lambda), uniform in [0.9, 1.1]^2, shape (B, 2)."""
    return rng("mu", seed).uniform(MU_LO, MU_HI, size=(B, 2))


def hr_rows(n_rows: int, n_sample: int, sub: int, seed: int = SEED_HR) -> np.ndarray:
    """Collocation rows of one subdomain: n_sample distinct local residual-row ids
    drawn uniformly without replacement, sorted ascending (int32)."""
    if n_sample > n_rows:
        raise ValueError("more HR rows than residual rows")
    r = rng("hr", seed, sub)
    return np.sort(r.choice(n_rows, size=n_sample, replace=False)).astype(np.int32)


def test_matrix(n_c: int, n_a: int, seed: int = SEED_C) -> np.ndarray:
    """Gaussian test matrix C (n_c x n_a, row-major FP64), entries N(0,1)/sqrt(n_a)."""
    return rng("C", seed).standard_normal((n_c, n_a)) / math.sqrt(max(n_a, 1))


def band_mask(n_out: int, width: int, nnz_band: int) -> np.ndarray:
    """Three-band decoder output mask (Sec. 7.3), as ELL column ids (n_out x 3*nnz_band, -1 pad).

    Row r has three bands of ``nnz_band`` contiguous columns; the centre band starts at
    floor(r * width / n_out) (so the band shifts right with r), and the outer bands sit
    ``nnz_band * shift`` columns to the left and right of it, shift = max(1, floor(width/n_out)).
    Columns outside [0, width) are dropped.
    """
    shift = max(1, width // n_out)
    sep = nnz_band * shift
    r = np.arange(n_out, dtype=np.int64)[:, None]
    c0 = (r * width) // n_out
    offs = np.concatenate([np.arange(nnz_band) - sep, np.arange(nnz_band), np.arange(nnz_band) + sep])
    cols = c0 + offs[None, :]
    ok = (cols >= 0) & (cols < width)
    # compact the valid columns of every row to the front, keeping their ascending order
    order = np.argsort(~ok, axis=1, kind="stable")
    out = np.take_along_axis(cols, order, axis=1).astype(np.int32)
    out[~np.take_along_axis(ok, order, axis=1)] = -1
    return out


def decoder(n_out: int, width: int, n_lat: int, nnz_band: int, key: tuple,
            offset: np.ndarray | None = None, scale: np.ndarray | None = None,
            act: str = "swish", seed: int = SEED_DEC) -> dict:
    """Random-init sparse-masked shallow decoder  g(x) = offset + scale * (W2 act(W1 x + b1)).

    W1 ~ N(0, 1/n_lat), b1 ~ N(0, 1/n_lat), W2 (masked) ~ N(0, 1/nnz_row)  (fan-in scaling).
    Returned as a dict of FP64 arrays; W2 in ELL form (cols int32 with -1 padding, vals).
    """
    r = rng("dec", seed, *key)
    W1 = r.standard_normal((width, n_lat)) / math.sqrt(n_lat)
    b1 = r.standard_normal(width) / math.sqrt(n_lat)
    cols = band_mask(n_out, width, nnz_band)
    nnz_row = (cols >= 0).sum(axis=1)
    vals = r.standard_normal(cols.shape) / np.sqrt(np.maximum(nnz_row, 1))[:, None]
    vals[cols < 0] = 0.0
    if offset is None:
        offset = np.zeros(n_out)
    if scale is None:
        scale = np.ones(n_out)
    return dict(N=n_out, w=width, n=n_lat, act=act, W1=W1, b1=b1, cols=cols, vals=vals,
                offset=np.asarray(offset, dtype=np.float64), scale=np.asarray(scale, dtype=np.float64))


# ------------------------------------------------------------ de-normalisation statistics

def _uv_exact(x, y, a, lam, nu):
    # closed-form exact solution of the steady 2D Burgers equation (Sec. 7.1)
    ep = np.exp(lam * (x - 1.0))
    em = np.exp(-lam * (x - 1.0))
    psi = a * (1.0 + x) + (ep + em) * np.cos(lam * y)
    u = -2.0 * nu * (a + lam * (ep - em) * np.cos(lam * y)) / psi
    v = 2.0 * nu * (lam * (ep + em) * np.sin(lam * y)) / psi
    return u, v


def denormalisation(var_ids: np.ndarray, nx: int, ny: int, nu: float = 0.1,
                    n_grid: int = 4, box=(-1.0, 1.0, -1.0, 1.0)) -> tuple[np.ndarray, np.ndarray]:
    """(offset, scale) of the de-normalisation layer for the outputs ``var_ids``.

    ``var_ids`` are global state ids in the ordering x = [u; v], each block x-fastest
    (u at node p is id p, v at node p is id nx*ny + p).  offset = (max+min)/2 and
    scale = (max-min)/2 over the exact solution sampled at an n_grid x n_grid grid of mu,
    i.e. the affine map that takes [-1, 1] onto the sampled range.
    """
    N = nx * ny
    var_ids = np.asarray(var_ids, dtype=np.int64)
    node = var_ids % N
    comp_v = var_ids >= N
    hx = (box[1] - box[0]) / (nx + 1)
    hy = (box[3] - box[2]) / (ny + 1)
    x = box[0] + (node % nx + 1) * hx
    y = box[2] + (node // nx + 1) * hy
    g = np.linspace(MU_LO, MU_HI, n_grid)
    samples = []
    for a in g:
        for lam in g:
            u, v = _uv_exact(x, y, a, lam, nu)
            samples.append(np.where(comp_v, v, u))
    S = np.stack(samples)
    hi, lo = S.max(axis=0), S.min(axis=0)
    offset = 0.5 * (hi + lo)
    scale = np.maximum(0.5 * (hi - lo), 1e-4)
    return offset, scale


def decoders_for(wl: Workload, interior_ids: list, interface_ids: list, act: str = "swish",
                 denorm: bool = True) -> tuple[list, list]:
    """Interior and interface decoders of every subdomain, given the global variable ids
    of each subdomain's interior and interface states (from either side's DD setup)."""
    dec_o, dec_g = [], []
    for i in range(wl.n_sub):
        for kind, ids, n_lat, out in ((0, interior_ids[i], wl.n_omega[i], dec_o),
                                      (1, interface_ids[i], wl.n_gamma[i], dec_g)):
            off, sc = (denormalisation(ids, wl.nx, wl.ny, wl.nu) if denorm else (None, None))
            out.append(decoder(len(ids), wl.width[i], n_lat, wl.band, (wl.seed_offset, i, kind),
                               off, sc, act=act))
    return dec_o, dec_g


def transposed_mask(cols: np.ndarray, width: int) -> np.ndarray:
    """The decoder output mask (ELL column ids per output row, -1 padding) transposed: per hidden unit, the
    output rows whose mask holds it, ascending, as ELL (width x Kt, -1 padding).  The encoder input layer uses
    this mask (Sec. 5.1: the encoder is symmetric to the decoder across the latent layer).  Index bookkeeping
    only."""
    cols = np.asarray(cols)
    r, k = np.nonzero(cols >= 0)
    j = cols[r, k].astype(np.int64)
    order = np.lexsort((r, j))
    j, r = j[order], r[order]
    counts = np.bincount(j, minlength=width)
    Kt = max(int(counts.max()) if counts.size else 0, 1)
    out = np.full((width, Kt), -1, dtype=np.int32)
    start = np.concatenate([[0], np.cumsum(counts)])
    pos = np.arange(j.size) - start[j]
    out[j, pos] = r
    return out


def encoder(n_in: int, width: int, n_lat: int, cols_t: np.ndarray, key: tuple, seed: int = SEED_DEC) -> dict:
    """Random-init sparse-masked shallow encoder h(x) = W2 sigma(W1 x + b1) (Sec. 5.1, Eq.
    autoencoder_architecture a/c) on the transposed decoder mask ``cols_t`` (width x Kt, -1 padding).
    W1 values ~ N(0, 1/nnz_row), b1 = 0, W2 (n_lat x width) ~ N(0, 1/width)."""
    r = rng("enc", seed, *key)
    nnz = (cols_t >= 0).sum(axis=1)
    vals = r.standard_normal(cols_t.shape) / np.sqrt(np.maximum(nnz, 1))[:, None]
    vals[cols_t < 0] = 0.0
    W2 = r.standard_normal((n_lat, width)) / math.sqrt(width)
    return dict(N=n_in, w=width, n=n_lat, cols=np.asarray(cols_t, dtype=np.int32), vals=vals, b1=np.zeros(width),
                W2=W2)


def snapshot_mu(n_side: int) -> np.ndarray:
    """Training parameters: an n_side x n_side uniform grid of mu over [0.9, 1.1]^2 (Sec. 7.2 samples its
    training snapshots on a uniform (a, lambda) grid), shape (n_side^2, 2), a slowest."""
    g = np.linspace(MU_LO, MU_HI, n_side)
    return np.array([(a, l) for a in g for l in g])


def ae_order(n: int, epochs: int, seed: int = SEED_DEC) -> np.ndarray:
    """Sample order of each autoencoder training epoch (epochs x n, int32): one permutation per epoch."""
    r = rng("ae", seed, n, epochs)
    return np.stack([r.permutation(n) for _ in range(epochs)]).astype(np.int32)


def hr_sets(wl: Workload) -> list[np.ndarray]:
    return [hr_rows(nr, nb, i, SEED_HR + wl.seed_offset)
            for i, (nr, nb) in enumerate(zip(wl.residual_rows(), wl.hr_counts()))]


# ------------------------------------------------------------ learned warm start (MLP)

def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round FP32/FP64 values to the nearest bfloat16 (round to nearest even), returned as float32."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).reshape(f.shape)


def mlp_init(n_in: int, hidden: int, n_out: int, seed: int = SEED_MLP) -> np.ndarray:
    """Initial parameters of the warm-start MLP n_in -> hidden -> hidden -> n_out, flat float32 in the order
    W1 (hidden x n_in), b1, W2 (hidden x hidden), b2, W3 (n_out x hidden), b3.  Weights ~ N(0, 1/fan_in),
    biases 0, all bf16-representable."""
    r = rng("mlp", seed, n_in, hidden, n_out)
    parts = []
    for fo, fi in ((hidden, n_in), (hidden, hidden), (n_out, hidden)):
        parts.append(bf16_round(r.standard_normal((fo, fi)) / math.sqrt(fi)).ravel())
        parts.append(np.zeros(fo, dtype=np.float32))
    return np.concatenate(parts).astype(np.float32)


def mlp_order(n: int, epochs: int, seed: int = SEED_MLP) -> np.ndarray:
    """Sample order of each training epoch (epochs x n, int32): one permutation per epoch."""
    r = rng("mlp", seed, 999, n, epochs)
    return np.stack([r.permutation(n) for _ in range(epochs)]).astype(np.int32)
