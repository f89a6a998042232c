"""Build oracle objects for a seeded workload from ``inputs``.

Test infrastructure only (see ``oracle/__init__``).
"""
from __future__ import annotations

import numpy as np

import inputs

from .autoencoder import MaskedAutoencoder
from .burgers import Burgers
from .dd import decompose
from .decoders import EllDecoder, MaskedDecoder
from .rom import DDROM


def build(wl: inputs.Workload, act: str = "swish", denorm: bool = True, ell: bool | None = None):
    """(fom, dd, rom, raw) for workload ``wl``; ``raw`` holds the generator outputs
    (decoder specs, HR rows, C) so that the same inputs can be fed to the CUDA path.
    ell: decoders kept in ELL form (EllDecoder) instead of a dense W2 (MaskedDecoder); by default
    when a dense W2 would exceed 4M entries."""
    fom = Burgers(wl.nx, wl.ny, wl.nu)
    dd = decompose(wl.nx, wl.ny, wl.xb, wl.yb)
    dec_o, dec_g = inputs.decoders_for(wl, [s.interior for s in dd.subs],
                                       [s.interface for s in dd.subs], act=act, denorm=denorm)
    hr = getattr(wl, "hr_override", None)      # explicit collocation rows of a test case, else the seeded draw
    if hr is None:
        hr = inputs.hr_sets(wl)
    C = inputs.test_matrix(wl.n_c(), dd.N_A, inputs.SEED_C + wl.seed_offset)
    if ell is None:
        ell = max(d["N"] * d["w"] for d in dec_o + dec_g) > 4_000_000
    Dec = EllDecoder if ell else MaskedDecoder
    rom = DDROM(fom, dd, [Dec(d) for d in dec_o], [Dec(d) for d in dec_g], hr, C)
    raw = dict(dec_o=dec_o, dec_g=dec_g, hr=hr, C=C)
    return fom, dd, rom, raw


def snapshots(fom: Burgers, mus):
    """FOM solutions at the parameters mus (n x 2), one per row (Sec. 7.2: monolithic solves, restricted to
    the subdomain states afterwards); Newton from the exact solution sampled at the nodes."""
    return np.array([fom.newton(m, x0=fom.exact_state(m))[0] for m in np.asarray(mus).reshape(-1, 2)])


def train_autoencoder(wl: inputs.Workload, i: int, kind: int, Xs, epochs: int, batch: int = 32, lr: float = 1e-3,
                      act: str = "swish") -> MaskedAutoencoder:
    """The interior (kind 0) or interface (kind 1) autoencoder of subdomain i, from its seeded initial weights,
    trained on Xs (n_snap x N: the snapshots restricted to those states; Sec. 7.2-7.3).  The epoch losses
    are kept in ``.losses``."""
    n_lat = (wl.n_omega if kind == 0 else wl.n_gamma)[i]
    dec = inputs.decoder(Xs.shape[1], wl.width[i], n_lat, wl.band, (wl.seed_offset, i, kind), act=act)
    enc = inputs.encoder(Xs.shape[1], wl.width[i], n_lat, inputs.transposed_mask(dec["cols"], wl.width[i]),
                         (wl.seed_offset, i, kind))
    ae = MaskedAutoencoder(enc, dec, act)
    ae.losses = ae.train(Xs, epochs, batch, lr, inputs.ae_order(Xs.shape[0], epochs))
    return ae


def train_autoencoders(wl: inputs.Workload, dd, X, epochs: int, batch: int = 32, lr: float = 1e-3,
                       act: str = "swish"):
    """Interior and interface autoencoders of every subdomain trained on the FOM snapshots X (n_snap x N_x)
    restricted to each subdomain's interior / interface states (Sec. 7.2-7.3), from the seeded initial
    weights.  Returns (autoencoders, decoder specs interior, decoder specs interface)."""
    aes, dec_o, dec_g = [], [], []
    for i, sd in enumerate(dd.subs):
        for kind, ids, out in ((0, sd.interior, dec_o), (1, sd.interface, dec_g)):
            ae = train_autoencoder(wl, i, kind, X[:, ids], epochs, batch, lr, act)
            aes.append(ae)
            out.append(ae.decoder_spec())
    return aes, dec_o, dec_g


def build_trained(wl: inputs.Workload, n_side: int = 8, epochs: int = 300, batch: int = 32, lr: float = 1e-3):
    """(fom, dd, rom, raw) like build(), with decoders trained on FOM snapshots at an n_side x n_side grid of
    mu instead of the random-init decoders."""
    fom = Burgers(wl.nx, wl.ny, wl.nu)
    dd = decompose(wl.nx, wl.ny, wl.xb, wl.yb)
    X = snapshots(fom, inputs.snapshot_mu(n_side))
    aes, dec_o, dec_g = train_autoencoders(wl, dd, X, epochs, batch, lr)
    hr = getattr(wl, "hr_override", None)
    if hr is None:
        hr = inputs.hr_sets(wl)
    C = inputs.test_matrix(wl.n_c(), dd.N_A, inputs.SEED_C + wl.seed_offset)
    rom = DDROM(fom, dd, [MaskedDecoder(d) for d in dec_o], [MaskedDecoder(d) for d in dec_g], hr, C)
    raw = dict(dec_o=dec_o, dec_g=dec_g, hr=hr, C=C, snapshots=X, autoencoders=aes)
    return fom, dd, rom, raw
