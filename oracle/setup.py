"""Build oracle objects for a seeded workload from ``inputs``.

Test infrastructure only (see ``oracle/__init__``).
"""
from __future__ import annotations

import inputs

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
