"""Seeded SRPC test case shared by the oracle pins and the GPU parity tests: the ports of a workload's
decomposition (oracle.srpc), one random sparse decoder per port (inputs.decoder, swish as in Sec. 7.5, fan-in scaled,
de-normalised by the exact-solution statistics of the port's variables), the assembled interface decoders and
A^_i.  Port latent sizes n_j^p = max(min(N_j^p - 1, n~), 1) (Sec. 7.5)."""
import numpy as np

import inputs
from oracle.burgers import Burgers
from oracle.dd import decompose
from oracle.decoders import MaskedDecoder
from oracle.rom import DDROM
from oracle.srpc import interface_decoder, port_latent_sizes, ports, rom_port_constraints, subdomain_ports


def srpc_case(name, n_tilde=2):
    wl = inputs.workload(name)
    dd = decompose(wl.nx, wl.ny, wl.xb, wl.yb)
    pl = ports(dd)
    n_p = port_latent_sizes(pl, n_tilde)
    Q, n_gamma = subdomain_ports(dd, pl, n_p)
    Ah = rom_port_constraints(dd, pl, n_p, Q, n_gamma)
    port_decs = []
    for j, (key, vs) in enumerate(pl):
        off, sc = inputs.denormalisation(vs, wl.nx, wl.ny, wl.nu)
        w = max(8, min(64, 2 * len(vs)))
        port_decs.append(inputs.decoder(len(vs), w, n_p[j], 3, (wl.seed_offset, 1000 + j, 2), off, sc))
    dec_g = [interface_decoder(sd, pl, port_decs, Q[i]) for i, sd in enumerate(dd.subs)]
    return wl, dd, pl, n_p, Q, n_gamma, Ah, port_decs, dec_g


def srpc_rom(name, n_tilde=2):
    """The oracle's SRPC ROM on every residual row (B_i = I): with sampled rows a small corner port can be missed
    by all of them, and its latent is then fixed by nothing."""
    wl, dd, pl, n_p, Q, n_gamma, Ah, port_decs, dec_g = srpc_case(name, n_tilde)
    fom = Burgers(wl.nx, wl.ny, wl.nu)
    dec_o = inputs.decoders_for(wl, [sd.interior for sd in dd.subs], [sd.interface for sd in dd.subs])[0]
    rom = DDROM(fom, dd, [MaskedDecoder(d) for d in dec_o], [MaskedDecoder(d) for d in dec_g],
                None, np.zeros((Ah[0].shape[0], dd.N_A)), Ahat=Ah)
    return wl, dd, rom, dec_o, port_decs, Ah, n_gamma
