"""The library's SRPC bookkeeping (ddnm_get_ports, ddnm_set_srpc, ddnm_get_port_matrix; Sec. 3.2 Eq.
dd_lspg_NLP_rom_port, Sec. 5.2 Eq. interface_decoder_rom_port_blocks, port latent sizes of Sec. 7.5) against the
oracle's: the ports (their subdomains, N_j^p, n_j^p), the interface latent sizes and every A^_i are integer or
{-1, 0, 1} results and must be identical.  No device is needed."""
import numpy as np
import pytest

from srpc_case import srpc_case

lib = pytest.importorskip("paper_2305_15163_gb300")


@pytest.mark.parametrize("name,n_tilde", [("tiny12x10_2x2", 2), ("tiny12x10_2x2", 4), ("tiny13x9_3x2", 1),
                                          ("tiny13x9_3x2", 5), ("c1", 3), ("c3", 2)])
def test_ports_and_constraints_match_oracle(name, n_tilde):
    wl, dd, pl, n_p, Q, n_gamma, Ah, _, _ = srpc_case(name, n_tilde)
    n_A = Ah[0].shape[0]
    # the ports can be read off any context of the decomposition
    plain = lib.Solver(wl)
    got, ng = lib.ddnm_get_ports(plain.ctx, n_tilde)
    plain.close()
    assert [g[0] for g in got] == [k for k, _ in pl]
    assert [g[1] for g in got] == [len(v) for _, v in pl]
    assert [g[2] for g in got] == n_p
    assert list(ng) == n_gamma
    if max(n_gamma) > 11 or max(o + g for o, g in zip(wl.n_omega, n_gamma)) > 16:
        # beyond the library's latent sizes (n_i^G <= 11, n_i^O + n_i^G <= 16): refused at set-up
        with pytest.raises(lib.DDNMError) as e:
            lib.Solver(wl, n_gamma=n_gamma, n_c=n_A)
        assert e.value.code == lib.DDNM_E_UNSUPPORTED
        return
    s = lib.Solver(wl, n_gamma=n_gamma, n_c=n_A)
    lib.ddnm_set_srpc(s.ctx, n_tilde)
    for i in range(wl.n_sub):
        assert np.array_equal(lib.ddnm_get_port_matrix(s.ctx, i, n_gamma[i]), Ah[i]), f"A^_{i}"
    s.close()


def test_srpc_rejects_mismatched_sizes():
    wl, dd, pl, n_p, Q, n_gamma, Ah, port_decs, _ = srpc_case("tiny12x10_2x2", 2)
    n_A = Ah[0].shape[0]
    for ng, nc in ((n_gamma, n_A + 1), ([g + 1 for g in n_gamma], n_A)):
        s = lib.Solver(wl, n_gamma=ng, n_c=nc)
        with pytest.raises(lib.DDNMError) as e:
            lib.ddnm_set_srpc(s.ctx, 2)
        assert e.value.code == lib.DDNM_E_INVALID
        s.close()
    s = lib.Solver(wl, n_gamma=n_gamma, n_c=n_A)
    with pytest.raises(lib.DDNMError) as e:           # port decoders before ddnm_set_srpc
        lib.ddnm_load_port_decoder(s.ctx, 0, port_decs[0])
    assert e.value.code == lib.DDNM_E_STATE
    lib.ddnm_set_srpc(s.ctx, 2)
    bad = dict(port_decs[0], n=port_decs[0]["n"] + 1, W1=np.zeros((port_decs[0]["w"], port_decs[0]["n"] + 1)))
    with pytest.raises(lib.DDNMError) as e:           # latent size not the port's n_j^p
        lib.ddnm_load_port_decoder(s.ctx, 0, bad)
    assert e.value.code == lib.DDNM_E_INVALID
    with pytest.raises(lib.DDNMError):
        lib.ddnm_load_port_decoder(s.ctx, len(pl), port_decs[0])
    s.close()


@pytest.mark.parametrize("name,n_tilde,order", [("tiny12x10_2x2", 2, 1), ("tiny12x10_2x2", 4, -1), ("tiny13x9_3x2", 1, -1),
                                                ("c1", 3, 1)])
def test_assembled_interface_decoders_match_oracle(name, n_tilde, order):
    """The library assembles each subdomain's interface decoder from its port decoders once all of them are
    loaded (Eq. interface_decoder_rom_port_blocks): W1, b1, the masked W2 values, scale and offset identical to
    the oracle's assembly, whatever order the ports are loaded in."""
    import inputs
    wl, dd, pl, n_p, Q, n_gamma, Ah, port_decs, dec_g = srpc_case(name, n_tilde)
    s = lib.Solver(wl, n_gamma=n_gamma, n_c=Ah[0].shape[0])
    lib.ddnm_set_srpc(s.ctx, n_tilde)
    dec_o = inputs.decoders_for(wl, [sd.interior for sd in dd.subs], [sd.interface for sd in dd.subs])[0]
    for i, d in enumerate(dec_o):
        lib.ddnm_load_decoders(s.ctx, i, lib.DDNM_DECODER_INTERIOR, d)
    for j in list(range(len(pl)))[::order]:
        lib.ddnm_load_port_decoder(s.ctx, j, port_decs[j])
    for i in range(wl.n_sub):
        got = lib.ddnm_get_decoder(s.ctx, i, lib.DDNM_DECODER_INTERFACE, dec_g[i])
        for k in ("W1", "b1", "vals", "scale", "offset"):
            assert np.array_equal(got[k], dec_g[i][k]), f"subdomain {i}: {k}"
    s.close()
