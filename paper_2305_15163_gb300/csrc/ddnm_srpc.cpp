// Strong ROM-port constraint (SRPC) formulation (Sec. 3.2, Eq. dd_lspg_NLP_rom_port; Sec. 5.2, Eq.
// interface_decoder_rom_port_blocks), host bookkeeping.
//
// Ports group the interface variables by the set P(j) of subdomains sharing them (Sec. 2): ports in ascending
// lexicographic order of P(j), each port's variables in ascending global order.  Port j has its own decoder
// g_j^p with n_j^p = max(min(N_j^p - 1, n~), 1) latents (Sec. 7.5); subdomain i's interface latents are its
// ports' latents stacked in port order, and its interface decoder is their block-diagonal assembly (W1 and W2
// block-diagonal over the ports, every interface row taking its port decoder's row).  The constraints are
// linear: for every port, every latent component c and every pair s_k < s_{k+1} of consecutive subdomains of
// P(j), a row x^_{s_k}[c] - x^_{s_{k+1}}[c]; rows by port, then component, then k.  D_i = A^_i is constant
// and Atil = sum_i A^_i x^_i^G (the evaluation and the constraint kernel read A^_i).
#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "ddnm_ctx.h"

namespace {

// the ports of ctx's decomposition and each port's latent size under n~
void build_ports(const ddnm_ctx* ctx, int n_tilde, std::vector<PortHost>& out) {
    std::map<int, std::vector<int>> owners;
    for (int s = 0; s < ctx->n_sub; ++s)
        for (int v : ctx->subs[s].interface) owners[v].push_back(s);
    std::map<std::vector<int>, std::vector<int>> groups;
    for (auto& kv : owners) {
        std::vector<int> key = kv.second;
        std::sort(key.begin(), key.end());
        groups[key].push_back(kv.first);
    }
    out.clear();
    for (auto& g : groups) {                       // std::map orders the keys lexicographically
        PortHost p;
        p.subs = g.first;
        p.vars = g.second;                          // ascending: the owners map iterates variables in order
        p.N = (int)p.vars.size();
        p.n = std::max(std::min(p.N - 1, n_tilde), 1);
        out.push_back(p);
    }
}

// subdomain s's ports in order with the offset of each port's latents in x^_s^G
std::vector<std::pair<int, int>> ports_of(const ddnm_ctx* ctx, int s) {
    std::vector<std::pair<int, int>> q;
    int off = 0;
    for (size_t j = 0; j < ctx->ports.size(); ++j)
        if (std::binary_search(ctx->ports[j].subs.begin(), ctx->ports[j].subs.end(), s)) {
            q.push_back({(int)j, off});
            off += ctx->ports[j].n;
        }
    return q;
}

// assemble and load subdomain s's interface decoder from its port decoders (all loaded)
int assemble_interface(ddnm_ctx* ctx, int s) {
    const SubHost& sd = ctx->subs[s];
    const auto q = ports_of(ctx, s);
    int w = 0, n = 0, K = 1, act = -1;
    std::vector<int> hid_off;
    for (auto& pq : q) {
        const DecoderHost& d = ctx->port_dec[pq.first];
        hid_off.push_back(w);
        w += d.w;
        n += d.n;
        K = std::max(K, d.K);
        if (act >= 0 && act != d.act)
            return ddnm_fail(ctx, DDNM_E_INVALID, "SRPC: the ports of subdomain " + std::to_string(s) +
                                                      " have different activations");
        act = d.act;
    }
    const int N = (int)sd.interface.size();
    std::vector<double> W1((size_t)w * n, 0.0), b1(w, 0.0), vals((size_t)N * K, 0.0), scale(N, 1.0), offset(N, 0.0);
    std::vector<int> cols((size_t)N * K, -1);
    for (size_t a = 0; a < q.size(); ++a) {
        const DecoderHost& d = ctx->port_dec[q[a].first];
        const PortHost& p = ctx->ports[q[a].first];
        const int h0 = hid_off[a], l0 = q[a].second;
        for (int r = 0; r < d.w; ++r) {
            b1[h0 + r] = d.b1[r];
            for (int c = 0; c < d.n; ++c) W1[(size_t)(h0 + r) * n + l0 + c] = d.W1[(size_t)r * d.n + c];
        }
        for (int k = 0; k < p.N; ++k) {
            const int row = (int)(std::lower_bound(sd.interface.begin(), sd.interface.end(), p.vars[k]) -
                                  sd.interface.begin());
            for (int t = 0; t < d.K; ++t) {
                const int c = d.cols[(size_t)k * d.K + t];
                cols[(size_t)row * K + t] = c >= 0 ? c + h0 : -1;
                vals[(size_t)row * K + t] = c >= 0 ? d.vals[(size_t)k * d.K + t] : 0.0;
            }
            scale[row] = d.scale[k];
            offset[row] = d.offset[k];
        }
    }
    ddnm_decoder dd{N, w, n, act, K, W1.data(), b1.data(), cols.data(), vals.data(), scale.data(), offset.data()};
    return ddnm_load_decoders(ctx, s, DDNM_DECODER_INTERFACE, &dd);
}

}  // namespace

extern "C" int ddnm_get_ports(const ddnm_ctx* ctx, int n_tilde, int cap, int* n_ports, int* port_subs, int* port_N,
                              int* port_n, int* n_gamma) {
    if (!ctx || !n_ports || n_tilde < 1) return DDNM_E_INVALID;
    std::vector<PortHost> ps;
    build_ports(ctx, n_tilde, ps);
    *n_ports = (int)ps.size();
    if (n_gamma)
        for (int s = 0; s < ctx->n_sub; ++s) {
            int g = 0;
            for (auto& p : ps)
                if (std::binary_search(p.subs.begin(), p.subs.end(), s)) g += p.n;
            n_gamma[s] = g;
        }
    if ((int)ps.size() > cap) return port_subs || port_N || port_n ? DDNM_E_INVALID : DDNM_OK;
    for (size_t j = 0; j < ps.size(); ++j) {
        if (port_subs)
            for (int k = 0; k < 4; ++k) port_subs[j * 4 + k] = k < (int)ps[j].subs.size() ? ps[j].subs[k] : -1;
        if (port_N) port_N[j] = ps[j].N;
        if (port_n) port_n[j] = ps[j].n;
    }
    return DDNM_OK;
}

extern "C" int ddnm_set_srpc(ddnm_ctx* ctx, int n_tilde) {
    if (!ctx) return DDNM_E_INVALID;
    if (n_tilde < 1) return ddnm_fail(ctx, DDNM_E_INVALID, "SRPC: n~ >= 1");
    std::vector<PortHost> ps;
    build_ports(ctx, n_tilde, ps);
    int n_A = 0;
    for (auto& p : ps) {
        if (p.subs.size() > 4) return ddnm_fail(ctx, DDNM_E_UNSUPPORTED, "SRPC: a port shared by more than 4 subdomains");
        n_A += ((int)p.subs.size() - 1) * p.n;
    }
    if (n_A != ctx->n_C)
        return ddnm_fail(ctx, DDNM_E_INVALID, "SRPC: the context's n_C must equal the port constraints' count n_A = " +
                                                  std::to_string(n_A));
    ctx->ports = ps;
    for (int s = 0; s < ctx->n_sub; ++s) {
        int g = 0;
        for (auto& pq : ports_of(ctx, s)) g += ctx->ports[pq.first].n;
        if (g != ctx->subs[s].nG)
            return ddnm_fail(ctx, DDNM_E_INVALID, "SRPC: n_gamma of subdomain " + std::to_string(s) +
                                                      " must be " + std::to_string(g) + " (its ports' latents)");
    }
    // A^_i, n_C x n_i^G each, rows by port, component, chain position
    ctx->Ahat.assign(ctx->n_sub, std::vector<double>());
    for (int s = 0; s < ctx->n_sub; ++s) ctx->Ahat[s].assign((size_t)ctx->n_C * ctx->subs[s].nG, 0.0);
    std::vector<std::map<int, int>> loff(ctx->n_sub);
    for (int s = 0; s < ctx->n_sub; ++s)
        for (auto& pq : ports_of(ctx, s)) loff[s][pq.first] = pq.second;
    int row = 0;
    for (size_t j = 0; j < ctx->ports.size(); ++j) {
        const PortHost& p = ctx->ports[j];
        for (int c = 0; c < p.n; ++c)
            for (size_t k = 0; k + 1 < p.subs.size(); ++k, ++row) {
                const int lo = p.subs[k], hi = p.subs[k + 1];
                ctx->Ahat[lo][(size_t)row * ctx->subs[lo].nG + loff[lo][(int)j] + c] = 1.0;
                ctx->Ahat[hi][(size_t)row * ctx->subs[hi].nG + loff[hi][(int)j] + c] = -1.0;
            }
    }
    ctx->port_dec.assign(ctx->ports.size(), DecoderHost{});
    ctx->srpc = true;
    ctx->C.assign((size_t)ctx->n_C * ctx->N_A, 0.0);   // the WFPC test matrix is not used
    ctx->have_C = true;
    for (int s = 0; s < ctx->n_sub; ++s) ctx->decG[s].loaded = false;
    ctx->finalized = false;
    return DDNM_OK;
}

extern "C" int ddnm_get_port_matrix(const ddnm_ctx* ctx, int sub, double* out) {
    if (!ctx || !ctx->srpc || sub < 0 || sub >= ctx->n_sub || !out) return DDNM_E_INVALID;
    std::copy(ctx->Ahat[sub].begin(), ctx->Ahat[sub].end(), out);
    return DDNM_OK;
}

extern "C" int ddnm_load_port_decoder(ddnm_ctx* ctx, int port, const ddnm_decoder* d) {
    if (!ctx) return DDNM_E_INVALID;
    if (!ctx->srpc) return ddnm_fail(ctx, DDNM_E_STATE, "SRPC not set (ddnm_set_srpc)");
    if (!d || port < 0 || port >= (int)ctx->ports.size()) return ddnm_fail(ctx, DDNM_E_INVALID, "bad port decoder");
    const PortHost& p = ctx->ports[port];
    if (d->N != p.N || d->n != p.n) return ddnm_fail(ctx, DDNM_E_INVALID, "port decoder size does not match the port");
    if (d->w < 1 || d->K < 1 || d->K > ddnm::MAX_K || !d->W1 || !d->b1 || !d->cols || !d->vals)
        return ddnm_fail(ctx, DDNM_E_INVALID, "port decoder arrays or sizes out of range");
    DecoderHost h;
    h.N = d->N; h.w = d->w; h.n = d->n; h.act = d->act; h.K = d->K;
    h.W1.assign(d->W1, d->W1 + (size_t)d->w * d->n);
    h.b1.assign(d->b1, d->b1 + d->w);
    h.cols.assign(d->cols, d->cols + (size_t)d->N * d->K);
    h.vals.assign(d->vals, d->vals + (size_t)d->N * d->K);
    for (int c : h.cols)
        if (c < -1 || c >= d->w) return ddnm_fail(ctx, DDNM_E_INVALID, "port decoder column outside [-1, w)");
    h.scale = d->scale ? std::vector<double>(d->scale, d->scale + d->N) : std::vector<double>(d->N, 1.0);
    h.offset = d->offset ? std::vector<double>(d->offset, d->offset + d->N) : std::vector<double>(d->N, 0.0);
    h.loaded = true;
    ctx->port_dec[port] = std::move(h);
    for (int s : p.subs) {                         // assemble the subdomains whose ports are all loaded
        bool all = true;
        for (auto& pq : ports_of(ctx, s)) all = all && ctx->port_dec[pq.first].loaded;
        if (all) {
            const int rc = assemble_interface(ctx, s);
            if (rc) return rc;
        }
    }
    ctx->finalized = false;
    return DDNM_OK;
}
