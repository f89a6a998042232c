// Host set-up of the DD NM-ROM-HR solve: algebraic domain decomposition (Sec. 2),
// HR stencil tables (Sec. 5.3), HR subnets (Sec. 5.4), device upload.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>

#include "ddnm_ctx.h"

using namespace ddnm;

// message of the last failed ddnm_setup on this thread (there is no context to hold it)
static thread_local std::string g_setup_err;

int ddnm_fail(ddnm_ctx* ctx, int code, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return code;
}

static int cuda_fail(ddnm_ctx* ctx, cudaError_t e, const char* what) {
    return ddnm_fail(ctx, DDNM_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                  \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);  \
    } while (0)

static int find_sorted(const std::vector<int>& v, int key) {
    auto it = std::lower_bound(v.begin(), v.end(), key);
    return (it != v.end() && *it == key) ? int(it - v.begin()) : -1;
}

// ------------------------------------------------------------------------------- set-up

extern "C" int ddnm_setup(const ddnm_problem* p, ddnm_ctx** out) {
    if (!out) return DDNM_E_INVALID;
    *out = nullptr;
    if (!p) {
        g_setup_err = "ddnm_setup: problem is NULL";
        return DDNM_E_INVALID;
    }
    ddnm_ctx* ctx = new (std::nothrow) ddnm_ctx();
    if (!ctx) return DDNM_E_NOMEM;
    auto bail = [&](int code, const std::string& msg) {
        g_setup_err = "ddnm_setup: " + msg;
        delete ctx;
        return code;
    };
    g_setup_err.clear();
    if (p->nx < 2 || p->ny < 2 || p->kx < 1 || p->ky < 1 || !p->xb || !p->yb || !p->n_omega || !p->n_gamma ||
        !p->hr_count || !p->hr_rows)
        return bail(DDNM_E_INVALID, "missing or non-positive problem fields");
    if (p->kx * p->ky < 2) return bail(DDNM_E_UNSUPPORTED, "at least two subdomains are needed (WFPC constraints)");
    if (p->kx * p->ky > MAX_SUB) return bail(DDNM_E_UNSUPPORTED, "at most 256 subdomains");
    if (p->device < 0) return bail(DDNM_E_INVALID, "negative device ordinal");
    if (!(p->nu > 0) || !(p->box[1] > p->box[0]) || !(p->box[3] > p->box[2]))
        return bail(DDNM_E_INVALID, "nu and the box must be positive");
    if (p->precision != DDNM_FP64 && p->precision != DDNM_MIXED) return bail(DDNM_E_INVALID, "unknown precision");
    if (p->n_c < 1 || p->n_c > MAX_NC) return bail(DDNM_E_UNSUPPORTED, "n_c must be in 1..128");
    if ((long long)p->nx * p->ny * 2 >= (1LL << OP_SHIFT)) return bail(DDNM_E_UNSUPPORTED, "grid too large");

    ctx->nx = p->nx; ctx->ny = p->ny; ctx->kx = p->kx; ctx->ky = p->ky;
    ctx->n_sub = p->kx * p->ky;
    ctx->N = p->nx * p->ny;
    ctx->nu = p->nu;
    std::memcpy(ctx->box, p->box, sizeof(ctx->box));
    ctx->hx = (p->box[1] - p->box[0]) / (p->nx + 1);
    ctx->hy = (p->box[3] - p->box[2]) / (p->ny + 1);
    ctx->precision = p->precision;
    ctx->device = p->device;
    ctx->n_C = p->n_c;
    ctx->xb.assign(p->xb, p->xb + p->kx + 1);
    ctx->yb.assign(p->yb, p->yb + p->ky + 1);
    if (ctx->xb.front() != 0 || ctx->xb.back() != p->nx || ctx->yb.front() != 0 || ctx->yb.back() != p->ny)
        return bail(DDNM_E_INVALID, "breakpoints must start at 0 and end at nx / ny");
    for (int k = 0; k < p->kx; ++k)
        if (ctx->xb[k + 1] <= ctx->xb[k]) return bail(DDNM_E_INVALID, "x breakpoints must increase");
    for (int k = 0; k < p->ky; ++k)
        if (ctx->yb[k + 1] <= ctx->yb[k]) return bail(DDNM_E_INVALID, "y breakpoints must increase");

    // the set-up is host bookkeeping only; the device is first touched when the first
    // solve / evaluation uploads the tables (ddnm_finalize)
    const int nx = p->nx, ny = p->ny, N = ctx->N, ns = ctx->n_sub;
    // owner of each node
    std::vector<int> owner(N);
    ctx->subs.resize(ns);
    for (int sy = 0; sy < p->ky; ++sy)
        for (int sx = 0; sx < p->kx; ++sx) {
            int s = sy * p->kx + sx;
            for (int j = ctx->yb[sy]; j < ctx->yb[sy + 1]; ++j)
                for (int i = ctx->xb[sx]; i < ctx->xb[sx + 1]; ++i) {
                    owner[j * nx + i] = s;
                    ctx->subs[s].owned.push_back(j * nx + i);
                }
        }
    for (auto& sd : ctx->subs) std::sort(sd.owned.begin(), sd.owned.end());

    // sharing set of each node: the owners of the node and of its in-grid 5-point neighbours
    // (node q enters the residual of subdomain s iff s owns q or a neighbour of q)
    std::vector<unsigned char> nshare(N);
    std::vector<int> share(5 * (size_t)N);
    for (int q = 0; q < N; ++q) {
        int i = q % nx, j = q / nx, c = 0;
        int tmp[5];
        tmp[c++] = owner[q];
        if (i > 0) tmp[c++] = owner[q - 1];
        if (i < nx - 1) tmp[c++] = owner[q + 1];
        if (j > 0) tmp[c++] = owner[q - nx];
        if (j < ny - 1) tmp[c++] = owner[q + nx];
        std::sort(tmp, tmp + c);
        int m = int(std::unique(tmp, tmp + c) - tmp);
        nshare[q] = (unsigned char)m;
        for (int k = 0; k < m; ++k) share[5 * (size_t)q + k] = tmp[k];
    }
    // interior and interface variables of each subdomain
    std::vector<int> stamp(N, -1);
    for (int s = 0; s < ns; ++s) {
        SubHost& sd = ctx->subs[s];
        std::vector<int> dep;
        for (int q : sd.owned) {
            int i = q % nx, j = q / nx;
            int nb[5] = {q, i > 0 ? q - 1 : -1, i < nx - 1 ? q + 1 : -1, j > 0 ? q - nx : -1, j < ny - 1 ? q + nx : -1};
            for (int v : nb)
                if (v >= 0 && stamp[v] != s) {
                    stamp[v] = s;
                    dep.push_back(v);
                }
        }
        std::sort(dep.begin(), dep.end());
        std::vector<int> in_n, face_n;
        for (int q : dep) (nshare[q] > 1 ? face_n : in_n).push_back(q);
        for (int comp = 0; comp < 2; ++comp) {
            for (int q : in_n) sd.interior.push_back(comp * N + q);
            for (int q : face_n) sd.interface.push_back(comp * N + q);
        }
        sd.nO = p->n_omega[s];
        sd.nG = p->n_gamma[s];
        if (sd.nO < 1 || sd.nG < 0 || sd.nO + sd.nG > MAX_NI || sd.nG > MAX_NG)
            return bail(DDNM_E_UNSUPPORTED, "latent dims must satisfy 1 <= n^O, n^G <= 11, n^O + n^G <= 16");
        if (ns > 1 && sd.nG < 1) return bail(DDNM_E_INVALID, "n^G must be >= 1 with more than one subdomain");
    }
    // compatibility rows
    ctx->goff.assign(ns + 1, 0);
    for (int s = 0; s < ns; ++s) ctx->goff[s + 1] = ctx->goff[s] + (int)ctx->subs[s].interface.size();
    ctx->sum_NG = ctx->goff[ns];
    for (int var = 0; var < 2 * N; ++var) {
        int q = var % N, m = nshare[q];
        for (int k = 0; k + 1 < m; ++k) {
            int lo = share[5 * (size_t)q + k], hi = share[5 * (size_t)q + k + 1];
            int li = find_sorted(ctx->subs[lo].interface, var), hj = find_sorted(ctx->subs[hi].interface, var);
            if (li < 0 || hj < 0) return bail(DDNM_E_INVALID, "internal: shared variable missing from an interface");
            ctx->con_var.push_back(var);
            ctx->con_lo.push_back(lo);
            ctx->con_hi.push_back(hi);
            ctx->con_lo_flat.push_back(ctx->goff[lo] + li);
            ctx->con_hi_flat.push_back(ctx->goff[hi] + hj);
        }
    }
    ctx->N_A = (int)ctx->con_var.size();
    if (ns > 1 && ctx->N_A == 0) return bail(DDNM_E_INVALID, "internal: no compatibility rows");

    // HR rows and their stencil operands
    std::map<long long, int> bnd_id;
    int hr_pos = 0;
    for (int s = 0; s < ns; ++s) {
        SubHost& sd = ctx->subs[s];
        int nb = p->hr_count[s];
        int nown = (int)sd.owned.size();
        if (nb < sd.nO + sd.nG || nb > 2 * nown)
            return bail(DDNM_E_INVALID, "hr_count must be in [n^O + n^G, N_r]");
        sd.hr_rows.assign(p->hr_rows + hr_pos, p->hr_rows + hr_pos + nb);
        hr_pos += nb;
        for (int k = 0; k < nb; ++k) {
            if (sd.hr_rows[k] < 0 || sd.hr_rows[k] >= 2 * nown || (k && sd.hr_rows[k] <= sd.hr_rows[k - 1]))
                return bail(DDNM_E_INVALID, "hr_rows must be ascending local residual-row ids");
        }
        // first pass: interior outputs the stencils need (I_o)
        std::vector<int> raw;   // (comp, var or -(boundary key)-1) per operand
        for (int l : sd.hr_rows) {
            int comp = l / nown, q = sd.owned[l % nown];
            int i = q % nx, j = q / nx;
            // operands: centre, E, W, N, S of component comp, then the other component at the centre
            int I[6] = {i, i + 1, i - 1, i, i, i}, J[6] = {j, j, j, j + 1, j - 1, j};
            int cmp[6] = {comp, comp, comp, comp, comp, 1 - comp};
            raw.push_back(comp);
            for (int o = 0; o < 6; ++o) {
                if (I[o] >= 0 && I[o] < nx && J[o] >= 0 && J[o] < ny) {
                    raw.push_back(cmp[o] * N + J[o] * nx + I[o]);
                } else {
                    long long key = (long long)(J[o] + 1) * (nx + 2) + (I[o] + 1);   // 1-based grid point
                    auto it = bnd_id.find(key);
                    int id;
                    if (it == bnd_id.end()) {
                        id = (int)bnd_id.size();
                        bnd_id[key] = id;
                        ctx->bnd_ij.push_back(I[o] + 1);
                        ctx->bnd_ij.push_back(J[o] + 1);
                    } else {
                        id = it->second;
                    }
                    raw.push_back(-(2 * id + cmp[o]) - 1);
                }
            }
        }
        // outputs the stencils use: interior (I_o of the interior subnet) and interface; the operand codes
        // and the chunking of the collocation rows are made when the tables are uploaded
        for (int k = 0; k < nb; ++k)
            for (int o = 0; o < 6; ++o) {
                const int v = raw[k * HR_INTS + 1 + o];
                if (v < 0) continue;
                const int li = find_sorted(sd.interior, v);
                if (li >= 0) {
                    sd.need.push_back(li);
                } else {
                    const int gi = find_sorted(sd.interface, v);
                    if (gi < 0) return bail(DDNM_E_INVALID, "internal: stencil operand outside the subdomain");
                    sd.needG.push_back(gi);
                }
            }
        for (auto* v : {&sd.need, &sd.needG}) {
            std::sort(v->begin(), v->end());
            v->erase(std::unique(v->begin(), v->end()), v->end());
        }
        sd.hr_raw = std::move(raw);
        ctx->sum_NB += nb;
        ctx->n_D += sd.nO + sd.nG;
    }
    ctx->decO.resize(ns);
    ctx->decG.resize(ns);
    *out = ctx;
    return DDNM_OK;
}

extern "C" void ddnm_destroy(ddnm_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaFree(ctx->d_vpool);
    cudaFree(ctx->d_ipool);
    cudaFree(ctx->d_hr);
    cudaFree(ctx->d_con);
    cudaFree(ctx->d_C);
    cudaFree(ctx->d_Ct);
    cudaFree(ctx->d_Qtc);
    cudaFree(ctx->d_Ahat);
    cudaFree(ctx->d_err);
    cudaFree(ctx->d_bnd_ij);
    cudaFree(ctx->d_sub);
    cudaFree(ctx->d_chunk);
    cudaFree(ctx->d_tiles);
    cudaFree(ctx->d_classes);
    cudaFree(ctx->d_ws);
    if (ctx->h_active) cudaFreeHost(ctx->h_active);
    ddnm_release_graph(ctx);
    ddnm_release_events(ctx);
    ddnm_ws_release(ctx);
    ddnm_fom_release(ctx);
    ddnm_ae_release(ctx);
    delete ctx;
}

extern "C" const char* ddnm_last_error(const ddnm_ctx* ctx) { return ctx ? ctx->err.c_str() : g_setup_err.c_str(); }

extern "C" int ddnm_get_sizes(const ddnm_ctx* ctx, ddnm_sizes* out) {
    if (!ctx || !out) return DDNM_E_INVALID;
    out->n_sub = ctx->n_sub;
    out->N_x = 2 * ctx->N;
    out->n_D = ctx->n_D;
    out->n_C = ctx->n_C;
    out->N_A = ctx->N_A;
    out->sum_hr = ctx->sum_NB;
    out->sum_gamma = ctx->sum_NG;
    return DDNM_OK;
}

extern "C" int ddnm_get_subdomain(const ddnm_ctx* ctx, int sub, int* info, int* interior_ids, int* interface_ids) {
    if (!ctx || sub < 0 || sub >= ctx->n_sub) return DDNM_E_INVALID;
    const SubHost& sd = ctx->subs[sub];
    if (info) {
        info[0] = 2 * (int)sd.owned.size();
        info[1] = (int)sd.interior.size();
        info[2] = (int)sd.interface.size();
        info[3] = sd.nO;
        info[4] = sd.nG;
        info[5] = (int)sd.hr_rows.size();
    }
    if (interior_ids) std::copy(sd.interior.begin(), sd.interior.end(), interior_ids);
    if (interface_ids) std::copy(sd.interface.begin(), sd.interface.end(), interface_ids);
    return DDNM_OK;
}

extern "C" int ddnm_get_constraints(const ddnm_ctx* ctx, int* row_var, int* row_lo, int* row_hi) {
    if (!ctx) return DDNM_E_INVALID;
    if (row_var) std::copy(ctx->con_var.begin(), ctx->con_var.end(), row_var);
    if (row_lo) std::copy(ctx->con_lo.begin(), ctx->con_lo.end(), row_lo);
    if (row_hi) std::copy(ctx->con_hi.begin(), ctx->con_hi.end(), row_hi);
    return DDNM_OK;
}

extern "C" int ddnm_set_test_matrix(ddnm_ctx* ctx, const double* C) {
    if (!ctx) return DDNM_E_INVALID;
    if (!C) return ddnm_fail(ctx, DDNM_E_INVALID, "C is NULL");
    size_t n = (size_t)ctx->n_C * ctx->N_A;
    for (size_t k = 0; k < n; ++k)
        if (!std::isfinite(C[k])) return ddnm_fail(ctx, DDNM_E_INVALID, "C has a non-finite entry");
    ctx->C.assign(C, C + n);
    ctx->have_C = true;
    ctx->finalized = false;
    return DDNM_OK;
}

extern "C" int ddnm_set_options(ddnm_ctx* ctx, const ddnm_options* o) {
    if (!ctx || !o) return DDNM_E_INVALID;
    if (!(o->tol >= 0) || o->max_iter < 0 || !(o->armijo_c1 >= 0 && o->armijo_c1 < 0.5) || !(o->beta > 0 && o->beta < 1) ||
        o->max_backtracks < 0 || o->max_iter > 100000 || o->max_backtracks > 60 || !(o->step_tol >= 0.0 &&
        o->step_tol < 1.0))
        return ddnm_fail(ctx, DDNM_E_INVALID, "options out of range");
    ctx->opt = *o;
    return DDNM_OK;
}

extern "C" int ddnm_set_hr_projection(ddnm_ctx* ctx, int sub, int nr, const double* proj) {
    if (!ctx) return DDNM_E_INVALID;
    if (sub < 0 || sub >= ctx->n_sub || nr < 0 || nr > MAX_NR || (nr && !proj))
        return ddnm_fail(ctx, DDNM_E_INVALID, "hr projection: sub in range, 0 <= nr <= 64, proj given when nr > 0");
    SubHost& sd = ctx->subs[sub];
    const size_t nb = sd.hr_rows.size();
    if ((size_t)nr > nb) return ddnm_fail(ctx, DDNM_E_INVALID, "hr projection: nr above the subdomain's HR rows");
    for (size_t k = 0; k < (size_t)nr * nb; ++k)
        if (!std::isfinite(proj[k])) return ddnm_fail(ctx, DDNM_E_INVALID, "hr projection: non-finite entry");
    sd.nr = nr;
    sd.proj.assign(proj, proj + (size_t)nr * nb);
    ctx->finalized = false;      // the next compute call uploads it
    return DDNM_OK;
}

extern "C" int ddnm_load_decoders(ddnm_ctx* ctx, int sub, int kind, const ddnm_decoder* d) {
    if (!ctx) return DDNM_E_INVALID;
    if (!d || sub < 0 || sub >= ctx->n_sub || (kind != DDNM_DECODER_INTERIOR && kind != DDNM_DECODER_INTERFACE))
        return ddnm_fail(ctx, DDNM_E_INVALID, "bad decoder arguments");
    const SubHost& sd = ctx->subs[sub];
    int N = kind == DDNM_DECODER_INTERIOR ? (int)sd.interior.size() : (int)sd.interface.size();
    int n = kind == DDNM_DECODER_INTERIOR ? sd.nO : sd.nG;
    if (d->N != N || d->n != n) return ddnm_fail(ctx, DDNM_E_INVALID, "decoder size does not match the decomposition");
    if (d->w < 1 || d->K < 1 || d->K > MAX_K) return ddnm_fail(ctx, DDNM_E_UNSUPPORTED, "decoder width or K out of range");
    if (d->act < DDNM_ACT_SWISH || d->act > DDNM_ACT_IDENTITY) return ddnm_fail(ctx, DDNM_E_INVALID, "unknown activation");
    if (!d->W1 || !d->b1 || !d->cols || !d->vals) return ddnm_fail(ctx, DDNM_E_INVALID, "decoder array is NULL");
    DecoderHost h;
    h.N = N; h.w = d->w; h.n = n; h.act = d->act; h.K = d->K;
    h.W1.assign(d->W1, d->W1 + (size_t)d->w * n);
    h.b1.assign(d->b1, d->b1 + d->w);
    h.cols.assign(d->cols, d->cols + (size_t)N * d->K);
    h.vals.assign(d->vals, d->vals + (size_t)N * d->K);
    for (int r = 0; r < N; ++r) {
        bool pad = false;
        for (int t = 0; t < d->K; ++t) {
            int c = h.cols[(size_t)r * d->K + t];
            if (c < -1 || c >= d->w) return ddnm_fail(ctx, DDNM_E_INVALID, "decoder column outside [-1, w)");
            if (c < 0) pad = true;
            else if (pad) return ddnm_fail(ctx, DDNM_E_INVALID, "decoder row has a column after -1 padding");
        }
    }
    h.scale = d->scale ? std::vector<double>(d->scale, d->scale + N) : std::vector<double>(N, 1.0);
    h.offset = d->offset ? std::vector<double>(d->offset, d->offset + N) : std::vector<double>(N, 0.0);
    for (double v : h.W1) if (!std::isfinite(v)) return ddnm_fail(ctx, DDNM_E_INVALID, "non-finite W1");
    h.loaded = true;
    (kind == DDNM_DECODER_INTERIOR ? ctx->decO : ctx->decG)[sub] = std::move(h);
    ctx->finalized = false;
    return DDNM_OK;
}

// ------------------------------------------------------------------- finalize (upload)

namespace {
struct Pools {
    std::vector<double> v;
    std::vector<int> i;
    long long addv(const double* p, size_t n) {
        long long o = (long long)v.size();
        v.insert(v.end(), p, p + n);
        while (v.size() % 4) v.push_back(0.0);   // 16-byte alignment of every array, float and double views
        return o;
    }
    long long addi(const int* p, size_t n) {
        long long o = (long long)i.size();
        i.insert(i.end(), p, p + n);
        while (i.size() % 4) i.push_back(0);
        return o;
    }
};

// Hidden layer of the HR subnet (Sec. 5.4): I_h = union of the mask columns of the rows Io, ascending;
// W1~ = W1[I_h] (rows padded to round4(n)), b1~ = b1[I_h].  pos maps a hidden unit to its place in I_h.
void subnet_hidden(const DecoderHost& d, const std::vector<int>& Io, Pools& P, long long& w1, long long& b1, int& h,
                   std::vector<int>& pos) {
    std::vector<int> Ih;
    for (int r : Io)
        for (int t = 0; t < d.K; ++t) {
            int c = d.cols[(size_t)r * d.K + t];
            if (c >= 0) Ih.push_back(c);
        }
    std::sort(Ih.begin(), Ih.end());
    Ih.erase(std::unique(Ih.begin(), Ih.end()), Ih.end());
    pos.assign(d.w, -1);
    for (size_t k = 0; k < Ih.size(); ++k) pos[Ih[k]] = (int)k;
    const int n4 = round4(d.n);
    std::vector<double> W1s((size_t)Ih.size() * n4, 0.0), b1s;
    for (size_t k = 0; k < Ih.size(); ++k) {
        for (int j = 0; j < d.n; ++j) W1s[k * n4 + j] = d.W1[(size_t)Ih[k] * d.n + j];
        b1s.push_back(d.b1[Ih[k]]);
    }
    h = (int)Ih.size();
    w1 = P.addv(W1s.data(), W1s.size());
    b1 = P.addv(b1s.data(), b1s.size());
}

// d's row-major ELL W2 widened to K slots a row (the extra slots column -1, value 0)
void pad_ell(const DecoderHost& d, int K, std::vector<int>& cols, std::vector<double>& vals) {
    cols.assign((size_t)d.N * K, -1);
    vals.assign((size_t)d.N * K, 0.0);
    for (int r = 0; r < d.N; ++r)
        for (int t = 0; t < d.K; ++t) {
            cols[(size_t)r * K + t] = d.cols[(size_t)r * d.K + t];
            vals[(size_t)r * K + t] = d.vals[(size_t)r * d.K + t];
        }
}

// Output rows `rows` of the subnet W2~ (Eq. subnet) in slot-major ELL (Kp slots; padding column 0 value 0),
// columns renumbered into I_h, followed by their scale and offset.
void subnet_rows(const DecoderHost& d, const std::vector<int>& rows, const std::vector<int>& pos, int Kp, Pools& P,
                 long long& col, long long& val, long long& so) {
    const size_t m = rows.size();
    std::vector<int> cs(Kp * m, 0);
    std::vector<double> vs(Kp * m, 0.0), sc;
    for (size_t r = 0; r < m; ++r)
        for (int t = 0; t < d.K; ++t) {
            int c = d.cols[(size_t)rows[r] * d.K + t];
            if (c >= 0) {
                cs[t * m + r] = pos[c];
                vs[t * m + r] = d.vals[(size_t)rows[r] * d.K + t];
            }
        }
    for (int r : rows) sc.push_back(d.scale[r]);
    for (int r : rows) sc.push_back(d.offset[r]);
    col = P.addi(cs.data(), cs.size());
    val = P.addv(vs.data(), vs.size());
    so = P.addv(sc.data(), sc.size());
}
// The same rows as dense-window tiles (TileDev) for the banded masks of Sec. 5.1, where consecutive rows
// share most of their columns: a warp then reads each hidden record of a tile's window once (a broadcast)
// instead of once per row and mask entry.  Returns false, adding nothing, when the windows would hold
// more than 2.5 values per mask entry (a scattered mask keeps the ELL table).
bool subnet_tiles(const DecoderHost& d, const std::vector<int>& rows, const std::vector<int>& pos, int h, Pools& P,
                  std::vector<TileDev>& tiles, int& tile0, int& ntiles) {
    const size_t m = rows.size();
    const int hpad = round4(h);
    size_t nnz = 0, stored = 0;
    std::vector<TileDev> loc;
    std::vector<std::vector<double>> vals;
    for (size_t t0 = 0; t0 < m; t0 += 32) {
        const size_t t1 = std::min(m, t0 + 32);
        int lo = 1 << 30, hi = -1;
        for (size_t r = t0; r < t1; ++r)
            for (int k = 0; k < d.K; ++k) {
                const int c = d.cols[(size_t)rows[r] * d.K + k];
                if (c < 0) continue;
                lo = std::min(lo, pos[c]);
                hi = std::max(hi, pos[c]);
                ++nnz;
            }
        if (hi < 0) lo = hi = 0;
        const int tw = round4(hi - lo + 1);
        if (tw > hpad) return false;
        const int c0 = std::min(lo, hpad - tw);
        std::vector<double> v((size_t)tw * 32, 0.0);
        for (size_t r = t0; r < t1; ++r)
            for (int k = 0; k < d.K; ++k) {
                const int c = d.cols[(size_t)rows[r] * d.K + k];
                if (c < 0) continue;
                const int j = pos[c] - c0, lane = (int)(r - t0);
                v[(size_t)(j / 4) * 128 + lane * 4 + j % 4] = d.vals[(size_t)rows[r] * d.K + k];
            }
        stored += v.size();
        loc.push_back(TileDev{c0, tw, 0});
        vals.push_back(std::move(v));
    }
    if (m == 0 || (double)stored > 2.5 * (double)nnz) return false;
    tile0 = (int)tiles.size();
    ntiles = (int)loc.size();
    for (size_t t = 0; t < loc.size(); ++t) {
        loc[t].voff = P.addv(vals[t].data(), vals[t].size());
        tiles.push_back(loc[t]);
    }
    return true;
}
// Distinct mask columns over the outputs `rows` (the hidden width |I_h| of their subnet).
int hidden_count(const DecoderHost& d, const std::vector<int>& rows) {
    std::vector<char> used(d.w, 0);
    int n = 0;
    for (int r : rows)
        for (int t = 0; t < d.K; ++t) {
            const int c = d.cols[(size_t)r * d.K + t];
            if (c >= 0 && !used[c]) {
                used[c] = 1;
                ++n;
            }
        }
    return n;
}

// The collocation rows of a subdomain cut into chunks of hc rows: the interior outputs each chunk's
// stencils use (chunk-local slots, ascending) and, with ops, the operand codes of every row (component,
// then per operand: interior -> chunk slot, interface -> slot among the interface outputs the stencils
// use, Dirichlet point -> 2 * point + component).
void chunk_rows(const SubHost& sd, int hc, std::vector<std::vector<int>>& chunk_need, std::vector<int>* ops) {
    const int nb = (int)sd.hr_rows.size();
    chunk_need.assign((nb + hc - 1) / hc, {});
    for (int k = 0; k < nb; ++k)
        for (int o = 0; o < 6; ++o) {
            const int v = sd.hr_raw[(size_t)k * HR_INTS + 1 + o];
            if (v < 0) continue;
            const int li = find_sorted(sd.interior, v);
            if (li >= 0) chunk_need[k / hc].push_back(li);
        }
    for (auto& cn : chunk_need) {
        std::sort(cn.begin(), cn.end());
        cn.erase(std::unique(cn.begin(), cn.end()), cn.end());
    }
    if (!ops) return;
    ops->clear();
    for (int k = 0; k < nb; ++k) {
        ops->push_back(sd.hr_raw[(size_t)k * HR_INTS]);
        for (int o = 0; o < 6; ++o) {
            const int v = sd.hr_raw[(size_t)k * HR_INTS + 1 + o];
            int code;
            if (v >= 0) {
                const int li = find_sorted(sd.interior, v);
                if (li >= 0) code = (OP_INTERIOR << OP_SHIFT) | find_sorted(chunk_need[k / hc], li);
                else code = (OP_INTERFACE << OP_SHIFT) | find_sorted(sd.needG, find_sorted(sd.interface, v));
            } else {
                code = (OP_BOUNDARY << OP_SHIFT) | (-v - 1);
            }
            ops->push_back(code);
        }
    }
}
}  // namespace

int ddnm_finalize(ddnm_ctx* ctx) {
    if (ctx->finalized) return DDNM_OK;
    if (!ctx->have_C) return ddnm_fail(ctx, DDNM_E_STATE, "test matrix C not set");
    for (int s = 0; s < ctx->n_sub; ++s)
        if (!ctx->decO[s].loaded || !ctx->decG[s].loaded)
            return ddnm_fail(ctx, DDNM_E_STATE, "decoder of subdomain " + std::to_string(s) + " not loaded");
    CK(cudaSetDevice(ctx->device));
    const int ns = ctx->n_sub, nC = ctx->n_C;
    Pools P;
    std::vector<int> hr_all;
    ctx->hsub.assign(ns, SubDev{});
    ctx->hchunk.clear();
    ctx->htiles.clear();
    // an instance's block area: the n_sub merits ||rho_i||^2, then per subdomain ||s_i||^2 and ||x_i||^2 of the
    // last Gauss-Newton step (the step test), padded to an even count, then the blocks
    int xoff = 0, hr_off = 0, blk = (3 * ctx->n_sub + 1) & ~1;
    long long pg_stride = 0;
    std::vector<float> qtc;        // mixed path: every Q_i split and tiled for the tensor-core D_i GEMM
    std::vector<double> ahat_all;  // SRPC: every A^_i
    ctx->max_nG = 1;
    const size_t tsize = ctx->precision == DDNM_FP64 ? 8 : 4;
    ctx->eval_smem = 0;
    ctx->rec_smem = 0;
    ctx->nnzO.assign(ns, 0);
    ctx->nnzG.assign(ns, 0);
    ctx->nnzGn.assign(ns, 0);
    int dev_max = 0, sm_smem = 0;
    CK(cudaDeviceGetAttribute(&dev_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
    CK(cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, ctx->device));
    // collocation rows per chunk, among 128, 64, ..., 8: among the candidates with the most evaluation CTAs
    // per SM (shared memory against the register budget), the largest whose CTAs leave the SM at least
    // L1_KEEP bytes of its unified L1 / shared memory for caching the decoder tables, else the largest.
    // Resident CTAs hide the evaluation's latency and every chunk adds barriers and a round of table loads,
    // but the tables are re-read per instance.  Measured (k_eval, one 1024-instance launch): 1024^2 / 8 x 8
    // mixed, 32 rows at 3 CTAs per SM 12.1 ms, 16 rows at 3 CTAs 16.0 ms, 64 rows at 2 CTAs 12.8 ms, 128 rows
    // at 2 CTAs (208 kB of shared memory per SM) 18.1 ms; the same in FP64 at one CTA per SM, 32 rows
    // 161 ms, 128 rows (about 200 kB) 252 ms; 128 x 128 / 4 x 4 mixed at 4 CTAs, 128 rows 0.83 ms, 32 rows
    // 1.16 ms.  It must fit one CTA.
    int hc = 0;
    {
        std::vector<int> hO(ns), hG(ns);
        for (int s = 0; s < ns; ++s) {
            std::vector<int> allG(ctx->subs[s].interface.size());
            for (size_t r = 0; r < allG.size(); ++r) allG[r] = (int)r;
            hO[s] = hidden_count(ctx->decO[s], ctx->subs[s].need);
            hG[s] = hidden_count(ctx->decG[s], allG);
        }
        int smallest = 1 << 30;
        struct Cand { int chunk, ctas, bytes; };
        std::vector<Cand> cands;                    // the candidates that fit, largest first
        for (int cand = HR_CHUNK; cand >= 8; cand /= 2) {
            int bytes = 0, ctas = 1 << 30;
            for (int s = 0; s < ns; ++s) {
                const SubHost& sd = ctx->subs[s];
                std::vector<std::vector<int>> cn;
                chunk_rows(sd, cand, cn, nullptr);
                SubDev T{};
                T.nO = sd.nO; T.nG = sd.nG; T.ni = sd.nO + sd.nG; T.hO = hO[s]; T.hG = hG[s];
                T.NG = (int)sd.interface.size(); T.NGn = (int)sd.needG.size(); T.hr_chunk = cand; T.nr = sd.nr;
                for (const auto& c : cn) T.mmax = std::max(T.mmax, (int)c.size());
                const int b = eval_smem(T, nC, (int)tsize).bytes;
                bytes = std::max(bytes, b);
                const int by_smem = sm_smem / (b + 1024);      // 1 KB per CTA is the runtime's own
                ctas = std::min(ctas, std::min(by_smem, eval_ctas_by_regs((int)tsize, round4(T.nO + 1), round4(T.nG + 1))));
            }
            smallest = std::min(smallest, bytes);
            if (bytes <= dev_max) cands.push_back({cand, ctas, bytes});
        }
        int best = 0;
        for (const auto& c : cands) best = std::max(best, c.ctas);
        constexpr int L1_KEEP = 88 * 1024;           // of the 256 kB unified L1 / shared memory of an SM
        for (const auto& c : cands)
            if (!hc && c.ctas == best && c.ctas * (c.bytes + 1024) <= 256 * 1024 - L1_KEEP) hc = c.chunk;
        for (const auto& c : cands)
            if (!hc && c.ctas == best) hc = c.chunk;
        if (!hc)
            return ddnm_fail(ctx, DDNM_E_UNSUPPORTED, "a subdomain's evaluation needs " + std::to_string(smallest) +
                                                          " bytes of shared memory (device limit " +
                                                          std::to_string(dev_max) + ")");
    }
    for (int s = 0; s < ns; ++s) {
        const SubHost& sd = ctx->subs[s];
        const DecoderHost &dO = ctx->decO[s], &dG = ctx->decG[s];
        SubDev& S = ctx->hsub[s];
        S.nO = sd.nO; S.nG = sd.nG; S.ni = sd.nO + sd.nG; S.xoff = xoff; xoff += S.ni;
        S.NB = (int)sd.hr_rows.size(); S.hr_off = hr_off; hr_off += S.NB;
        S.nr = sd.nr;
        S.ahat = 0;
        if (ctx->srpc) {
            S.ahat = (long long)ahat_all.size();
            ahat_all.insert(ahat_all.end(), ctx->Ahat[s].begin(), ctx->Ahat[s].end());
        }
        S.gp = sd.nr ? P.addv(sd.proj.data(), sd.proj.size()) : 0;
        // one ELL row length per subdomain (the shorter decoder's rows padded with -1 slots)
        S.K = std::max(dO.K, dG.K); S.Kp = (S.K + 7) & ~7; S.actO = dO.act; S.actG = dG.act;
        S.goff = ctx->goff[s];
        S.NG = (int)sd.interface.size();
        // interior subnet over I_o = all outputs the stencils need; one slot-major table per HR chunk
        std::vector<int> posO, posG;
        subnet_hidden(dO, sd.need, P, S.w1O, S.b1O, S.hO, posO);
        std::vector<std::vector<int>> chunk_need;
        std::vector<int> hr_ops;
        chunk_rows(sd, hc, chunk_need, &hr_ops);
        S.hr_chunk = hc;
        S.n_chunks = (int)chunk_need.size();
        S.chunk0 = (int)ctx->hchunk.size();
        S.mmax = 0;
        for (int q = 0; q < S.n_chunks; ++q) {
            ChunkDev c{};
            c.q0 = q * hc;
            c.nq = std::min(hc, S.NB - c.q0);
            c.m = (int)chunk_need[q].size();
            subnet_rows(dO, chunk_need[q], posO, S.Kp, P, c.col, c.val, c.so);
            if (!subnet_tiles(dO, chunk_need[q], posO, S.hO, P, ctx->htiles, c.tile0, c.ntiles)) c.ntiles = 0;
            S.mmax = std::max(S.mmax, c.m);
            ctx->hchunk.push_back(c);
        }
        for (int r : sd.need)
            for (int t = 0; t < dO.K; ++t) ctx->nnzO[s] += dO.cols[(size_t)r * dO.K + t] >= 0;
        // interface subnet over all interface outputs (the WFPC constraint is not hyper-reduced)
        std::vector<int> allG(S.NG);
        for (int r = 0; r < S.NG; ++r) allG[r] = r;
        subnet_hidden(dG, allG, P, S.w1G, S.b1G, S.hG, posG);
        subnet_rows(dG, allG, posG, S.Kp, P, S.colG, S.valG, S.soG);
        if (!subnet_tiles(dG, allG, posG, S.hG, P, ctx->htiles, S.tileG0, S.ntilesG)) S.ntilesG = 0;
        for (int c : dG.cols) ctx->nnzG[s] += c >= 0;
        // the interface outputs the stencils use, with Jacobian rows
        S.NGn = (int)sd.needG.size();
        subnet_rows(dG, sd.needG, posG, S.Kp, P, S.colGn, S.valGn, S.soGn);
        for (int r : sd.needG)
            for (int t = 0; t < dG.K; ++t) ctx->nnzGn[s] += dG.cols[(size_t)r * dG.K + t] >= 0;
        // M_i = C A_i (N^G x n_C), then Q_i^T = (M_i^T diag(scale) W2~)^T (h_G x n_C): D_i = Q_i P_G
        std::vector<double> M((size_t)S.NG * nC, 0.0);
        for (int r = 0; r < ctx->N_A; ++r) {
            if (ctx->con_lo[r] == s) {
                int li = ctx->con_lo_flat[r] - S.goff;
                for (int c = 0; c < nC; ++c) M[(size_t)li * nC + c] += ctx->C[(size_t)c * ctx->N_A + r];
            }
            if (ctx->con_hi[r] == s) {
                int li = ctx->con_hi_flat[r] - S.goff;
                for (int c = 0; c < nC; ++c) M[(size_t)li * nC + c] -= ctx->C[(size_t)c * ctx->N_A + r];
            }
        }
        const int qld = round4(nC);
        std::vector<double> Qt((size_t)S.hG * qld, 0.0);
        for (int r = 0; r < S.NG; ++r)
            for (int t = 0; t < dG.K; ++t) {
                const int col = dG.cols[(size_t)r * dG.K + t];
                if (col < 0) continue;
                const double coef = dG.scale[r] * dG.vals[(size_t)r * dG.K + t];
                double* q = &Qt[(size_t)posG[col] * qld];
                for (int c = 0; c < nC; ++c) q[c] += coef * M[(size_t)r * nC + c];
            }
        S.Qt = P.addv(Qt.data(), Qt.size());
        S.qtc = 0;
        S.hGp = 0;
        if (tsize == 4 && nC <= MAX_NC) ddnm_tile_q_tc(qtc, Qt.data(), S.hG, qld, nC, S.qtc, S.hGp);
        S.pgoff = pg_stride;
        pg_stride += (long long)S.hG * S.nG;
        ctx->max_nG = std::max(ctx->max_nG, S.nG);
        // full decoders and ownership for reconstruction
        S.NO_full = dO.N; S.wO_full = dO.w; S.wG_full = dG.w;
        std::vector<double> so(dO.scale);
        so.insert(so.end(), dO.offset.begin(), dO.offset.end());
        S.fw1O = P.addv(dO.W1.data(), dO.W1.size());
        S.fb1O = P.addv(dO.b1.data(), dO.b1.size());
        std::vector<int> pcol;
        std::vector<double> pval;
        pad_ell(dO, S.K, pcol, pval);
        S.fw2O = P.addv(pval.data(), pval.size());
        S.foutO = P.addv(so.data(), so.size());
        S.fcolO = P.addi(pcol.data(), pcol.size());
        std::vector<double> sg(dG.scale);
        sg.insert(sg.end(), dG.offset.begin(), dG.offset.end());
        S.fw1G = P.addv(dG.W1.data(), dG.W1.size());
        S.fb1G = P.addv(dG.b1.data(), dG.b1.size());
        pad_ell(dG, S.K, pcol, pval);
        S.fw2G = P.addv(pval.data(), pval.size());
        S.foutG = P.addv(sg.data(), sg.size());
        S.fcolG = P.addi(pcol.data(), pcol.size());
        std::vector<int> own, ids;
        for (int v : sd.interior) { own.push_back(std::binary_search(sd.owned.begin(), sd.owned.end(), v % ctx->N) ? 1 : 0); ids.push_back(v); }
        for (int v : sd.interface) { own.push_back(std::binary_search(sd.owned.begin(), sd.owned.end(), v % ctx->N) ? 1 : 0); ids.push_back(v); }
        S.own = P.addi(own.data(), own.size());
        S.ids = P.addi(ids.data(), ids.size());
        S.blk = blk;
        S.phio = s;
        blk += blk_layout(S.ni, S.nG, nC).size;
        for (int o = 0; o < HR_INTS; ++o)            // operand-major: consecutive rows are consecutive ints
            for (int q = 0; q < S.NB; ++q) hr_all.push_back(hr_ops[(size_t)q * HR_INTS + o]);
        S.smem_bytes = eval_smem(S, nC, (int)tsize).bytes;
        ctx->eval_smem = std::max(ctx->eval_smem, S.smem_bytes);
        ctx->rec_smem = std::max(ctx->rec_smem, (int)(std::max(dO.w, dG.w) * tsize));
    }
    // width classes of the evaluation kernel
    ctx->eval_classes.clear();
    std::vector<int> cls;
    for (int ro = 4; ro <= 16; ro += 4)
        for (int rg = 4; rg <= 12; rg += 4) {
            EvalClass c{ro, rg, (int)cls.size(), 0, 0, 0, 1, 0};
            for (int s = 0; s < ns; ++s) {
                const SubDev& S = ctx->hsub[s];
                if (round4(S.nO + 1) == ro && round4(S.nG + 1) == rg) {
                    cls.push_back(s);
                    c.smem = std::max(c.smem, S.smem_bytes);
                }
            }
            c.n = (int)cls.size() - c.off;
            // largest subdomains first: the persistent evaluation hands out items in this order
            auto cost = [&](int s) {
                const SubDev& S = ctx->hsub[s];
                return (double)ctx->nnzO[s] * (S.nO + 1) + (double)ctx->nnzG[s] * (S.nG + 1) +
                       (double)S.NB * S.ni * (S.ni + 6);
            };
            std::stable_sort(cls.begin() + c.off, cls.end(), [&](int a, int b) { return cost(a) > cost(b); });
            c.stride = (c.smem + 127) & ~127;
            c.nt = eval_threads((int)tsize, ro, rg);
            c.groups = std::max(1, std::min({eval_ctas_by_regs((int)tsize, ro, rg), sm_smem / (c.stride + 1024),
                                             dev_max / std::max(c.stride, 1), 1024 / c.nt}));
            if (c.n) ctx->eval_classes.push_back(c);
        }
    if ((int)cls.size() != ns) return ddnm_fail(ctx, DDNM_E_UNSUPPORTED, "latent dims outside the kernel classes");
    if (ctx->eval_smem > dev_max)
        return ddnm_fail(ctx, DDNM_E_UNSUPPORTED, "a subdomain needs " + std::to_string(ctx->eval_smem) +
                                                      " bytes of shared memory (device limit " + std::to_string(dev_max) + ")");
    if (ctx->rec_smem > dev_max) return ddnm_fail(ctx, DDNM_E_UNSUPPORTED, "decoder too wide for reconstruction");
    int fac_stride = 0, sum_nG = 0;
    for (const SubDev& S : ctx->hsub) {
        fac_stride = std::max(fac_stride, S.ni * S.ni + 4 * S.ni + S.nG * S.nG);
        sum_nG += S.nG;
    }
    fac_stride = (fac_stride + 1) & ~1;
    ctx->ss_rows = std::min(sum_nG, std::max(MAX_NG, SS_ROWS_DBL / nC));   // staged rows of W per chunk
    // k_kkt: S, rhs, Atil, pivots, sum u, then one area used in turn by the staging of the Schur sums (W,
    // D_G^{-1} W, u) and Z, T of the border solve (k_factor: fac_stride doubles per subdomain of a CTA)
    const size_t work = std::max({(size_t)3 * ctx->ss_rows * nC,
                                  (size_t)nC * (MAX_MF + 1) + MAX_MF * MAX_MF + 2 * MAX_MF});
    ctx->kkt_smem = (int)(((size_t)nC * nC + 4 * nC + work) * 8);
    if (ctx->kkt_smem > dev_max)
        return ddnm_fail(ctx, DDNM_E_UNSUPPORTED, "KKT step needs " + std::to_string(ctx->kkt_smem) +
                                                      " bytes of shared memory (device limit " + std::to_string(dev_max) + ")");
    // Schur-sum chunks: consecutive subdomains whose interface rows fit the staging area
    std::vector<int> ss_chunk{0};
    {
        int rows = 0;
        for (int i = 0; i < ns; ++i) {
            if (rows + ctx->hsub[i].nG > ctx->ss_rows) {
                ss_chunk.push_back(i);
                rows = 0;
            }
            rows += ctx->hsub[i].nG;
        }
        ss_chunk.push_back(ns);
    }
    const long long ss_chunk_off = P.addi(ss_chunk.data(), ss_chunk.size());
    // upload
    cudaFree(ctx->d_vpool); cudaFree(ctx->d_ipool); cudaFree(ctx->d_hr); cudaFree(ctx->d_con);
    cudaFree(ctx->d_C); cudaFree(ctx->d_bnd_ij); cudaFree(ctx->d_sub); cudaFree(ctx->d_chunk);
    ctx->d_vpool = nullptr; ctx->d_ipool = nullptr; ctx->d_hr = nullptr; ctx->d_con = nullptr;
    ctx->d_C = nullptr; ctx->d_bnd_ij = nullptr; ctx->d_sub = nullptr; ctx->d_chunk = nullptr;
    if (tsize == 8) {
        CK(cudaMalloc(&ctx->d_vpool, P.v.size() * 8));
        CK(cudaMemcpy(ctx->d_vpool, P.v.data(), P.v.size() * 8, cudaMemcpyHostToDevice));
    } else {
        std::vector<float> f(P.v.begin(), P.v.end());
        CK(cudaMalloc(&ctx->d_vpool, f.size() * 4));
        CK(cudaMemcpy(ctx->d_vpool, f.data(), f.size() * 4, cudaMemcpyHostToDevice));
    }
    CK(cudaMalloc(&ctx->d_ipool, std::max<size_t>(P.i.size(), 1) * 4));
    CK(cudaMemcpy(ctx->d_ipool, P.i.data(), P.i.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMalloc(&ctx->d_hr, hr_all.size() * 4));
    CK(cudaMemcpy(ctx->d_hr, hr_all.data(), hr_all.size() * 4, cudaMemcpyHostToDevice));
    std::vector<int> con(ctx->con_lo_flat);
    con.insert(con.end(), ctx->con_hi_flat.begin(), ctx->con_hi_flat.end());
    CK(cudaMalloc(&ctx->d_con, std::max<size_t>(con.size(), 1) * 4));
    CK(cudaMemcpy(ctx->d_con, con.data(), con.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMalloc(&ctx->d_C, std::max<size_t>(ctx->C.size(), 1) * 8));
    CK(cudaMemcpy(ctx->d_C, ctx->C.data(), ctx->C.size() * 8, cudaMemcpyHostToDevice));
    cudaFree(ctx->d_Ahat);
    ctx->d_Ahat = nullptr;
    if (!ahat_all.empty()) {
        CK(cudaMalloc(&ctx->d_Ahat, ahat_all.size() * 8));
        CK(cudaMemcpy(ctx->d_Ahat, ahat_all.data(), ahat_all.size() * 8, cudaMemcpyHostToDevice));
    }
    cudaFree(ctx->d_Qtc);
    ctx->d_Qtc = nullptr;
    if (!qtc.empty()) {
        CK(cudaMalloc(&ctx->d_Qtc, qtc.size() * 4));
        CK(cudaMemcpy(ctx->d_Qtc, qtc.data(), qtc.size() * 4, cudaMemcpyHostToDevice));
    }
    if (!ctx->d_err) {
        CK(cudaMalloc(&ctx->d_err, sizeof(int)));
        CK(cudaMemset(ctx->d_err, 0, sizeof(int)));
    }
    // mixed path: C transposed (constraint row l, then test-matrix row c) and split into two floats per entry,
    // hi = fl32(C) and lo = fl32(C - hi), rows padded with zeros to ldct (the double-float Atil of k_atil_df)
    cudaFree(ctx->d_Ct);
    ctx->d_Ct = nullptr;
    const int ldct = nC <= 32 ? 32 : (nC <= 64 ? 64 : (nC + 127) / 128 * 128);
    if (tsize == 4 && nC > 0) {
        std::vector<float> ct((size_t)2 * ctx->N_A * ldct, 0.f);
        float* lo = ct.data() + (size_t)ctx->N_A * ldct;
        for (int c = 0; c < nC; ++c)
            for (int l = 0; l < ctx->N_A; ++l) {
                const double v = ctx->C[(size_t)c * ctx->N_A + l];
                const float h = (float)v;
                ct[(size_t)l * ldct + c] = h;
                lo[(size_t)l * ldct + c] = (float)(v - (double)h);
            }
        CK(cudaMalloc(&ctx->d_Ct, ct.size() * 4));
        CK(cudaMemcpy(ctx->d_Ct, ct.data(), ct.size() * 4, cudaMemcpyHostToDevice));
    }
    CK(cudaMalloc(&ctx->d_bnd_ij, std::max<size_t>(ctx->bnd_ij.size(), 1) * 4));
    CK(cudaMemcpy(ctx->d_bnd_ij, ctx->bnd_ij.data(), ctx->bnd_ij.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMalloc(&ctx->d_sub, ns * sizeof(SubDev)));
    CK(cudaMemcpy(ctx->d_sub, ctx->hsub.data(), ns * sizeof(SubDev), cudaMemcpyHostToDevice));
    cudaFree(ctx->d_classes);
    ctx->d_classes = nullptr;
    CK(cudaMalloc(&ctx->d_classes, cls.size() * sizeof(int)));
    CK(cudaMemcpy(ctx->d_classes, cls.data(), cls.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMalloc(&ctx->d_chunk, std::max<size_t>(ctx->hchunk.size(), 1) * sizeof(ChunkDev)));
    CK(cudaMemcpy(ctx->d_chunk, ctx->hchunk.data(), ctx->hchunk.size() * sizeof(ChunkDev), cudaMemcpyHostToDevice));
    cudaFree(ctx->d_tiles);
    ctx->d_tiles = nullptr;
    CK(cudaMalloc(&ctx->d_tiles, std::max<size_t>(ctx->htiles.size(), 1) * sizeof(TileDev)));
    if (!ctx->htiles.empty())
        CK(cudaMemcpy(ctx->d_tiles, ctx->htiles.data(), ctx->htiles.size() * sizeof(TileDev), cudaMemcpyHostToDevice));

    ProbDev& pd = ctx->pd;
    pd = ProbDev{};
    pd.n_sub = ns; pd.n_D = ctx->n_D; pd.n_C = nC; pd.N_A = ctx->N_A;
    pd.sum_NG = ctx->sum_NG; pd.sum_NB = ctx->sum_NB; pd.n_bnd = (int)ctx->bnd_ij.size() / 2;
    pd.N_x = 2 * ctx->N; pd.nx = ctx->nx; pd.ny = ctx->ny;
    pd.fac_stride = fac_stride;
    pd.ss_rows = ctx->ss_rows;
    pd.n_ss_chunks = (int)ss_chunk.size() - 1;
    pd.ss_chunk = ctx->d_ipool + ss_chunk_off;
    // factorisation CTAs of k_constraint (8 subdomains each): their Schur-sum shares when the staging of W,
    // D_G^{-1} W and u fits FAC_SHARE_SMEM, else the KKT step sums the blocks
    pd.nfc = (ns + 2 * FAC_WARPS - 1) / (2 * FAC_WARPS);
    pd.fac_rows = 0;
    for (int f = 0; f < pd.nfc; ++f) {
        int rows = 0;
        for (int i = 2 * FAC_WARPS * f; i < std::min(ns, 2 * FAC_WARPS * (f + 1)); ++i) rows += ctx->hsub[i].nG;
        pd.fac_rows = std::max(pd.fac_rows, rows);
    }
    {
        const size_t share = (size_t)(2 * pd.fac_rows + 2 * FAC_WARPS) * nC * 8;
        ctx->fac_share = share <= (size_t)FAC_SHARE_SMEM;
        ctx->fac_smem = (int)std::max((size_t)2 * FAC_WARPS * fac_stride * 8, ctx->fac_share ? share : 0);
    }
    pd.Spart = nullptr;            // set by ddnm_reserve when the shares are formed
    pd.con_split = CON_SPLIT;
    pd.n_split = (ctx->N_A + CON_SPLIT - 1) / CON_SPLIT;
    // A block pivot at or below piv_eps times the block's largest diagonal entry is a rounding remainder of a
    // direction the collocation rows do not see: the block is treated as singular there.  The scale is the
    // relative rounding of H_i (FP64 sums, or FP32 sums in the mixed path) times a safety factor.
    pd.piv_eps = ctx->precision == DDNM_FP64 ? 1e-11 : 1e-5;
    pd.hx = ctx->hx; pd.hy = ctx->hy; pd.nu = ctx->nu; pd.bx0 = ctx->box[0]; pd.by0 = ctx->box[2];
    pd.cst[0] = 0.5 / ctx->hx;
    pd.cst[1] = 0.5 / ctx->hy;
    pd.cst[2] = ctx->nu / (ctx->hx * ctx->hx);
    pd.cst[3] = ctx->nu / (ctx->hy * ctx->hy);
    for (int k = 0; k < 4; ++k) pd.cstf[k] = (float)pd.cst[k];
    pd.blk_stride = blk;
    pd.qld = round4(nC);
    {
        long long big = 0;
        for (const SubDev& S : ctx->hsub) big = std::max(big, (long long)S.hG * nC);
        ctx->dgemm_auto = big >= 65536 ? 1 : 0;
    }
    ctx->atil_auto = (long long)nC * ctx->N_A >= (1LL << 20) ? 1 : 0;
    pd.ldct = ldct;
    pd.Cthi = ctx->d_Ct;
    pd.Ctlo = ctx->d_Ct ? ctx->d_Ct + (size_t)ctx->N_A * ldct : nullptr;
    pd.atil_df = 0;
    pd.Qtc = ctx->d_Qtc;
    pd.srpc = ctx->srpc ? 1 : 0;
    pd.Ahat = ctx->d_Ahat;
    pd.err = ctx->d_err;
    pd.pg_stride = std::max(pg_stride, 1LL);
    pd.sub = ctx->d_sub; pd.chunk = ctx->d_chunk; pd.tiles = ctx->d_tiles; pd.vpool = ctx->d_vpool; pd.ipool = ctx->d_ipool;
    pd.hr = ctx->d_hr;
    pd.con_lo = ctx->d_con; pd.con_hi = ctx->d_con + ctx->N_A; pd.C = ctx->d_C; pd.bnd_ij = ctx->d_bnd_ij;
    ctx->cap_B = 0;   // workspace pointers are re-carved on the next reserve
    ++ctx->gen;
    ctx->finalized = true;
    return DDNM_OK;
}

// Workspace for B instances: one allocation, carved into the per-instance arrays.
int ddnm_reserve(ddnm_ctx* ctx, int B) {
    ProbDev& pd = ctx->pd;
    if (B <= ctx->cap_B && ctx->d_ws) return DDNM_OK;
    int cap = std::max(B, 2 * ctx->cap_B);
    const size_t tsize = ctx->precision == DDNM_FP64 ? 8 : 4;
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    size_t o = 0;
    size_t o_mu = o; o = al(o + (size_t)cap * 2 * 8);
    size_t o_x = o; o = al(o + (size_t)cap * pd.n_D * 8);
    size_t o_lam = o; o = al(o + (size_t)cap * pd.n_C * 8);
    size_t o_xt = o; o = al(o + (size_t)cap * pd.n_D * 8);
    size_t o_lamt = o; o = al(o + (size_t)cap * pd.n_C * 8);
    size_t o_s = o; o = al(o + (size_t)cap * pd.n_D * 8);
    size_t o_slam = o; o = al(o + (size_t)cap * pd.n_C * 8);
    const size_t max_split = ((size_t)pd.N_A + MIN_CON_SPLIT - 1) / MIN_CON_SPLIT;   // any con_split of the plan
    size_t o_At = o; o = al(o + (size_t)cap * max_split * pd.n_C * 8);
    size_t o_Ss = o; o = al(o + (ctx->fac_share ? (size_t)cap * pd.nfc * ((size_t)pd.n_C * (pd.n_C + 1) / 2 + pd.n_C) * 8 : 0));
    size_t o_dst = o; o = al(o + (size_t)cap * INST_DBLS * 8);
    size_t o_ist = o; o = al(o + (size_t)cap * INST_INTS * 4);
    size_t o_bnd = o; o = al(o + (size_t)cap * std::max(pd.n_bnd, 1) * 2 * tsize);
    size_t o_gG = o; o = al(o + (size_t)cap * pd.sum_NG * tsize);
    size_t o_PG = o; o = al(o + (size_t)cap * pd.pg_stride * tsize);
    size_t o_blk = o; o = al(o + (size_t)cap * pd.blk_stride * 8);
    size_t o_act = o; o = al(o + (size_t)CTL_INTS * 4);
    cudaFree(ctx->d_ws);
    ctx->d_ws = nullptr;
    ctx->cap_B = 0;
    CK(cudaSetDevice(ctx->device));
    cudaError_t e = cudaMalloc(&ctx->d_ws, o);
    if (e != cudaSuccess) return ddnm_fail(ctx, DDNM_E_NOMEM, std::string("workspace: ") + cudaGetErrorString(e));
    if (!ctx->h_active) CK(cudaMallocHost(&ctx->h_active, 64));
    char* base = (char*)ctx->d_ws;
    pd.mu = (double*)(base + o_mu);
    pd.x = (double*)(base + o_x);
    pd.lam = (double*)(base + o_lam);
    pd.xt = (double*)(base + o_xt);
    pd.lamt = (double*)(base + o_lamt);
    pd.s = (double*)(base + o_s);
    pd.slam = (double*)(base + o_slam);
    pd.Atil = (double*)(base + o_At);
    pd.Spart = ctx->fac_share ? (double*)(base + o_Ss) : nullptr;
    pd.dst = (double*)(base + o_dst);
    pd.ist = (int*)(base + o_ist);
    pd.bnd = (void*)(base + o_bnd);
    pd.gG = (void*)(base + o_gG);
    pd.PG = (void*)(base + o_PG);
    pd.blk = (double*)(base + o_blk);
    pd.active = (int*)(base + o_act);
    pd.pass = pd.active + MAX_CHAINS;
    pd.ctr = pd.pass + MAX_CHAINS;
    pd.arrive = pd.ctr + MAX_CHAINS * MAX_CLASSES;
    ctx->cap_B = cap;
    ++ctx->gen;   // captured solve graphs hold workspace pointers
    return DDNM_OK;
}

// ------------------------------------------------------------------- work counts

extern "C" int ddnm_get_work(ddnm_ctx* ctx, ddnm_work* out) {
    if (!ctx || !out) return DDNM_E_INVALID;
    if (!ctx->finalized) {
        int rc = ddnm_finalize(ctx);
        if (rc) return rc;
    }
    const double nC = ctx->n_C, tsz = ctx->precision == DDNM_FP64 ? 8.0 : 4.0;
    double f = 0, f64 = 0, bytes = 0, step = 0, fac = 0, table = 0, inst = 0;
    for (int s = 0; s < ctx->n_sub; ++s) {
        const SubDev& S = ctx->hsub[s];
        const double ni = S.ni, nO = S.nO, nG = S.nG;
        const double mO = (double)ctx->subs[s].need.size();   // |I_o|: distinct interior outputs the stencils use
        // hidden layers: z = W1 x + b1 (2 h n), P = sigma'(z) W1 (h n)
        f += 3.0 * (S.hO * nO + S.hG * nG);
        // outputs and Jacobian rows over the mask nonzeros, then de-normalisation
        // (interior: values and Jacobian rows of the needed outputs; interface: values of every output,
        // Jacobian rows of the needed ones)
        f += 2.0 * ctx->nnzO[s] * (nO + 1) + 2.0 * ctx->nnzG[s] + 2.0 * ctx->nnzGn[s] * nG + mO * (nO + 2) +
             2.0 * S.NG + S.NGn * nG;
        // residual row, 6 partials, chain rule R = sum_o d_o J_o
        f += S.NB * (30.0 + 12.0 * ni);
        // H = R^T R (upper triangle) and R^T r
        f += 2.0 * S.NB * (ni * (ni + 1) / 2 + ni);
        // D_i = Q_i P_G over the interface hidden units
        f += 2.0 * nC * S.hG * nG;
        // FP64 in the evaluation: rho += D^T lambda, ||rho_i||^2
        f64 += 2 * nC * nG + 2 * ni;
        // FP64 at an accepted point: L D L^T, t, W = L_GG^{-1} D^T, u (k_factor); lower triangle of
        // W^T D_G^{-1} W summed into S (k_ssum)
        fac += ni * ni * ni / 3.0 + ni * ni + nC * nG * nG + 3 * nC * nG + nC * (nC + 1) * nG + nC;
        // bytes shared by all instances (read once per launch at best): the subnet weights, the mask values
        // and columns of the needed rows, scale/offset, Q_i, the collocation-row table
        const double shared = tsz * (S.hO * (nO + 1) + S.hG * (nG + 1) + ctx->nnzO[s] + ctx->nnzG[s] +
                                     2.0 * (mO + S.NG) + (double)S.hG * nC) +
                              4.0 * (mO * S.K + (double)S.NG * S.K + 7.0 * S.NB);
        // bytes of one instance: the block outputs H, rho, D (FP64), the interface values, the Dirichlet
        // values its stencils read
        const double own = 8.0 * (ni * ni + ni + nC * nG) + tsz * S.NG;
        table += shared;
        inst += own;
        bytes += shared + own;
        // back-substitution per subdomain (in the next evaluation)
        step += 2.0 * nG * nC + ni * ni;
    }
    const double lat = 8.0 * (ctx->n_D + nC + 2) + tsz * 2.0 * ctx->bnd_ij.size() / 2;   // latents, lambda, mu, Dirichlet
    bytes += lat;
    inst += lat;
    step += nC * nC * nC / 3.0 + 2.0 * nC * nC;
    out->table_bytes = table;
    out->instance_bytes = inst;
    out->eval_flops = f;
    out->eval_fp64_flops = f64;
    out->eval_bytes = bytes;
    out->constraint_fp64_flops = 2.0 * nC * ctx->N_A + ctx->N_A;
    out->step_fp64_flops = step + fac;
    return DDNM_OK;
}
