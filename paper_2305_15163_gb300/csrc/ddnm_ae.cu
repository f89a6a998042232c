// sm_103a offline training of the sparse-masked shallow autoencoders (Sec. 3.4 "Nonlinear-manifold ROM",
// Sec. 5.1, Sec. 7.2-7.3): for every subdomain, one autoencoder for its interior states and one for its
// interface states, trained on FOM snapshots restricted to those states ("top-down").
//
// For one autoencoder with N states and width w (masks: Wd2 the three-band decoder mask, We1 its transpose):
//   xt = (x - offset) / scale                (normalisation onto [-1, 1] over the training snapshots)
//   z1 = We1 xt + be1, a1 = sigma(z1), xh = We2 a1            (encoder, Eq. autoencoder_architecture a/c)
//   z2 = Wd1 xh + bd1, a2 = sigma(z2), y = Wd2 a2             (decoder, Eq. autoencoder_architecture b/d)
//   L = (1/n_b) sum_b || y_b - xt_b ||^2                      (Eq. autoencoder_AbsMSE_loss on the batch)
// trained by mini-batch Adam.  The trained decoder, with the de-normalisation offset + scale o y, replaces
// the context's decoder, so the next solve uploads it.
//
// All 2 n_sub autoencoders of the context train together, one set of launches per mini-batch, each launch
// spanning every autoencoder through a flat row table:
//   k_ae_gather   xt of the batch (FP64 normalisation, FP32 result)
//   k_ae_enc      z1, a1: a warp per hidden unit, lanes over its (transposed-mask) inputs, the n_b samples of
//                 the batch in registers so that every weight is read once per batch
//   k_ae_lat      xh = We2 a1: a warp per (autoencoder, latent coordinate)
//   k_ae_dec1     z2, a2: a thread per (hidden unit, sample)
//   k_ae_out      y, the loss, dL/dy and dL/dWd2: a thread per output row, its mask slots in registers
//   k_ae_back2    dL/da2 = Wd2^T dL/dy through the transposed mask (a warp per hidden unit, no atomics),
//                 dL/dz2, dL/dWd1, dL/dbd1
//   k_ae_glat     dL/dxh = Wd1^T dL/dz2: a warp per (autoencoder, latent coordinate)
//   k_ae_back1    dL/dWe2, dL/da1 = We2^T dL/dxh, dL/dz1, dL/dbe1: a thread per hidden unit
//   k_ae_enc_grad dL/dWe1 on the transposed mask: a warp per hidden unit
//   k_ae_adam     Adam on the flat FP32 parameter vector (padding slots have zero gradient and stay zero)
// Every sum runs in a fixed order: results are reproducible bit for bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "ddnm_ctx.h"

namespace {

constexpr int AE_MAXB = 32;      // largest mini-batch
constexpr int AE_T = 256;

struct AeDev {
    int N, w, n, K, Kt, act;
    int row0, hid0;              // first output row / hidden unit of this autoencoder in the flat tables
    long long pWe1, pbe1, pWe2, pWd1, pbd1, pWd2, nP;   // parameter offsets (floats) and count
    long long iColsT, iTslot, iCols, iIds;              // int-table offsets
};

struct EncoderHost {
    bool loaded = false;
    int N = 0, w = 0, n = 0, Kt = 0;
    std::vector<int> cols;       // w x Kt
    std::vector<double> vals, b1, W2;
};

struct AeState {
    std::vector<EncoderHost> enc;          // 2 n_sub: interior of s at 2s, interface at 2s + 1
    std::vector<AeDev> hae;
    int n_ae = 0, R = 0, H = 0, Nmax = 0;  // outputs and hidden units over all autoencoders
    long long P = 0, I = 0;
    AeDev* d_ae = nullptr;
    int* d_int = nullptr;        // colsT, tslot, cols, ids of every autoencoder
    int* d_row_ae = nullptr;     // R: autoencoder of each flat output row
    int* d_hid_ae = nullptr;     // H: autoencoder of each flat hidden unit
    float* p = nullptr;          // parameters (FP32 master)
    float* g = nullptr;          // gradient
    float* m = nullptr;
    float* v = nullptr;
    double* off = nullptr;       // R normalisation offsets
    double* sc = nullptr;        // R scales
    float* xt = nullptr;         // AE_MAXB x R   normalised batch (sample-major per autoencoder: row0*nb + b*N + r)
    float* gy = nullptr;         // AE_MAXB x R   dL/dy
    float* z1 = nullptr;         // AE_MAXB x H
    float* a1 = nullptr;
    float* z2 = nullptr;
    float* a2 = nullptr;
    float* gz2 = nullptr;
    float* gz1 = nullptr;
    float* lat = nullptr;        // AE_MAXB x n_ae x 16
    float* glat = nullptr;
    double* loss = nullptr;      // n_ae x (R / AE_T + n_ae) block partials of the loss
    int loss_slots = 0;
    double* snap = nullptr;      // n_snap x N_x snapshots on the device
    int snap_cap = 0;
    int* d_idx = nullptr;        // AE_MAXB sample ids of the batch
    long long steps = 0;         // Adam steps taken
    bool ready = false;
};

__device__ __forceinline__ void act_fn(int act, float z, float& s, float& ds) {
    if (act == DDNM_ACT_SWISH) {
        const float g = 1.f / (1.f + expf(-z));
        s = z * g;
        ds = g + z * g * (1.f - g);
    } else if (act == DDNM_ACT_SIGMOID) {
        const float g = 1.f / (1.f + expf(-z));
        s = g;
        ds = g * (1.f - g);
    } else {
        s = z;
        ds = 1.f;
    }
}

__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// activation offset of autoencoder `a` (sample-major): rows of the batch lie at base * nb + b * size + r
__device__ __forceinline__ size_t aoff(int base, int nb, int b, int size, int r) {
    return (size_t)base * nb + (size_t)b * size + r;
}

// min / max of every state over the snapshots -> normalisation of each autoencoder row (FP64)
__global__ void k_ae_norm(const AeDev* ae, const int* row_ae, const int* itab, const double* snap, int n_snap, int Nx,
                          int R, double* off, double* sc) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const AeDev A = ae[row_ae[r]];
    const int id = itab[A.iIds + (r - A.row0)];
    double lo = snap[id], hi = snap[id];
    for (int k = 1; k < n_snap; ++k) {
        const double x = snap[(size_t)k * Nx + id];
        lo = fmin(lo, x);
        hi = fmax(hi, x);
    }
    const double s = 0.5 * (hi - lo);
    off[r] = 0.5 * (hi + lo);
    sc[r] = s > 0.0 ? s : 1.0;
}

__global__ void k_ae_gather(const AeDev* ae, const int* row_ae, const int* itab, const double* snap, int Nx,
                            const int* idx, int nb, int R, const double* off, const double* sc, float* xt) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const AeDev A = ae[row_ae[r]];
    const int loc = r - A.row0;
    const int id = itab[A.iIds + loc];
    for (int b = 0; b < nb; ++b)
        xt[aoff(A.row0, nb, b, A.N, loc)] = (float)((snap[(size_t)idx[b] * Nx + id] - off[r]) / sc[r]);
}

// z1 = We1 xt + be1, a1 = sigma(z1): a warp per flat hidden unit
template <int NB>
__global__ void k_ae_enc(const AeDev* ae, const int* hid_ae, const int* itab, const float* p, const float* xt, int nb,
                         int H, float* z1, float* a1) {
    const int h = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x % 32;
    if (h >= H) return;
    const AeDev A = ae[hid_ae[h]];
    const int j = h - A.hid0;
    const int* cols = itab + A.iColsT + (size_t)j * A.Kt;
    const float* vals = p + A.pWe1 + (size_t)j * A.Kt;
    float acc[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) acc[b] = 0.f;
    for (int k = lane; k < A.Kt; k += 32) {
        const int c = cols[k];
        if (c < 0) break;
        const float w = vals[k];
#pragma unroll
        for (int b = 0; b < NB; ++b)
            if (b < nb) acc[b] = fmaf(w, xt[aoff(A.row0, nb, b, A.N, c)], acc[b]);
    }
    const float bias = p[A.pbe1 + j];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        if (b >= nb) break;
        const float z = warp_sumf(acc[b]) + bias;
        if (lane == 0) {
            float s, ds;
            act_fn(A.act, z, s, ds);
            z1[aoff(A.hid0, nb, b, A.w, j)] = z;
            a1[aoff(A.hid0, nb, b, A.w, j)] = s;
        }
    }
}

// xh = We2 a1: a warp per (autoencoder, latent coordinate l)
template <int NB>
__global__ void k_ae_lat(const AeDev* ae, int n_ae, const float* p, const float* a1, int nb, float* lat) {
    const int q = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x % 32;
    const int a = q / 16, l = q % 16;
    if (a >= n_ae) return;
    const AeDev A = ae[a];
    if (l >= A.n) return;
    float acc[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) acc[b] = 0.f;
    const float* W = p + A.pWe2 + (size_t)l * A.w;
    for (int j = lane; j < A.w; j += 32) {
        const float w = W[j];
#pragma unroll
        for (int b = 0; b < NB; ++b)
            if (b < nb) acc[b] = fmaf(w, a1[aoff(A.hid0, nb, b, A.w, j)], acc[b]);
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        if (b >= nb) break;
        const float s = warp_sumf(acc[b]);
        if (lane == 0) lat[((size_t)a * AE_MAXB + b) * 16 + l] = s;
    }
}

// z2 = Wd1 xh + bd1, a2 = sigma(z2): a thread per (flat hidden unit, sample)
__global__ void k_ae_dec1(const AeDev* ae, const int* hid_ae, const float* p, const float* lat, int nb, int H,
                          float* z2, float* a2) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)H * nb) return;
    const int h = (int)(t / nb), b = (int)(t % nb);
    const int ai = hid_ae[h];
    const AeDev A = ae[ai];
    const int j = h - A.hid0;
    float z = p[A.pbd1 + j];
    const float* W = p + A.pWd1 + (size_t)j * A.n;
    const float* x = lat + ((size_t)ai * AE_MAXB + b) * 16;
    for (int l = 0; l < A.n; ++l) z = fmaf(W[l], x[l], z);
    float s, ds;
    act_fn(A.act, z, s, ds);
    z2[aoff(A.hid0, nb, b, A.w, j)] = z;
    a2[aoff(A.hid0, nb, b, A.w, j)] = s;
}

// y = Wd2 a2, e = y - xt, loss, dL/dy = 2 e / n_b, dL/dWd2: a thread per flat output row
template <int NB>
__global__ void k_ae_out(const AeDev* ae, const int* row_ae, const int* itab, const float* p, const float* a2,
                         const float* xt, int nb, int R, float* gy, float* g, double* loss_part) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    __shared__ double red[AE_T];
    double my = 0.0;
    int ai = -1;
    if (r < R) {
        ai = row_ae[r];
        const AeDev A = ae[ai];
        const int loc = r - A.row0;
        const int* cols = itab + A.iCols + (size_t)loc * A.K;
        const float* vals = p + A.pWd2 + (size_t)loc * A.K;
        float e[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) e[b] = 0.f;
        for (int k = 0; k < A.K; ++k) {
            const int c = cols[k];
            if (c < 0) break;
            const float w = vals[k];
#pragma unroll
            for (int b = 0; b < NB; ++b)
                if (b < nb) e[b] = fmaf(w, a2[aoff(A.hid0, nb, b, A.w, c)], e[b]);
        }
        const float s2 = 2.f / nb;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            if (b >= nb) break;
            const float d = e[b] - xt[aoff(A.row0, nb, b, A.N, loc)];
            my += (double)d * d;
            e[b] = s2 * d;
            gy[aoff(A.row0, nb, b, A.N, loc)] = e[b];
        }
        float* gw = g + A.pWd2 + (size_t)loc * A.K;
        for (int k = 0; k < A.K; ++k) {
            const int c = cols[k];
            if (c < 0) {
                gw[k] = 0.f;
                continue;
            }
            float acc = 0.f;
#pragma unroll
            for (int b = 0; b < NB; ++b)
                if (b < nb) acc = fmaf(e[b], a2[aoff(A.hid0, nb, b, A.w, c)], acc);
            gw[k] = acc;
        }
    }
    // loss partials of this block, per autoencoder (a block spans at most a few autoencoders): the sum of the
    // block's rows that belong to autoencoder a0 = the block's first row's autoencoder goes to slot
    // (a0, block); other autoencoders of the block are rare (block straddling a boundary) and use the
    // (a, block) slot of their own
    red[threadIdx.x] = my;
    __syncthreads();
    if (threadIdx.x == 0) {
        const int r0 = blockIdx.x * blockDim.x;
        int cur = -1;
        double s = 0.0;
        for (int t = 0; t < (int)blockDim.x && r0 + t < R; ++t) {
            const int a = row_ae[r0 + t];
            if (a != cur) {
                if (cur >= 0) loss_part[(size_t)cur * gridDim.x + blockIdx.x] = s;
                cur = a;
                s = 0.0;
            }
            s += red[t];
        }
        if (cur >= 0) loss_part[(size_t)cur * gridDim.x + blockIdx.x] = s;
    }
}

// dL/da2 = Wd2^T dL/dy through the transposed mask, dL/dz2 = dL/da2 o sigma'(z2), dL/dWd1, dL/dbd1:
// a warp per flat hidden unit
template <int NB>
__global__ void k_ae_back2(const AeDev* ae, const int* hid_ae, const int* itab, const float* p, const float* gy,
                           const float* z2, const float* lat, int nb, int H, float* gz2, float* g) {
    const int h = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x % 32;
    if (h >= H) return;
    const int ai = hid_ae[h];
    const AeDev A = ae[ai];
    const int j = h - A.hid0;
    const int* rows = itab + A.iColsT + (size_t)j * A.Kt;
    const int* slot = itab + A.iTslot + (size_t)j * A.Kt;
    float acc[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) acc[b] = 0.f;
    for (int k = lane; k < A.Kt; k += 32) {
        const int r = rows[k];
        if (r < 0) break;
        const float w = p[A.pWd2 + slot[k]];
#pragma unroll
        for (int b = 0; b < NB; ++b)
            if (b < nb) acc[b] = fmaf(w, gy[aoff(A.row0, nb, b, A.N, r)], acc[b]);
    }
    float gz[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        gz[b] = 0.f;
        if (b >= nb) continue;
        const float ga = warp_sumf(acc[b]);
        float s, ds;
        act_fn(A.act, z2[aoff(A.hid0, nb, b, A.w, j)], s, ds);
        gz[b] = ga * ds;
        if (lane == 0) gz2[aoff(A.hid0, nb, b, A.w, j)] = gz[b];
    }
    // dL/dWd1[j, l] = sum_b gz2_b lat_b[l]; dL/dbd1[j] = sum_b gz2_b (lanes over l)
    if (lane < A.n) {
        float s = 0.f;
        for (int b = 0; b < nb; ++b) s = fmaf(gz[b], lat[((size_t)ai * AE_MAXB + b) * 16 + lane], s);
        g[A.pWd1 + (size_t)j * A.n + lane] = s;
    }
    if (lane == 0) {
        float s = 0.f;
        for (int b = 0; b < nb; ++b) s += gz[b];
        g[A.pbd1 + j] = s;
    }
}

// dL/dxh = Wd1^T dL/dz2: a warp per (autoencoder, latent coordinate l)
template <int NB>
__global__ void k_ae_glat(const AeDev* ae, int n_ae, const float* p, const float* gz2, int nb, float* glat) {
    const int q = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x % 32;
    const int a = q / 16, l = q % 16;
    if (a >= n_ae) return;
    const AeDev A = ae[a];
    if (l >= A.n) return;
    float acc[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) acc[b] = 0.f;
    for (int j = lane; j < A.w; j += 32) {
        const float w = p[A.pWd1 + (size_t)j * A.n + l];
#pragma unroll
        for (int b = 0; b < NB; ++b)
            if (b < nb) acc[b] = fmaf(w, gz2[aoff(A.hid0, nb, b, A.w, j)], acc[b]);
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        if (b >= nb) break;
        const float s = warp_sumf(acc[b]);
        if (lane == 0) glat[((size_t)a * AE_MAXB + b) * 16 + l] = s;
    }
}

// dL/dWe2[l, j] = sum_b glat_b[l] a1_b[j]; dL/da1 = We2^T glat; dL/dz1 = dL/da1 o sigma'(z1); dL/dbe1:
// a thread per flat hidden unit
__global__ void k_ae_back1(const AeDev* ae, const int* hid_ae, const float* p, const float* glat, const float* z1,
                           const float* a1, int nb, int H, float* gz1, float* g) {
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= H) return;
    const int ai = hid_ae[h];
    const AeDev A = ae[ai];
    const int j = h - A.hid0;
    const float* gl = glat + (size_t)ai * AE_MAXB * 16;
    for (int l = 0; l < A.n; ++l) {
        float s = 0.f;
        for (int b = 0; b < nb; ++b) s = fmaf(gl[b * 16 + l], a1[aoff(A.hid0, nb, b, A.w, j)], s);
        g[A.pWe2 + (size_t)l * A.w + j] = s;
    }
    float gb = 0.f;
    for (int b = 0; b < nb; ++b) {
        float ga = 0.f;
        for (int l = 0; l < A.n; ++l) ga = fmaf(p[A.pWe2 + (size_t)l * A.w + j], gl[b * 16 + l], ga);
        float s, ds;
        act_fn(A.act, z1[aoff(A.hid0, nb, b, A.w, j)], s, ds);
        const float gz = ga * ds;
        gz1[aoff(A.hid0, nb, b, A.w, j)] = gz;
        gb += gz;
    }
    g[A.pbe1 + j] = gb;
}

// dL/dWe1[j, k] = sum_b gz1_b[j] xt_b[colsT[j, k]]: a warp per flat hidden unit
template <int NB>
__global__ void k_ae_enc_grad(const AeDev* ae, const int* hid_ae, const int* itab, const float* xt, const float* gz1,
                              int nb, int H, float* g) {
    const int h = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x % 32;
    if (h >= H) return;
    const AeDev A = ae[hid_ae[h]];
    const int j = h - A.hid0;
    float gz[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) gz[b] = b < nb ? gz1[aoff(A.hid0, nb, b, A.w, j)] : 0.f;
    const int* cols = itab + A.iColsT + (size_t)j * A.Kt;
    float* gw = g + A.pWe1 + (size_t)j * A.Kt;
    for (int k = lane; k < A.Kt; k += 32) {
        const int c = cols[k];
        if (c < 0) {
            gw[k] = 0.f;
            continue;
        }
        float s = 0.f;
#pragma unroll
        for (int b = 0; b < NB; ++b)
            if (b < nb) s = fmaf(gz[b], xt[aoff(A.row0, nb, b, A.N, c)], s);
        gw[k] = s;
    }
}

__global__ void k_ae_adam(float* p, const float* g, float* m, float* v, long long n, float lr, float b1, float b2,
                          float eps, float bc1, float bc2) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const float gk = g[k];
        const float mk = b1 * m[k] + (1.f - b1) * gk;
        const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
        m[k] = mk;
        v[k] = vk;
        p[k] -= lr * (mk / bc1) / (sqrtf(vk / bc2) + eps);
    }
}

int afail(ddnm_ctx* ctx, cudaError_t e, const char* what) {
    return ddnm_fail(ctx, DDNM_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define AK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return afail(ctx, e_, #call);       \
    } while (0)

AeState* ae_state(ddnm_ctx* ctx) {
    if (!ctx->ae) {
        AeState* S = new AeState();
        S->enc.resize(2 * ctx->n_sub);
        ctx->ae = S;
    }
    return (AeState*)ctx->ae;
}

void ae_free_device(AeState* S) {
    for (void* q : {(void*)S->d_ae, (void*)S->d_int, (void*)S->d_row_ae, (void*)S->d_hid_ae, (void*)S->p, (void*)S->g,
                    (void*)S->m, (void*)S->v, (void*)S->off, (void*)S->sc, (void*)S->xt, (void*)S->gy, (void*)S->z1,
                    (void*)S->a1, (void*)S->z2, (void*)S->a2, (void*)S->gz2, (void*)S->gz1, (void*)S->lat,
                    (void*)S->glat, (void*)S->loss, (void*)S->snap, (void*)S->d_idx})
        cudaFree(q);
    S->d_ae = nullptr;
    S->d_int = S->d_row_ae = S->d_hid_ae = S->d_idx = nullptr;
    S->p = S->g = S->m = S->v = S->xt = S->gy = S->z1 = S->a1 = S->z2 = S->a2 = S->gz2 = S->gz1 = S->lat = S->glat = nullptr;
    S->off = S->sc = S->loss = S->snap = nullptr;
    S->snap_cap = 0;
    S->ready = false;
}

// the decoder of autoencoder a (2 s + kind)
DecoderHost& dec_of(ddnm_ctx* ctx, int a) { return (a % 2 == 0 ? ctx->decO : ctx->decG)[a / 2]; }

// upload the initial weights (loaded decoders and encoders) and the index tables of every autoencoder
int ae_setup(ddnm_ctx* ctx, AeState* S) {
    const int n_ae = 2 * ctx->n_sub;
    for (int a = 0; a < n_ae; ++a) {
        if (!dec_of(ctx, a).loaded || !S->enc[a].loaded)
            return ddnm_fail(ctx, DDNM_E_STATE, "autoencoder training needs the decoder and the encoder of every "
                                                "subdomain and kind loaded (subdomain " + std::to_string(a / 2) + ")");
    }
    ae_free_device(S);
    S->n_ae = n_ae;
    S->hae.assign(n_ae, AeDev{});
    std::vector<float> P;
    std::vector<int> I, row_ae, hid_ae;
    auto padP = [&]() { while (P.size() % 4) P.push_back(0.f); };
    auto padI = [&]() { while (I.size() % 4) I.push_back(-1); };
    int R = 0, H = 0;
    S->Nmax = 0;
    for (int a = 0; a < n_ae; ++a) {
        const DecoderHost& d = dec_of(ctx, a);
        const EncoderHost& e = S->enc[a];
        const SubHost& sd = ctx->subs[a / 2];
        const std::vector<int>& ids = a % 2 == 0 ? sd.interior : sd.interface;
        AeDev A{};
        A.N = d.N; A.w = d.w; A.n = d.n; A.K = d.K; A.Kt = e.Kt; A.act = d.act;
        A.row0 = R; A.hid0 = H;
        padP();
        A.pWe1 = (long long)P.size();
        for (double x : e.vals) P.push_back((float)x);
        padP(); A.pbe1 = (long long)P.size();
        for (double x : e.b1) P.push_back((float)x);
        padP(); A.pWe2 = (long long)P.size();
        for (double x : e.W2) P.push_back((float)x);
        padP(); A.pWd1 = (long long)P.size();
        for (double x : d.W1) P.push_back((float)x);
        padP(); A.pbd1 = (long long)P.size();
        for (double x : d.b1) P.push_back((float)x);
        padP(); A.pWd2 = (long long)P.size();
        for (size_t k = 0; k < d.vals.size(); ++k) P.push_back(d.cols[k] >= 0 ? (float)d.vals[k] : 0.f);
        padP();
        A.nP = (long long)P.size() - A.pWe1;
        // tslot[j][t]: the flat Wd2 slot r K + k whose column is j, for the t-th row r of the transposed mask
        std::vector<int> tslot((size_t)A.w * A.Kt, -1);
        std::vector<int> fill(A.w, 0);
        for (int r = 0; r < A.N; ++r)
            for (int k = 0; k < A.K; ++k) {
                const int c = d.cols[(size_t)r * A.K + k];
                if (c < 0) break;
                const int t = fill[c]++;
                if (t >= A.Kt || e.cols[(size_t)c * A.Kt + t] != r)
                    return ddnm_fail(ctx, DDNM_E_INVALID, "encoder mask of autoencoder " + std::to_string(a) +
                                                              " is not the transpose of its decoder's mask");
                tslot[(size_t)c * A.Kt + t] = r * A.K + k;
            }
        for (int c = 0; c < A.w; ++c)
            if (fill[c] < A.Kt && e.cols[(size_t)c * A.Kt + fill[c]] >= 0)
                return ddnm_fail(ctx, DDNM_E_INVALID, "encoder mask of autoencoder " + std::to_string(a) +
                                                          " has inputs outside its decoder's mask");
        padI(); A.iColsT = (long long)I.size();
        I.insert(I.end(), e.cols.begin(), e.cols.end());
        padI(); A.iTslot = (long long)I.size();
        I.insert(I.end(), tslot.begin(), tslot.end());
        padI(); A.iCols = (long long)I.size();
        I.insert(I.end(), d.cols.begin(), d.cols.end());
        padI(); A.iIds = (long long)I.size();
        I.insert(I.end(), ids.begin(), ids.end());
        for (int r = 0; r < A.N; ++r) row_ae.push_back(a);
        for (int j = 0; j < A.w; ++j) hid_ae.push_back(a);
        R += A.N;
        H += A.w;
        S->Nmax = std::max(S->Nmax, A.N);
        S->hae[a] = A;
    }
    S->R = R;
    S->H = H;
    S->P = (long long)P.size();
    S->I = (long long)I.size();
    const int nblk = (R + AE_T - 1) / AE_T;
    S->loss_slots = nblk;
    AK(cudaMalloc(&S->d_ae, n_ae * sizeof(AeDev)));
    AK(cudaMalloc(&S->d_int, S->I * 4));
    AK(cudaMalloc(&S->d_row_ae, (size_t)R * 4));
    AK(cudaMalloc(&S->d_hid_ae, (size_t)H * 4));
    for (float** q : {&S->p, &S->g, &S->m, &S->v}) AK(cudaMalloc(q, S->P * 4));
    AK(cudaMalloc(&S->off, (size_t)R * 8));
    AK(cudaMalloc(&S->sc, (size_t)R * 8));
    for (float** q : {&S->xt, &S->gy}) AK(cudaMalloc(q, (size_t)AE_MAXB * R * 4));
    for (float** q : {&S->z1, &S->a1, &S->z2, &S->a2, &S->gz2, &S->gz1}) AK(cudaMalloc(q, (size_t)AE_MAXB * H * 4));
    for (float** q : {&S->lat, &S->glat}) AK(cudaMalloc(q, (size_t)n_ae * AE_MAXB * 16 * 4));
    AK(cudaMalloc(&S->loss, (size_t)n_ae * nblk * 8));
    AK(cudaMalloc(&S->d_idx, AE_MAXB * 4));
    AK(cudaMemcpy(S->d_ae, S->hae.data(), n_ae * sizeof(AeDev), cudaMemcpyHostToDevice));
    AK(cudaMemcpy(S->d_int, I.data(), S->I * 4, cudaMemcpyHostToDevice));
    AK(cudaMemcpy(S->d_row_ae, row_ae.data(), (size_t)R * 4, cudaMemcpyHostToDevice));
    AK(cudaMemcpy(S->d_hid_ae, hid_ae.data(), (size_t)H * 4, cudaMemcpyHostToDevice));
    AK(cudaMemcpy(S->p, P.data(), S->P * 4, cudaMemcpyHostToDevice));
    AK(cudaMemset(S->m, 0, S->P * 4));
    AK(cudaMemset(S->v, 0, S->P * 4));
    AK(cudaMemset(S->g, 0, S->P * 4));
    S->steps = 0;
    S->ready = true;
    return DDNM_OK;
}

template <int NB>
int ae_batch(ddnm_ctx* ctx, AeState* S, int nb, cudaStream_t st) {
    const AeDev* D = S->d_ae;
    const int wpb = AE_T / 32;
    const int gH = (S->H + wpb - 1) / wpb, gR = (S->R + AE_T - 1) / AE_T, gL = (S->n_ae * 16 + wpb - 1) / wpb;
    k_ae_enc<NB><<<gH, AE_T, 0, st>>>(D, S->d_hid_ae, S->d_int, S->p, S->xt, nb, S->H, S->z1, S->a1);
    k_ae_lat<NB><<<gL, AE_T, 0, st>>>(D, S->n_ae, S->p, S->a1, nb, S->lat);
    k_ae_dec1<<<(int)(((long long)S->H * nb + AE_T - 1) / AE_T), AE_T, 0, st>>>(D, S->d_hid_ae, S->p, S->lat, nb, S->H,
                                                                                S->z2, S->a2);
    k_ae_out<NB><<<gR, AE_T, 0, st>>>(D, S->d_row_ae, S->d_int, S->p, S->a2, S->xt, nb, S->R, S->gy, S->g, S->loss);
    k_ae_back2<NB><<<gH, AE_T, 0, st>>>(D, S->d_hid_ae, S->d_int, S->p, S->gy, S->z2, S->lat, nb, S->H, S->gz2, S->g);
    k_ae_glat<NB><<<gL, AE_T, 0, st>>>(D, S->n_ae, S->p, S->gz2, nb, S->glat);
    k_ae_back1<<<(S->H + AE_T - 1) / AE_T, AE_T, 0, st>>>(D, S->d_hid_ae, S->p, S->glat, S->z1, S->a1, nb, S->H, S->gz1,
                                                           S->g);
    k_ae_enc_grad<NB><<<gH, AE_T, 0, st>>>(D, S->d_hid_ae, S->d_int, S->xt, S->gz1, nb, S->H, S->g);
    AK(cudaGetLastError());
    return DDNM_OK;
}

int ae_batch_any(ddnm_ctx* ctx, AeState* S, int nb, cudaStream_t st) {
    if (nb <= 8) return ae_batch<8>(ctx, S, nb, st);
    if (nb <= 16) return ae_batch<16>(ctx, S, nb, st);
    return ae_batch<32>(ctx, S, nb, st);
}

// per-autoencoder loss of the last batch from the block partials (fixed order), host
int ae_losses(ddnm_ctx* ctx, AeState* S, std::vector<double>& out, cudaStream_t st) {
    std::vector<double> part((size_t)S->n_ae * S->loss_slots);
    AK(cudaMemcpyAsync(part.data(), S->loss, part.size() * 8, cudaMemcpyDeviceToHost, st));
    AK(cudaStreamSynchronize(st));
    out.assign(S->n_ae, 0.0);
    for (int a = 0; a < S->n_ae; ++a) {
        const int b0 = S->hae[a].row0 / AE_T, b1 = (S->hae[a].row0 + S->hae[a].N - 1) / AE_T;
        for (int b = b0; b <= b1; ++b) out[a] += part[(size_t)a * S->loss_slots + b];
    }
    return DDNM_OK;
}

// write the trained decoders (with the normalisation as the de-normalisation layer) back into the context
int ae_store(ddnm_ctx* ctx, AeState* S) {
    std::vector<float> P(S->P);
    std::vector<double> off(S->R), sc(S->R);
    AK(cudaMemcpy(P.data(), S->p, S->P * 4, cudaMemcpyDeviceToHost));
    AK(cudaMemcpy(off.data(), S->off, (size_t)S->R * 8, cudaMemcpyDeviceToHost));
    AK(cudaMemcpy(sc.data(), S->sc, (size_t)S->R * 8, cudaMemcpyDeviceToHost));
    for (int a = 0; a < S->n_ae; ++a) {
        const AeDev& A = S->hae[a];
        DecoderHost& d = dec_of(ctx, a);
        for (int j = 0; j < A.w; ++j) d.b1[j] = P[A.pbd1 + j];
        for (size_t k = 0; k < d.W1.size(); ++k) d.W1[k] = P[A.pWd1 + k];
        for (size_t k = 0; k < d.vals.size(); ++k) d.vals[k] = d.cols[k] >= 0 ? P[A.pWd2 + k] : 0.0;
        for (int r = 0; r < A.N; ++r) {
            d.offset[r] = off[A.row0 + r];
            d.scale[r] = sc[A.row0 + r];
        }
        EncoderHost& e = S->enc[a];
        for (size_t k = 0; k < e.vals.size(); ++k) e.vals[k] = e.cols[k] >= 0 ? P[A.pWe1 + k] : 0.0;
        for (int j = 0; j < A.w; ++j) e.b1[j] = P[A.pbe1 + j];
        for (size_t k = 0; k < e.W2.size(); ++k) e.W2[k] = P[A.pWe2 + k];
    }
    ctx->finalized = false;      // the next solve uploads the trained decoders
    return DDNM_OK;
}

}  // namespace

void ddnm_ae_release(ddnm_ctx* ctx) {
    AeState* S = (AeState*)ctx->ae;
    if (!S) return;
    ae_free_device(S);
    delete S;
    ctx->ae = nullptr;
}

extern "C" int ddnm_load_encoder(ddnm_ctx* ctx, int sub, int kind, const ddnm_encoder* e) {
    if (!ctx) return DDNM_E_INVALID;
    if (!e || sub < 0 || sub >= ctx->n_sub || (kind != DDNM_DECODER_INTERIOR && kind != DDNM_DECODER_INTERFACE))
        return ddnm_fail(ctx, DDNM_E_INVALID, "bad encoder arguments");
    const SubHost& sd = ctx->subs[sub];
    const int N = kind == DDNM_DECODER_INTERIOR ? (int)sd.interior.size() : (int)sd.interface.size();
    const int n = kind == DDNM_DECODER_INTERIOR ? sd.nO : sd.nG;
    if (e->N != N || e->n != n || e->n > 16) return ddnm_fail(ctx, DDNM_E_INVALID, "encoder size does not match the decomposition");
    if (e->w < 1 || e->Kt < 1) return ddnm_fail(ctx, DDNM_E_INVALID, "encoder width or Kt out of range");
    if (!e->cols || !e->vals || !e->b1 || !e->W2) return ddnm_fail(ctx, DDNM_E_INVALID, "encoder array is NULL");
    EncoderHost h;
    h.N = N; h.w = e->w; h.n = n; h.Kt = e->Kt;
    h.cols.assign(e->cols, e->cols + (size_t)e->w * e->Kt);
    h.vals.assign(e->vals, e->vals + (size_t)e->w * e->Kt);
    h.b1.assign(e->b1, e->b1 + e->w);
    h.W2.assign(e->W2, e->W2 + (size_t)n * e->w);
    for (int j = 0; j < h.w; ++j) {
        bool pad = false;
        for (int t = 0; t < h.Kt; ++t) {
            const int c = h.cols[(size_t)j * h.Kt + t];
            if (c < -1 || c >= N) return ddnm_fail(ctx, DDNM_E_INVALID, "encoder column outside [-1, N)");
            if (c < 0) pad = true;
            else if (pad) return ddnm_fail(ctx, DDNM_E_INVALID, "encoder row has a column after -1 padding");
        }
    }
    h.loaded = true;
    AeState* S = ae_state(ctx);
    S->enc[2 * sub + kind] = std::move(h);
    S->ready = false;            // the next training re-uploads the weights
    return DDNM_OK;
}

extern "C" int ddnm_ae_train(ddnm_ctx* ctx, int n_snap, const double* X, int epochs, int batch, double lr,
                             const int* order, double* losses, int mem_kind, void* stream) {
    if (!ctx) return DDNM_E_INVALID;
    if (n_snap < 1 || !X || epochs < 0 || batch < 1 || batch > AE_MAXB || !(lr > 0.0))
        return ddnm_fail(ctx, DDNM_E_INVALID, "ddnm_ae_train: n_snap >= 1, X, epochs >= 0, batch in 1..32, lr > 0");
    if (mem_kind != DDNM_MEM_HOST && mem_kind != DDNM_MEM_DEVICE) return ddnm_fail(ctx, DDNM_E_INVALID, "bad mem_kind");
    AK(cudaSetDevice(ctx->device));
    AeState* S = ae_state(ctx);
    int rc = ae_setup(ctx, S);            // every training starts from the loaded decoders and encoders
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int Nx = 2 * ctx->nx * ctx->ny;
    AK(cudaMalloc(&S->snap, (size_t)n_snap * Nx * 8));
    S->snap_cap = n_snap;
    AK(cudaMemcpyAsync(S->snap, X, (size_t)n_snap * Nx * 8,
                       mem_kind == DDNM_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
    k_ae_norm<<<(S->R + AE_T - 1) / AE_T, AE_T, 0, st>>>(S->d_ae, S->d_row_ae, S->d_int, S->snap, n_snap, Nx, S->R,
                                                          S->off, S->sc);
    AK(cudaGetLastError());
    std::vector<int> ord;
    if (order) {
        ord.assign(order, order + (size_t)epochs * n_snap);
        for (int v : ord)
            if (v < 0 || v >= n_snap) return ddnm_fail(ctx, DDNM_E_INVALID, "ddnm_ae_train: order entry outside [0, n_snap)");
    }
    int* h_idx = nullptr;
    AK(cudaMallocHost(&h_idx, AE_MAXB * 4));
    std::vector<double> acc(S->n_ae), bl;
    const float b1 = 0.9f, b2 = 0.999f;
    const int nblk = std::max(1, std::min(4096, (int)((S->P + AE_T - 1) / AE_T)));
    for (int ep = 0; ep < epochs; ++ep) {
        std::fill(acc.begin(), acc.end(), 0.0);
        int n_batches = 0;
        for (int b0 = 0; b0 < n_snap; b0 += batch) {
            const int nb = std::min(batch, n_snap - b0);
            AK(cudaStreamSynchronize(st));         // h_idx is reused batch to batch
            for (int k = 0; k < nb; ++k) h_idx[k] = order ? ord[(size_t)ep * n_snap + b0 + k] : b0 + k;
            AK(cudaMemcpyAsync(S->d_idx, h_idx, nb * 4, cudaMemcpyHostToDevice, st));
            k_ae_gather<<<(S->R + AE_T - 1) / AE_T, AE_T, 0, st>>>(S->d_ae, S->d_row_ae, S->d_int, S->snap, Nx, S->d_idx,
                                                                    nb, S->R, S->off, S->sc, S->xt);
            rc = ae_batch_any(ctx, S, nb, st);
            if (rc) { cudaFreeHost(h_idx); return rc; }
            S->steps += 1;
            const float bc1 = 1.f - powf(b1, (float)S->steps), bc2 = 1.f - powf(b2, (float)S->steps);
            k_ae_adam<<<nblk, AE_T, 0, st>>>(S->p, S->g, S->m, S->v, S->P, (float)lr, b1, b2, 1e-8f, bc1, bc2);
            if (losses) {
                rc = ae_losses(ctx, S, bl, st);
                if (rc) { cudaFreeHost(h_idx); return rc; }
                for (int a = 0; a < S->n_ae; ++a) acc[a] += bl[a] / nb;
            }
            ++n_batches;
        }
        if (losses)
            for (int a = 0; a < S->n_ae; ++a) losses[(size_t)ep * S->n_ae + a] = acc[a] / n_batches;
    }
    AK(cudaStreamSynchronize(st));
    cudaFreeHost(h_idx);
    AK(cudaGetLastError());
    cudaFree(S->snap);
    S->snap = nullptr;
    S->snap_cap = 0;
    return ae_store(ctx, S);
}

extern "C" int ddnm_ae_loss_grad(ddnm_ctx* ctx, int sub, int kind, int nb, const float* Xt, float* grad, double* loss) {
    if (!ctx) return DDNM_E_INVALID;
    if (sub < 0 || sub >= ctx->n_sub || (kind != 0 && kind != 1) || nb < 1 || nb > AE_MAXB || !Xt)
        return ddnm_fail(ctx, DDNM_E_INVALID, "ddnm_ae_loss_grad: bad arguments");
    AK(cudaSetDevice(ctx->device));
    AeState* S = ae_state(ctx);
    int rc = ae_setup(ctx, S);
    if (rc) return rc;
    const int a = 2 * sub + kind;
    const AeDev& A = S->hae[a];
    // every autoencoder gets the same batch layout; only autoencoder a's rows are filled
    std::vector<float> xt((size_t)AE_MAXB * S->R, 0.f);
    for (int b = 0; b < nb; ++b)
        for (int r = 0; r < A.N; ++r) xt[(size_t)A.row0 * nb + (size_t)b * A.N + r] = Xt[(size_t)b * A.N + r];
    AK(cudaMemcpy(S->xt, xt.data(), xt.size() * 4, cudaMemcpyHostToDevice));
    rc = ae_batch_any(ctx, S, nb, nullptr);
    if (rc) return rc;
    std::vector<double> bl;
    rc = ae_losses(ctx, S, bl, nullptr);
    if (rc) return rc;
    if (loss) *loss = bl[a] / nb;
    if (grad) AK(cudaMemcpy(grad, S->g + A.pWe1, A.nP * 4, cudaMemcpyDeviceToHost));
    return DDNM_OK;
}

extern "C" int ddnm_ae_layout(const ddnm_ctx* ctx, int sub, int kind, long long* offsets) {
    if (!ctx || !ctx->ae || sub < 0 || sub >= ctx->n_sub || (kind != 0 && kind != 1) || !offsets) return DDNM_E_INVALID;
    const AeState* S = (const AeState*)ctx->ae;
    if ((int)S->hae.size() != 2 * ctx->n_sub) return DDNM_E_STATE;
    const AeDev& A = S->hae[2 * sub + kind];
    const long long o = A.pWe1;
    offsets[0] = 0;
    offsets[1] = A.pbe1 - o;
    offsets[2] = A.pWe2 - o;
    offsets[3] = A.pWd1 - o;
    offsets[4] = A.pbd1 - o;
    offsets[5] = A.pWd2 - o;
    offsets[6] = A.nP;
    return DDNM_OK;
}

extern "C" int ddnm_get_decoder(const ddnm_ctx* ctx, int sub, int kind, double* W1, double* b1, double* vals,
                                double* scale, double* offset) {
    if (!ctx || sub < 0 || sub >= ctx->n_sub || (kind != 0 && kind != 1)) return DDNM_E_INVALID;
    const DecoderHost& d = (kind == 0 ? ctx->decO : ctx->decG)[sub];
    if (!d.loaded) return DDNM_E_STATE;
    if (W1) std::copy(d.W1.begin(), d.W1.end(), W1);
    if (b1) std::copy(d.b1.begin(), d.b1.end(), b1);
    if (vals) std::copy(d.vals.begin(), d.vals.end(), vals);
    if (scale) std::copy(d.scale.begin(), d.scale.end(), scale);
    if (offset) std::copy(d.offset.begin(), d.offset.end(), offset);
    return DDNM_OK;
}
