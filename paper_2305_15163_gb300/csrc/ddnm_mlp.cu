// Learned warm start for the batched SQP: an MLP mu -> xh0, trained on the device by the kernels below.
//
// The paper starts the SQP from RBF interpolants of snapshot latents (Sec. 7.2).  Here a small MLP
// (2 -> H -> H -> n_D, tanh hidden layers, linear output) is trained on solutions the SQP itself produces:
// forward, backward (chain rule layer by layer) and Adam (Kingma & Ba 2015) are hand-written kernels.
// The GEMMs read the weights as bfloat16 and accumulate in FP32; Adam keeps FP32 master weights and
// refreshes the bfloat16 copy after every step.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ddnm_ctx.h"

using namespace ddnm;

namespace {

constexpr int GT = 32;            // GEMM tile (outputs per side) and K-step
constexpr float ADAM_B1 = 0.9f, ADAM_B2 = 0.999f, ADAM_EPS = 1e-8f;

__device__ __forceinline__ float ldf(const float* p) { return *p; }
__device__ __forceinline__ float ldf(const __nv_bfloat16* p) { return __bfloat162float(*p); }

// C[m][n] (= or +=) sum_k A(m, k) B(n, k), A(m, k) = A[m*sam + k*sak], B(n, k) = B[n*sbn + k*sbk]; FP32 accumulation.
// 32 x 32 output tile per CTA (256 threads, 4 outputs each), K staged through shared memory in steps of 32.
template <typename TB>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, const float* A, long sam, long sak, const TB* Bm,
                                              long sbn, long sbk, float* C, long ldc, int accumulate) {
    __shared__ float As[GT][GT + 1];
    __shared__ float Bs[GT][GT + 1];
    const int tid = threadIdx.x;
    const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
    const int tm = tid / 8, tn = (tid % 8) * 4;       // thread: row tm, columns tn..tn+3
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k0 = 0; k0 < K; k0 += GT) {
        for (int e = tid; e < GT * GT; e += 256) {
            const int r = e / GT, k = e % GT;
            As[r][k] = (m0 + r < M && k0 + k < K) ? A[(long)(m0 + r) * sam + (long)(k0 + k) * sak] : 0.f;
            Bs[r][k] = (n0 + r < N && k0 + k < K) ? ldf(Bm + (long)(n0 + r) * sbn + (long)(k0 + k) * sbk) : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < GT; ++k) {
            const float a = As[tm][k];
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] += a * Bs[tn + u][k];
        }
        __syncthreads();
    }
    const int m = m0 + tm;
    if (m < M)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int n = n0 + tn + u;
            if (n < N) C[(long)m * ldc + n] = accumulate ? C[(long)m * ldc + n] + acc[u] : acc[u];
        }
}

// Y[b][j] = act(X[b][j] + bias[j]), act = tanh (act = 1) or identity
__global__ void k_bias_act(int nb, int n, const float* X, const float* bias, float* Y, int act) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long)nb * n) return;
    const float v = X[i] + bias[i % n];
    Y[i] = act ? tanhf(v) : v;
}

// dY = 2 (Y - T) / (nb n); per-CTA partial losses into part[blockIdx.x]
__global__ void k_loss_grad(int nb, int n, const float* Y, const float* Tt, float* dY, double* part) {
    __shared__ double red[256];
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (i < (long)nb * n) {
        const float d = Y[i] - Tt[i];
        dY[i] = 2.f * d / (float)((long)nb * n);
        l = (double)d * d;
    }
    red[threadIdx.x] = l;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// dZ = dA * (1 - A^2)   (tanh')
__global__ void k_tanh_back(long n, const float* A, const float* dA, float* dZ) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dZ[i] = dA[i] * (1.f - A[i] * A[i]);
}

// db[j] = sum_b dZ[b][j]
__global__ void k_colsum(int nb, int n, const float* dZ, float* db) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    float s = 0.f;
    for (int b = 0; b < nb; ++b) s += dZ[(long)b * n + j];
    db[j] = s;
}

// Adam step t on all parameters; refreshes the bfloat16 working copy
__global__ void k_adam(long n, float* p, const float* g, float* m, float* v, __nv_bfloat16* pb, float lr, float c1,
                       float c2) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = ADAM_B1 * m[i] + (1.f - ADAM_B1) * gi;
    const float vi = ADAM_B2 * v[i] + (1.f - ADAM_B2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + ADAM_EPS);
    p[i] = pi;
    pb[i] = __float2bfloat16_rn(pi);
}

__global__ void k_to_bf16(long n, const float* p, __nv_bfloat16* pb) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) pb[i] = __float2bfloat16_rn(p[i]);
}

// mini-batch: z = (mu - mu_c) / mu_s, t = (x - mean) / std for the rows order[0..nb)
__global__ void k_gather_batch(int nb, int nout, const int* order, const float* mu, const float* x, const float* norm,
                               float* z, float* t) {
    const int b = blockIdx.x;
    if (b >= nb) return;
    const int r = order[b];
    if (threadIdx.x < 2) z[b * 2 + threadIdx.x] = (mu[r * 2 + threadIdx.x] - norm[threadIdx.x]) / norm[2 + threadIdx.x];
    for (int k = threadIdx.x; k < nout; k += blockDim.x)
        t[(long)b * nout + k] = (x[(long)r * nout + k] - norm[4 + k]) / norm[4 + nout + k];
}

// prediction input: z = (mu - mu_c) / mu_s (mu in FP64)
__global__ void k_norm_in(int B, const double* mu, const float* norm, float* z) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 2 * B) z[i] = ((float)mu[i] - norm[i % 2]) / norm[2 + i % 2];
}

// prediction output: xh0 = mean + std * y; a row with a non-finite entry becomes the default start 0
__global__ void k_norm_out(int B, int nout, const float* y, const float* norm, double* x0, int* fell_back) {
    const int b = blockIdx.x;
    if (b >= B) return;
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int k = threadIdx.x; k < nout; k += blockDim.x) {
        const float v = norm[4 + k] + norm[4 + nout + k] * y[(long)b * nout + k];
        if (!isfinite(v)) bad = 1;
        x0[(long)b * nout + k] = (double)v;
    }
    __syncthreads();
    if (bad) {
        for (int k = threadIdx.x; k < nout; k += blockDim.x) x0[(long)b * nout + k] = 0.0;
        if (threadIdx.x == 0 && fell_back) fell_back[b] = 1;
    }
}

int mfail(ddnm_ctx* ctx, cudaError_t e, const char* what) {
    return ddnm_fail(ctx, DDNM_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
#define MK(call)                                                 \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return mfail(ctx, e_, #call);     \
    } while (0)

template <typename TB>
int gemm(ddnm_ctx* ctx, cudaStream_t st, int M, int N, int K, const float* A, long sam, long sak, const TB* Bm, long sbn,
         long sbk, float* C, long ldc, int acc) {
    dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT);
    k_gemm<TB><<<grid, 256, 0, st>>>(M, N, K, A, sam, sak, Bm, sbn, sbk, C, ldc, acc);
    MK(cudaGetLastError());
    ctx->tm.other_launches++;
    return DDNM_OK;
}

inline unsigned nblk(long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// parameter offsets (floats): W1 (H x 2), b1, W2 (H x H), b2, W3 (n x H), b3
struct Offs {
    long W1, b1, W2, b2, W3, b3, P;
};
Offs offs(int H, int n) {
    Offs o;
    o.W1 = 0;
    o.b1 = o.W1 + 2L * H;
    o.W2 = o.b1 + H;
    o.b2 = o.W2 + (long)H * H;
    o.W3 = o.b2 + H;
    o.b3 = o.W3 + (long)n * H;
    o.P = o.b3 + n;
    return o;
}

// forward on nb rows of z (nb x 2): a1, a2 (nb x H), y (nb x n)
int forward(ddnm_ctx* ctx, cudaStream_t st, int nb, const float* z, float* a1, float* a2, float* y) {
    WarmStart& w = ctx->ws;
    const Offs o = offs(w.H, w.n);
    int rc;
    if ((rc = gemm(ctx, st, nb, w.H, 2, z, 2, 1, w.pb + o.W1, 2, 1, a1, w.H, 0))) return rc;
    k_bias_act<<<nblk((long)nb * w.H), 256, 0, st>>>(nb, w.H, a1, w.p + o.b1, a1, 1);
    if ((rc = gemm(ctx, st, nb, w.H, w.H, a1, w.H, 1, w.pb + o.W2, w.H, 1, a2, w.H, 0))) return rc;
    k_bias_act<<<nblk((long)nb * w.H), 256, 0, st>>>(nb, w.H, a2, w.p + o.b2, a2, 1);
    if ((rc = gemm(ctx, st, nb, w.n, w.H, a2, w.H, 1, w.pb + o.W3, w.H, 1, y, w.n, 0))) return rc;
    k_bias_act<<<nblk((long)nb * w.n), 256, 0, st>>>(nb, w.n, y, w.p + o.b3, y, 0);
    MK(cudaGetLastError());
    ctx->tm.other_launches += 3;
    return DDNM_OK;
}

// loss and gradient (into w.g) of one batch (z, t already standardised)
int loss_grad(ddnm_ctx* ctx, cudaStream_t st, int nb, const float* z, const float* t) {
    WarmStart& w = ctx->ws;
    const Offs o = offs(w.H, w.n);
    const int H = w.H, n = w.n;
    float *a1 = w.a1, *a2 = w.a2, *y = w.y, *dy = w.dy, *d2 = w.d2, *d1 = w.d1;
    int rc;
    if ((rc = forward(ctx, st, nb, z, a1, a2, y))) return rc;
    k_loss_grad<<<nblk((long)nb * n), 256, 0, st>>>(nb, n, y, t, dy, w.lpart);
    // dW3 = dy^T a2, db3 = colsum dy
    if ((rc = gemm(ctx, st, n, H, nb, dy, 1, n, a2, 1, H, w.g + o.W3, H, 0))) return rc;
    k_colsum<<<nblk(n), 256, 0, st>>>(nb, n, dy, w.g + o.b3);
    // d2 = (dy W3) * (1 - a2^2)
    if ((rc = gemm(ctx, st, nb, H, n, dy, n, 1, w.pb + o.W3, 1, H, d2, H, 0))) return rc;
    k_tanh_back<<<nblk((long)nb * H), 256, 0, st>>>((long)nb * H, a2, d2, d2);
    if ((rc = gemm(ctx, st, H, H, nb, d2, 1, H, a1, 1, H, w.g + o.W2, H, 0))) return rc;
    k_colsum<<<nblk(H), 256, 0, st>>>(nb, H, d2, w.g + o.b2);
    // d1 = (d2 W2) * (1 - a1^2)
    if ((rc = gemm(ctx, st, nb, H, H, d2, H, 1, w.pb + o.W2, 1, H, d1, H, 0))) return rc;
    k_tanh_back<<<nblk((long)nb * H), 256, 0, st>>>((long)nb * H, a1, d1, d1);
    if ((rc = gemm(ctx, st, H, 2, nb, d1, 1, H, z, 1, 2, w.g + o.W1, 2, 0))) return rc;
    k_colsum<<<nblk(H), 256, 0, st>>>(nb, H, d1, w.g + o.b1);
    MK(cudaGetLastError());
    ctx->tm.other_launches += 6;
    return DDNM_OK;
}

int ws_alloc_batch(ddnm_ctx* ctx, int nb) {
    WarmStart& w = ctx->ws;
    if (nb <= w.cap) return DDNM_OK;
    cudaFree(w.act);
    w.act = nullptr;
    w.cap = 0;
    const size_t H = w.H, n = w.n, P = offs(w.H, w.n).P;
    const size_t floats = (size_t)nb * (2 + 3 * H + 2 * n + 2 * H + n) + P;
    MK(cudaMalloc(&w.act, floats * 4 + (size_t)nblk((long)nb * std::max<size_t>(n, H)) * 8 + 64));
    float* f = (float*)w.act;
    w.z = f; f += (size_t)nb * 2;
    w.a1 = f; f += (size_t)nb * H;
    w.a2 = f; f += (size_t)nb * H;
    w.y = f; f += (size_t)nb * n;
    w.t = f; f += (size_t)nb * n;
    w.dy = f; f += (size_t)nb * n;
    w.d2 = f; f += (size_t)nb * H;
    w.d1 = f; f += (size_t)nb * H;
    w.g = f; f += P;
    w.lpart = (double*)(((uintptr_t)f + 15) & ~(uintptr_t)15);
    w.cap = nb;
    return DDNM_OK;
}

}  // namespace

void ddnm_ws_release(ddnm_ctx* ctx) {
    WarmStart& w = ctx->ws;
    cudaFree(w.p);
    cudaFree(w.pb);
    cudaFree(w.m);
    cudaFree(w.v);
    cudaFree(w.norm);
    cudaFree(w.act);
    cudaFree(w.data);
    w = WarmStart{};
}

// prediction of B warm starts (device mu -> device x0); used by ddnm_solve_batch
int ddnm_ws_predict_dev(ddnm_ctx* ctx, int B, const double* mu_dev, double* x0_dev, int* fell_back, cudaStream_t st) {
    WarmStart& w = ctx->ws;
    int rc = ws_alloc_batch(ctx, B);
    if (rc) return rc;
    k_norm_in<<<nblk(2L * B), 256, 0, st>>>(B, mu_dev, w.norm, w.z);
    if ((rc = forward(ctx, st, B, w.z, w.a1, w.a2, w.y))) return rc;
    k_norm_out<<<B, 128, 0, st>>>(B, w.n, w.y, w.norm, x0_dev, fell_back);
    MK(cudaGetLastError());
    ctx->tm.other_launches += 2;
    return DDNM_OK;
}

extern "C" int ddnm_ws_init(ddnm_ctx* ctx, int hidden, const float* params) {
    if (!ctx) return DDNM_E_INVALID;
    if (hidden < 1 || hidden > 4096 || !params) return ddnm_fail(ctx, DDNM_E_INVALID, "hidden in 1..4096 and params required");
    MK(cudaSetDevice(ctx->device));
    ddnm_ws_release(ctx);
    WarmStart& w = ctx->ws;
    w.H = hidden;
    w.n = ctx->n_D;
    const long P = offs(w.H, w.n).P;
    for (long i = 0; i < P; ++i)
        if (!std::isfinite(params[i])) return ddnm_fail(ctx, DDNM_E_INVALID, "non-finite initial parameter");
    MK(cudaMalloc(&w.p, P * 4));
    MK(cudaMalloc(&w.pb, P * 2));
    MK(cudaMalloc(&w.m, P * 4));
    MK(cudaMalloc(&w.v, P * 4));
    MK(cudaMalloc(&w.norm, (4 + 2 * (size_t)w.n) * 4));
    MK(cudaMemcpy(w.p, params, P * 4, cudaMemcpyHostToDevice));
    MK(cudaMemset(w.m, 0, P * 4));
    MK(cudaMemset(w.v, 0, P * 4));
    std::vector<float> nrm(4 + 2 * (size_t)w.n, 0.f);
    nrm[2] = nrm[3] = 1.f;
    for (int k = 0; k < w.n; ++k) nrm[4 + w.n + k] = 1.f;
    MK(cudaMemcpy(w.norm, nrm.data(), nrm.size() * 4, cudaMemcpyHostToDevice));
    k_to_bf16<<<nblk(P), 256>>>(P, w.p, w.pb);
    MK(cudaGetLastError());
    MK(cudaDeviceSynchronize());
    w.steps = 0;
    w.ready = true;
    return DDNM_OK;
}

extern "C" int ddnm_ws_set_norm(ddnm_ctx* ctx, const double* mu_c, const double* mu_s, const double* out_mean,
                                const double* out_std) {
    if (!ctx) return DDNM_E_INVALID;
    WarmStart& w = ctx->ws;
    if (!w.ready) return ddnm_fail(ctx, DDNM_E_STATE, "warm start not initialised (ddnm_ws_init)");
    if (!mu_c || !mu_s || !out_mean || !out_std) return ddnm_fail(ctx, DDNM_E_INVALID, "NULL normalisation");
    std::vector<float> nrm(4 + 2 * (size_t)w.n);
    for (int k = 0; k < 2; ++k) {
        if (!(mu_s[k] > 0)) return ddnm_fail(ctx, DDNM_E_INVALID, "mu_s must be positive");
        nrm[k] = (float)mu_c[k];
        nrm[2 + k] = (float)mu_s[k];
    }
    for (int k = 0; k < w.n; ++k) {
        if (!(out_std[k] > 0)) return ddnm_fail(ctx, DDNM_E_INVALID, "out_std must be positive");
        nrm[4 + k] = (float)out_mean[k];
        nrm[4 + w.n + k] = (float)out_std[k];
    }
    MK(cudaSetDevice(ctx->device));
    MK(cudaMemcpy(w.norm, nrm.data(), nrm.size() * 4, cudaMemcpyHostToDevice));
    return DDNM_OK;
}

extern "C" int ddnm_ws_loss_grad(ddnm_ctx* ctx, int nb, const float* z, const float* t, float* grad, double* loss) {
    if (!ctx) return DDNM_E_INVALID;
    WarmStart& w = ctx->ws;
    if (!w.ready) return ddnm_fail(ctx, DDNM_E_STATE, "warm start not initialised (ddnm_ws_init)");
    if (nb < 1 || !z || !t) return ddnm_fail(ctx, DDNM_E_INVALID, "nb >= 1, z and t required");
    MK(cudaSetDevice(ctx->device));
    int rc = ws_alloc_batch(ctx, nb);
    if (rc) return rc;
    MK(cudaMemcpy(w.z, z, (size_t)nb * 2 * 4, cudaMemcpyHostToDevice));
    MK(cudaMemcpy(w.t, t, (size_t)nb * w.n * 4, cudaMemcpyHostToDevice));
    if ((rc = loss_grad(ctx, 0, nb, w.z, w.t))) return rc;
    MK(cudaDeviceSynchronize());
    const long P = offs(w.H, w.n).P;
    if (grad) MK(cudaMemcpy(grad, w.g, P * 4, cudaMemcpyDeviceToHost));
    if (loss) {
        const unsigned nbl = nblk((long)nb * w.n);
        std::vector<double> part(nbl);
        MK(cudaMemcpy(part.data(), w.lpart, nbl * 8, cudaMemcpyDeviceToHost));
        double s = 0.0;
        for (double v : part) s += v;
        *loss = s / ((double)nb * w.n);
    }
    return DDNM_OK;
}

extern "C" int ddnm_ws_train(ddnm_ctx* ctx, int n, const double* mu, const double* x_star, int epochs, int batch,
                             double lr, const int* order, double* losses) {
    if (!ctx) return DDNM_E_INVALID;
    WarmStart& w = ctx->ws;
    if (!w.ready) return ddnm_fail(ctx, DDNM_E_STATE, "warm start not initialised (ddnm_ws_init)");
    if (n < 1 || !mu || !x_star || epochs < 0 || batch < 1 || !(lr > 0))
        return ddnm_fail(ctx, DDNM_E_INVALID, "bad training arguments");
    if (order)
        for (long i = 0; i < (long)epochs * n; ++i)
            if (order[i] < 0 || order[i] >= n) return ddnm_fail(ctx, DDNM_E_INVALID, "order entry out of range");
    MK(cudaSetDevice(ctx->device));
    // standardisation of the training set (mu to [-1, 1], outputs to zero mean, unit deviation)
    const int nout = w.n;
    std::vector<double> mc(2), ms(2), om(nout, 0.0), os(nout, 0.0);
    for (int k = 0; k < 2; ++k) {
        double lo = mu[k], hi = mu[k];
        for (int i = 0; i < n; ++i) {
            lo = std::min(lo, mu[2 * i + k]);
            hi = std::max(hi, mu[2 * i + k]);
        }
        mc[k] = 0.5 * (hi + lo);
        ms[k] = std::max(0.5 * (hi - lo), 1e-12);
    }
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < nout; ++k) om[k] += x_star[(size_t)i * nout + k];
    for (int k = 0; k < nout; ++k) om[k] /= n;
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < nout; ++k) {
            const double d = x_star[(size_t)i * nout + k] - om[k];
            os[k] += d * d;
        }
    for (int k = 0; k < nout; ++k) os[k] = std::max(std::sqrt(os[k] / n), 1e-8);
    int rc = ddnm_ws_set_norm(ctx, mc.data(), ms.data(), om.data(), os.data());
    if (rc) return rc;
    // training data and orders on the device
    cudaFree(w.data);
    w.data = nullptr;
    const size_t nord = (size_t)std::max(epochs, 1) * n;
    MK(cudaMalloc(&w.data, ((size_t)n * (2 + nout)) * 4 + nord * 4));
    float* dmu = (float*)w.data;
    float* dx = dmu + (size_t)n * 2;
    int* dord = (int*)(dx + (size_t)n * nout);
    std::vector<float> hf((size_t)n * (2 + nout));
    for (size_t i = 0; i < (size_t)n * 2; ++i) hf[i] = (float)mu[i];
    for (size_t i = 0; i < (size_t)n * nout; ++i) hf[(size_t)n * 2 + i] = (float)x_star[i];
    MK(cudaMemcpy(dmu, hf.data(), hf.size() * 4, cudaMemcpyHostToDevice));
    std::vector<int> ho(nord);
    for (size_t i = 0; i < nord; ++i) ho[i] = order ? order[i] : (int)(i % n);
    MK(cudaMemcpy(dord, ho.data(), nord * 4, cudaMemcpyHostToDevice));
    if ((rc = ws_alloc_batch(ctx, batch))) return rc;
    const long P = offs(w.H, w.n).P;
    std::vector<double> part;
    for (int e = 0; e < epochs; ++e) {
        double tot = 0.0;
        int nbat = 0;
        for (int b0 = 0; b0 < n; b0 += batch) {
            const int nb = std::min(batch, n - b0);
            k_gather_batch<<<nb, 128>>>(nb, nout, dord + (size_t)e * n + b0, dmu, dx, w.norm, w.z, w.t);
            if ((rc = loss_grad(ctx, 0, nb, w.z, w.t))) return rc;
            ++w.steps;
            const float c1 = 1.f - std::pow(ADAM_B1, (float)w.steps), c2 = 1.f - std::pow(ADAM_B2, (float)w.steps);
            k_adam<<<nblk(P), 256>>>(P, w.p, w.g, w.m, w.v, w.pb, (float)lr, c1, c2);
            MK(cudaGetLastError());
            ctx->tm.other_launches += 2;
            const unsigned nbl = nblk((long)nb * nout);
            part.resize(nbl);
            MK(cudaMemcpy(part.data(), w.lpart, nbl * 8, cudaMemcpyDeviceToHost));
            double s = 0.0;
            for (double v : part) s += v;
            tot += s / ((double)nb * nout);
            ++nbat;
        }
        if (losses) losses[e] = tot / nbat;
    }
    MK(cudaDeviceSynchronize());
    return DDNM_OK;
}

extern "C" int ddnm_ws_predict(ddnm_ctx* ctx, int B, const double* mu, double* x0, int mem_kind, void* stream) {
    if (!ctx) return DDNM_E_INVALID;
    WarmStart& w = ctx->ws;
    if (!w.ready) return ddnm_fail(ctx, DDNM_E_STATE, "warm start not initialised (ddnm_ws_init)");
    if (B < 1 || !mu || !x0) return ddnm_fail(ctx, DDNM_E_INVALID, "B >= 1, mu and x0 required");
    MK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const bool host = mem_kind == DDNM_MEM_HOST;
    double *dmu = const_cast<double*>(mu), *dx = x0;
    void* tmp = nullptr;
    if (host) {
        MK(cudaMalloc(&tmp, (size_t)B * (2 + w.n) * 8));
        dmu = (double*)tmp;
        dx = dmu + 2 * (size_t)B;
        MK(cudaMemcpyAsync(dmu, mu, (size_t)B * 2 * 8, cudaMemcpyHostToDevice, st));
    }
    int rc = ddnm_ws_predict_dev(ctx, B, dmu, dx, nullptr, st);
    if (!rc && host) {
        cudaError_t e = cudaMemcpyAsync(x0, dx, (size_t)B * w.n * 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = mfail(ctx, e, "ddnm_ws_predict copy-out");
    }
    if (tmp) cudaFree(tmp);
    return rc;
}

extern "C" int ddnm_ws_get_params(const ddnm_ctx* ctx, float* params, double* norm) {
    if (!ctx) return DDNM_E_INVALID;
    const WarmStart& w = ctx->ws;
    if (!w.ready) return DDNM_E_STATE;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return DDNM_E_CUDA;
    const long P = offs(w.H, w.n).P;
    if (params && cudaMemcpy(params, w.p, P * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return DDNM_E_CUDA;
    if (norm) {
        std::vector<float> nrm(4 + 2 * (size_t)w.n);
        if (cudaMemcpy(nrm.data(), w.norm, nrm.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return DDNM_E_CUDA;
        for (size_t k = 0; k < nrm.size(); ++k) norm[k] = nrm[k];
    }
    return DDNM_OK;
}

extern "C" int ddnm_ws_enable(ddnm_ctx* ctx, int on) {
    if (!ctx) return DDNM_E_INVALID;
    if (on && !ctx->ws.ready) return ddnm_fail(ctx, DDNM_E_STATE, "warm start not initialised (ddnm_ws_init)");
    ctx->ws.enabled = on != 0;
    return DDNM_OK;
}

// file format: "DDNMWS01", int32 H, int32 n, int64 steps, P float32 params, (4 + 2n) float32 normalisation
extern "C" int ddnm_ws_save(const ddnm_ctx* ctx, const char* path) {
    if (!ctx || !path) return DDNM_E_INVALID;
    const WarmStart& w = ctx->ws;
    if (!w.ready) return DDNM_E_STATE;
    const long P = offs(w.H, w.n).P;
    std::vector<float> p(P);
    std::vector<double> nd(4 + 2 * (size_t)w.n);
    int rc = ddnm_ws_get_params(ctx, p.data(), nd.data());
    if (rc) return rc;
    std::vector<float> nf(nd.begin(), nd.end());
    FILE* f = std::fopen(path, "wb");
    if (!f) return DDNM_E_INVALID;
    const int32_t hdr[2] = {w.H, w.n};
    const int64_t steps = w.steps;
    bool ok = std::fwrite("DDNMWS01", 1, 8, f) == 8 && std::fwrite(hdr, 4, 2, f) == 2 &&
              std::fwrite(&steps, 8, 1, f) == 1 && std::fwrite(p.data(), 4, P, f) == (size_t)P &&
              std::fwrite(nf.data(), 4, nf.size(), f) == nf.size();
    ok = (std::fclose(f) == 0) && ok;
    return ok ? DDNM_OK : DDNM_E_INVALID;
}

extern "C" int ddnm_ws_load(ddnm_ctx* ctx, const char* path) {
    if (!ctx || !path) return DDNM_E_INVALID;
    FILE* f = std::fopen(path, "rb");
    if (!f) return ddnm_fail(ctx, DDNM_E_INVALID, std::string("cannot open ") + path);
    char magic[8];
    int32_t hdr[2];
    int64_t steps;
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "DDNMWS01", 8) == 0 &&
              std::fread(hdr, 4, 2, f) == 2 && std::fread(&steps, 8, 1, f) == 1;
    if (!ok || hdr[1] != ctx->n_D || hdr[0] < 1 || hdr[0] > 4096) {
        std::fclose(f);
        return ddnm_fail(ctx, DDNM_E_INVALID, "not a warm-start file for this problem");
    }
    const long P = offs(hdr[0], hdr[1]).P;
    std::vector<float> p(P), nf(4 + 2 * (size_t)hdr[1]);
    ok = std::fread(p.data(), 4, P, f) == (size_t)P && std::fread(nf.data(), 4, nf.size(), f) == nf.size();
    std::fclose(f);
    if (!ok) return ddnm_fail(ctx, DDNM_E_INVALID, "truncated warm-start file");
    int rc = ddnm_ws_init(ctx, hdr[0], p.data());
    if (rc) return rc;
    std::vector<double> nd(nf.begin(), nf.end());
    rc = ddnm_ws_set_norm(ctx, nd.data(), nd.data() + 2, nd.data() + 4, nd.data() + 4 + hdr[1]);
    ctx->ws.steps = steps;
    return rc;
}
