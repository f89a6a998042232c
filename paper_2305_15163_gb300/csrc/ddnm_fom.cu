// sm_103a batched solve of the full-order model: the steady 2D Burgers finite-difference system of
// Sec. 7.1 (Eq. burgers_discretized, Dirichlet data from Eq. burgers_pde_exact_solution), r(x; mu) = 0, for
// many parameters mu at once.  This is the FOM the paper measures its speed-ups and ROM errors against
// (Sec. 7.1, Eq. relative_error) and whose solutions are the training snapshots (Sec. 7.2).
//
// Newton's method, each step J(x) dx = -r(x) solved by right-preconditioned BiCGSTAB in FP64.  The
// preconditioner inverts the diffusion part exactly, M = nu (I (x) T_x + T_y (x) I) per component (T the
// second-difference matrix with Dirichlet ends): a discrete sine transform in x diagonalises T_x,
// T_x = (2 / (n_x + 1)) S Lambda S with S_ik = sin(pi i k / (n_x + 1)), after which every x-mode k is one
// tridiagonal system nu (T_y + lambda_k I) in y.  The sine transform is a dense product with S, run as an FP32
// GEMM over all rows of all instances and both components at once; the tridiagonal solves run one thread per
// (instance, component, mode) with the elimination factors precomputed.  The preconditioner only steers the
// Krylov iteration, so FP32 there does not change what the iteration converges to: the residual, the
// Jacobian products and every BiCGSTAB vector and scalar stay FP64.
//
// Stopping (the oracle's rule): Newton stops when ||r|| <= 1e-12 max(1, ||r(x0)||), or after a step that
// fails to halve ||r|| (the rounding floor; that step is kept), or after max_newton steps.  Each linear solve
// runs until ||J dx + r|| <= 1e-10 ||r|| or max_krylov iterations.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "ddnm_ctx.h"

namespace {

constexpr int FT = 256;          // threads of the vector kernels
constexpr int MAXG = 128;        // partial sums per instance of a dot product
constexpr int GB_M = 128, GB_N = 128, GB_K = 8;   // FP32 GEMM tile

struct FomWork {
    int cap = 0, nx = 0, ny = 0;
    double* vec = nullptr;       // cap x NV x N_x
    float* tmp = nullptr;        // cap x N_x
    float* S = nullptr;          // nx x nx sine transform
    float* cp = nullptr;         // ny x nx  Thomas factors c'_j of mode k
    float* inv = nullptr;        // ny x nx  1 / pivot_j of mode k
    double* bnd = nullptr;       // cap x 4 (nx + ny): u, v at the Dirichlet points (left, right, bottom, top)
    double* mu = nullptr;        // cap x 2
    double* part = nullptr;      // cap x 4 x MAXG dot-product partials
    double* sc = nullptr;        // cap x NSC per-instance scalars
    int* act = nullptr;          // cap  1 while the instance's linear solve runs
    double* h_sc = nullptr;      // pinned copy of sc
    int* h_act = nullptr;        // pinned copy of act
};

// vectors of one instance
enum { V_X, V_R, V_XL, V_RH, V_P, V_V, V_S, V_T, V_PH, V_SH, NV };
// scalars of one instance
enum { S_RHO, S_ALPHA, S_OMEGA, S_BN, S_RR, S_RV, S_TS, S_TT, S_ITERS, S_BREAK, NSC };

struct FomDev {
    int nx, ny, N, Nx;           // N = nx ny nodes, Nx = 2N unknowns
    double hx, hy, nu, bx0, by0;
    double ihx2, ihy2;           // 1/(2 h_x), 1/(2 h_y)
    double lx, ly;               // nu / h_x^2, nu / h_y^2
    const double* mu;
    double* bnd;
};

__device__ void exact_uv_fom(double x, double y, double a, double lam, double nu, double& u, double& v) {
    const double ep = exp(lam * (x - 1.0)), em = exp(-lam * (x - 1.0));
    const double cy = cos(lam * y), sy = sin(lam * y);
    const double psi = a * (1.0 + x) + (ep + em) * cy;
    u = -2.0 * nu * (a + lam * (ep - em) * cy) / psi;
    v = 2.0 * nu * lam * (ep + em) * sy / psi;
}

// Dirichlet values of instance b: left (x_0, y_1..y_ny), right (x_{nx+1}), bottom (y_0, x_1..x_nx), top
__global__ void k_fom_bnd(FomDev F, int B) {
    const int b = blockIdx.y;
    const int nb = 2 * (F.nx + F.ny);
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B || p >= nb) return;
    const double a = F.mu[2 * b], lm = F.mu[2 * b + 1];
    double x, y;
    if (p < F.ny) { x = F.bx0; y = F.by0 + (p + 1) * F.hy; }
    else if (p < 2 * F.ny) { x = F.bx0 + (F.nx + 1) * F.hx; y = F.by0 + (p - F.ny + 1) * F.hy; }
    else if (p < 2 * F.ny + F.nx) { x = F.bx0 + (p - 2 * F.ny + 1) * F.hx; y = F.by0; }
    else { x = F.bx0 + (p - 2 * F.ny - F.nx + 1) * F.hx; y = F.by0 + (F.ny + 1) * F.hy; }
    double u, v;
    exact_uv_fom(x, y, a, lm, F.nu, u, v);
    F.bnd[(size_t)b * 2 * nb + p] = u;
    F.bnd[(size_t)b * 2 * nb + nb + p] = v;
}

// the exact solution at the interior nodes (the default Newton start)
__global__ void k_fom_exact(FomDev F, int B, double* x, size_t stride) {
    const int b = blockIdx.y;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B || p >= F.N) return;
    const int i = p % F.nx, j = p / F.nx;
    double u, v;
    exact_uv_fom(F.bx0 + (i + 1) * F.hx, F.by0 + (j + 1) * F.hy, F.mu[2 * b], F.mu[2 * b + 1], F.nu, u, v);
    x[(size_t)b * stride + p] = u;
    x[(size_t)b * stride + F.N + p] = v;
}

// neighbour values of component c (0 = u, 1 = v) at node (i, j) of a state with Dirichlet ends
struct Nb {
    double E, W, Nn, S;
};

__device__ __forceinline__ Nb neighbours(const FomDev& F, const double* xc, const double* bc, int i, int j) {
    // bc: this component's Dirichlet values (left ny, right ny, bottom nx, top nx)
    const int p = j * F.nx + i;
    Nb n;
    n.W = i > 0 ? xc[p - 1] : bc[j];
    n.E = i < F.nx - 1 ? xc[p + 1] : bc[F.ny + j];
    n.S = j > 0 ? xc[p - F.nx] : bc[2 * F.ny + i];
    n.Nn = j < F.ny - 1 ? xc[p + F.nx] : bc[2 * F.ny + F.nx + i];
    return n;
}

__device__ __forceinline__ Nb neighbours0(const FomDev& F, const double* wc, int i, int j) {
    const int p = j * F.nx + i;
    Nb n;
    n.W = i > 0 ? wc[p - 1] : 0.0;
    n.E = i < F.nx - 1 ? wc[p + 1] : 0.0;
    n.S = j > 0 ? wc[p - F.nx] : 0.0;
    n.Nn = j < F.ny - 1 ? wc[p + F.nx] : 0.0;
    return n;
}

// r(x) of Eq. (burgers_discretized): r_u = u (B_x u - b_ux) + v (B_y u - b_uy) + L u + c_u, likewise r_v;
// written per node as -u (u_E - u_W)/(2h_x) - v (u_N - u_S)/(2h_y) + nu (u_E - 2u + u_W)/h_x^2 + ...
__global__ void k_fom_res(FomDev F, int B, const double* x, double* r, size_t stride, const int* act) {
    const int b = blockIdx.y;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B || p >= F.N || (act && !act[b])) return;
    const int i = p % F.nx, j = p / F.nx;
    const double* xu = x + (size_t)b * stride;
    const double* xv = xu + F.N;
    const int nb = 2 * (F.nx + F.ny);
    const double* bu = F.bnd + (size_t)b * 2 * nb;
    const double* bv = bu + nb;
    const Nb U = neighbours(F, xu, bu, i, j), V = neighbours(F, xv, bv, i, j);
    const double u = xu[p], v = xv[p];
    double* ru = r + (size_t)b * stride;
    ru[p] = -u * (U.E - U.W) * F.ihx2 - v * (U.Nn - U.S) * F.ihy2 + F.lx * (U.E - 2.0 * u + U.W) +
            F.ly * (U.Nn - 2.0 * u + U.S);
    ru[F.N + p] = -u * (V.E - V.W) * F.ihx2 - v * (V.Nn - V.S) * F.ihy2 + F.lx * (V.E - 2.0 * v + V.W) +
                  F.ly * (V.Nn - 2.0 * v + V.S);
}

// y = J(x) w, J the Jacobian of r (differentiating the node formula above term by term; w has zero ends)
__global__ void k_fom_jv(FomDev F, int B, const double* x, const double* w, double* y, size_t stride,
                         const int* act) {
    const int b = blockIdx.y;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B || p >= F.N || !act[b]) return;
    const int i = p % F.nx, j = p / F.nx;
    const double* xu = x + (size_t)b * stride;
    const double* xv = xu + F.N;
    const double* wu = w + (size_t)b * stride;
    const double* wv = wu + F.N;
    const int nb = 2 * (F.nx + F.ny);
    const double* bu = F.bnd + (size_t)b * 2 * nb;
    const double* bv = bu + nb;
    const Nb U = neighbours(F, xu, bu, i, j), V = neighbours(F, xv, bv, i, j);
    const Nb WU = neighbours0(F, wu, i, j), WV = neighbours0(F, wv, i, j);
    const double u = xu[p], v = xv[p], a = wu[p], c = wv[p];
    const double ux = -(U.E - U.W) * F.ihx2, uy = -(U.Nn - U.S) * F.ihy2;   // B_x u - b_ux, B_y u - b_uy
    const double vx = -(V.E - V.W) * F.ihx2, vy = -(V.Nn - V.S) * F.ihy2;
    double* yu = y + (size_t)b * stride;
    yu[p] = ux * a - u * (WU.E - WU.W) * F.ihx2 - v * (WU.Nn - WU.S) * F.ihy2 + uy * c +
            F.lx * (WU.E - 2.0 * a + WU.W) + F.ly * (WU.Nn - 2.0 * a + WU.S);
    yu[F.N + p] = vx * a - u * (WV.E - WV.W) * F.ihx2 + vy * c - v * (WV.Nn - WV.S) * F.ihy2 +
                  F.lx * (WV.E - 2.0 * c + WV.W) + F.ly * (WV.Nn - 2.0 * c + WV.S);
}

// C = scale A S: A (M x K, row-major, TA = double or float), S (K x N float, row-major), C (M x N, TC).
// 128 x 128 tiles, 8 deep, 256 threads with 8 x 8 outputs each; bounds-checked edges.
// One such product per blockIdx.z (an instance), at A + z sa and C + z sc; instances with act[z] = 0 skipped.
template <typename TA, typename TC>
__global__ void __launch_bounds__(256) k_fom_gemm(const TA* __restrict__ A, const float* __restrict__ S,
                                                  TC* __restrict__ C, int M, int N, int K, float scale, size_t sa,
                                                  size_t sc, const int* act) {
    __shared__ float As[GB_K][GB_M + 4];
    __shared__ float Bs[GB_K][GB_N + 4];
    if (!act[blockIdx.z]) return;
    A += blockIdx.z * sa;
    C += blockIdx.z * sc;
    const int tid = threadIdx.x;
    const int m0 = blockIdx.y * GB_M, n0 = blockIdx.x * GB_N;
    const int tx = tid % 16, ty = tid / 16;
    float acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[a][c] = 0.f;
    for (int k0 = 0; k0 < K; k0 += GB_K) {
        // A tile: 128 rows x 8 k, 4 per thread (row = tid / 2, k = 4 (tid % 2) ..)
        {
            const int r = tid / 2, kk = 4 * (tid % 2);
            const int gm = m0 + r;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int gk = k0 + kk + q;
                As[kk + q][r] = (gm < M && gk < K) ? (float)A[(size_t)gm * K + gk] : 0.f;
            }
        }
        // S tile: 8 k x 128 columns, 4 per thread
        {
            const int kk = tid / 32, c = 4 * (tid % 32);
            const int gk = k0 + kk;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int gn = n0 + c + q;
                Bs[kk][c + q] = (gk < K && gn < N) ? S[(size_t)gk * N + gn] : 0.f;
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GB_K; ++kk) {
            float a[8], bb[8];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = As[kk][4 * ty + q];
                a[4 + q] = As[kk][64 + 4 * ty + q];
                bb[q] = Bs[kk][4 * tx + q];
                bb[4 + q] = Bs[kk][64 + 4 * tx + q];
            }
#pragma unroll
            for (int x = 0; x < 8; ++x)
#pragma unroll
                for (int y = 0; y < 8; ++y) acc[x][y] = fmaf(a[x], bb[y], acc[x][y]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int x = 0; x < 8; ++x) {
        const int gm = m0 + (x < 4 ? 4 * ty + x : 64 + 4 * ty + x - 4);
        if (gm >= M) continue;
#pragma unroll
        for (int y = 0; y < 8; ++y) {
            const int gn = n0 + (y < 4 ? 4 * tx + y : 64 + 4 * tx + y - 4);
            if (gn < N) C[(size_t)gm * N + gn] = (TC)(scale * acc[x][y]);
        }
    }
}

// tridiagonal solves nu (T_y + lambda_k) v = a for every (instance, component, mode k), in place on the
// x-transformed rows (row (b, c, j), column k); inactive instances skipped.
__global__ void k_fom_thomas(float* A, const float* cp, const float* inv, int B, int nx, int ny, float off,
                             const int* act) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int bc = blockIdx.y;        // instance * 2 + component
    if (k >= nx || bc >= 2 * B || !act[bc / 2]) return;
    float* a = A + (size_t)bc * ny * nx + k;
    float d = 0.f;
    for (int j = 0; j < ny; ++j) {
        d = (a[(size_t)j * nx] - off * d) * inv[(size_t)j * nx + k];
        a[(size_t)j * nx] = d;
    }
    float v = 0.f;
    for (int j = ny - 1; j >= 0; --j) {
        v = a[(size_t)j * nx] - cp[(size_t)j * nx + k] * v;
        a[(size_t)j * nx] = v;
    }
}

// partial sums of up to three dot products (x0.y0, x1.y1, x2.y2) per instance; slot s of part
__global__ void k_fom_dots(const double* x0, const double* y0, const double* x1, const double* y1, const double* x2,
                           const double* y2, int n, size_t stride, double* part, int B, const int* act, int G) {
    const int b = blockIdx.y;
    if (b >= B || !act[b]) return;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    const size_t o = (size_t)b * stride;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += G * blockDim.x) {
        s0 += x0[o + k] * y0[o + k];
        if (x1) s1 += x1[o + k] * y1[o + k];
        if (x2) s2 += x2[o + k] * y2[o + k];
    }
    __shared__ double red[3][FT];
    red[0][threadIdx.x] = s0;
    red[1][threadIdx.x] = s1;
    red[2][threadIdx.x] = s2;
    __syncthreads();
    for (int w = FT / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int q = 0; q < 3; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 3) part[((size_t)b * 4 + threadIdx.x) * MAXG + blockIdx.x] = red[threadIdx.x][0];
}

__device__ __forceinline__ double sum_part(const double* part, int b, int slot, int G) {
    double s = 0.0;
    for (int g = 0; g < G; ++g) s += part[((size_t)b * 4 + slot) * MAXG + g];
    return s;
}

// the BiCGSTAB scalar steps, one thread per instance
enum { FIN_INIT, FIN_RHO, FIN_ALPHA, FIN_OMEGA, FIN_RES };
__global__ void k_fom_fin(double* sc, int* act, const double* part, int B, int G, int stage, double rtol,
                          int max_it) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B || !act[b]) return;
    double* s = sc + (size_t)b * NSC;
    if (stage == FIN_INIT) {          // part slot 0: (r, r) of the right-hand side
        const double rr = sum_part(part, b, 0, G);
        s[S_BN] = sqrt(rr);
        s[S_RR] = rr;
        s[S_RHO] = 1.0;
        s[S_ALPHA] = 1.0;
        s[S_OMEGA] = 1.0;
        s[S_ITERS] = 0.0;
        s[S_BREAK] = 0.0;
        if (!(rr > 0.0) || !isfinite(rr)) act[b] = 0;
    } else if (stage == FIN_RHO) {    // slot 0: (rh, r) -> beta into S_RV (read by the p update)
        const double rho = sum_part(part, b, 0, G);
        const double beta = (rho / s[S_RHO]) * (s[S_ALPHA] / s[S_OMEGA]);
        s[S_RV] = beta;
        s[S_RHO] = rho;
        if (!isfinite(beta) || rho == 0.0) { act[b] = 0; s[S_BREAK] = 1.0; }
    } else if (stage == FIN_ALPHA) {  // slot 0: (rh, v)
        const double rv = sum_part(part, b, 0, G);
        s[S_ALPHA] = s[S_RHO] / rv;
        if (!isfinite(s[S_ALPHA])) { act[b] = 0; s[S_BREAK] = 1.0; }
    } else if (stage == FIN_OMEGA) {  // slots 0, 1: (t, s), (t, t)
        const double ts = sum_part(part, b, 0, G), tt = sum_part(part, b, 1, G);
        s[S_OMEGA] = tt > 0.0 ? ts / tt : 0.0;
        s[S_TS] = ts;
        s[S_TT] = tt;
    } else {                          // slot 0: (r, r) after the update
        const double rr = sum_part(part, b, 0, G);
        s[S_RR] = rr;
        s[S_ITERS] += 1.0;
        if (sqrt(rr) <= rtol * s[S_BN] || s[S_ITERS] >= max_it || !isfinite(rr)) act[b] = 0;
        else if (s[S_OMEGA] == 0.0) { act[b] = 0; s[S_BREAK] = 1.0; }
    }
}

// the BiCGSTAB vector steps (instance b's vectors at vec + b * NV * n)
enum { VS_INIT, VS_P, VS_S, VS_X };
__global__ void k_fom_vec(double* vec, const double* sc, const int* act, int n, int B, int stage) {
    const int b = blockIdx.y;
    if (b >= B || !act[b]) return;
    double* V = vec + (size_t)b * NV * n;
    const double* s = sc + (size_t)b * NSC;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        if (stage == VS_INIT) {           // r = -r_newton already in V_R; xl = 0, rh = r, p = v = 0
            V[V_XL * n + k] = 0.0;
            V[V_RH * n + k] = V[V_R * n + k];
            V[V_P * n + k] = 0.0;
            V[V_V * n + k] = 0.0;
        } else if (stage == VS_P) {       // p = r + beta (p - omega v)
            V[V_P * n + k] = V[V_R * n + k] + s[S_RV] * (V[V_P * n + k] - s[S_OMEGA] * V[V_V * n + k]);
        } else if (stage == VS_S) {       // s = r - alpha v
            V[V_S * n + k] = V[V_R * n + k] - s[S_ALPHA] * V[V_V * n + k];
        } else {                          // xl += alpha ph + omega sh; r = s - omega t
            V[V_XL * n + k] += s[S_ALPHA] * V[V_PH * n + k] + s[S_OMEGA] * V[V_SH * n + k];
            V[V_R * n + k] = V[V_S * n + k] - s[S_OMEGA] * V[V_T * n + k];
        }
    }
}

// Newton update x += xl for the instances still iterating; the Newton residual r = -r(x) is formed next
__global__ void k_fom_update(double* vec, const int* nact, int n, int B) {
    const int b = blockIdx.y;
    if (b >= B || !nact[b]) return;
    double* V = vec + (size_t)b * NV * n;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) V[V_X * n + k] += V[V_XL * n + k];
}

__global__ void k_fom_neg(double* vec, const int* act, int n, int B) {
    const int b = blockIdx.y;
    if (b >= B || !act[b]) return;
    double* r = vec + (size_t)b * NV * n + V_R * n;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) r[k] = -r[k];
}

int ffail(ddnm_ctx* ctx, cudaError_t e, const char* what) {
    return ddnm_fail(ctx, DDNM_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define FK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return ffail(ctx, e_, #call);       \
    } while (0)

int fom_reserve(ddnm_ctx* ctx, FomWork*& W, int B) {
    if (!ctx->fom) ctx->fom = new FomWork();
    W = (FomWork*)ctx->fom;
    const int nx = ctx->nx, ny = ctx->ny;
    const size_t Nx = 2 * (size_t)nx * ny;
    if (!W->S) {
        W->nx = nx;
        W->ny = ny;
        // sine transform and the Thomas factors of every x-mode (host FP64, stored FP32)
        std::vector<float> S((size_t)nx * nx), cp((size_t)ny * nx), inv((size_t)ny * nx);
        const double pi = 3.14159265358979323846;
        for (int i = 0; i < nx; ++i)
            for (int k = 0; k < nx; ++k) S[(size_t)i * nx + k] = (float)std::sin(pi * (i + 1) * (k + 1) / (nx + 1));
        const double hx = ctx->hx, hy = ctx->hy, nu = ctx->nu;
        const double off = nu / (hy * hy);
        for (int k = 0; k < nx; ++k) {
            const double sk = std::sin(pi * (k + 1) / (2.0 * (nx + 1)));
            const double lam = -4.0 / (hx * hx) * sk * sk;
            const double diag = nu * (-2.0 / (hy * hy) + lam);
            double c = 0.0;
            for (int j = 0; j < ny; ++j) {
                const double piv = diag - off * c;
                c = off / piv;
                cp[(size_t)j * nx + k] = (float)c;
                inv[(size_t)j * nx + k] = (float)(1.0 / piv);
            }
        }
        FK(cudaMalloc(&W->S, S.size() * 4));
        FK(cudaMalloc(&W->cp, cp.size() * 4));
        FK(cudaMalloc(&W->inv, inv.size() * 4));
        FK(cudaMemcpy(W->S, S.data(), S.size() * 4, cudaMemcpyHostToDevice));
        FK(cudaMemcpy(W->cp, cp.data(), cp.size() * 4, cudaMemcpyHostToDevice));
        FK(cudaMemcpy(W->inv, inv.data(), inv.size() * 4, cudaMemcpyHostToDevice));
    }
    if (B > W->cap) {
        cudaFree(W->vec);
        cudaFree(W->tmp);
        cudaFree(W->bnd);
        cudaFree(W->mu);
        cudaFree(W->part);
        cudaFree(W->sc);
        cudaFree(W->act);
        if (W->h_sc) cudaFreeHost(W->h_sc);
        if (W->h_act) cudaFreeHost(W->h_act);
        W->vec = nullptr;
        W->tmp = nullptr;
        W->bnd = W->mu = W->part = W->sc = W->h_sc = nullptr;
        W->act = W->h_act = nullptr;
        W->cap = 0;
        if (cudaMalloc(&W->vec, (size_t)B * NV * Nx * 8) != cudaSuccess ||
            cudaMalloc(&W->tmp, (size_t)B * Nx * 4) != cudaSuccess ||
            cudaMalloc(&W->bnd, (size_t)B * 4 * (nx + ny) * 8) != cudaSuccess ||
            cudaMalloc(&W->mu, (size_t)B * 2 * 8) != cudaSuccess ||
            cudaMalloc(&W->part, (size_t)B * 4 * MAXG * 8) != cudaSuccess ||
            cudaMalloc(&W->sc, (size_t)B * NSC * 8) != cudaSuccess || cudaMalloc(&W->act, (size_t)B * 4) != cudaSuccess ||
            cudaMallocHost(&W->h_sc, (size_t)B * NSC * 8) != cudaSuccess ||
            cudaMallocHost(&W->h_act, (size_t)B * 4) != cudaSuccess) {
            (void)cudaGetLastError();
            return ddnm_fail(ctx, DDNM_E_NOMEM, "FOM workspace allocation failed for " + std::to_string(B) + " instances");
        }
        W->cap = B;
    }
    return DDNM_OK;
}

}  // namespace

void ddnm_fom_release(ddnm_ctx* ctx) {
    FomWork* W = (FomWork*)ctx->fom;
    if (!W) return;
    cudaFree(W->vec);
    cudaFree(W->tmp);
    cudaFree(W->S);
    cudaFree(W->cp);
    cudaFree(W->inv);
    cudaFree(W->bnd);
    cudaFree(W->mu);
    cudaFree(W->part);
    cudaFree(W->sc);
    cudaFree(W->act);
    if (W->h_sc) cudaFreeHost(W->h_sc);
    if (W->h_act) cudaFreeHost(W->h_act);
    delete W;
    ctx->fom = nullptr;
}

extern "C" int ddnm_fom_solve(ddnm_ctx* ctx, int B, const double* mu, const double* x0, double* x_out,
                              ddnm_fom_stats* stats, int max_newton, int max_krylov, int mem_kind, void* stream) {
    if (!ctx) return DDNM_E_INVALID;
    if (B < 1 || !mu || !x_out) return ddnm_fail(ctx, DDNM_E_INVALID, "ddnm_fom_solve: B >= 1, mu and x_out are required");
    if (mem_kind != DDNM_MEM_HOST && mem_kind != DDNM_MEM_DEVICE) return ddnm_fail(ctx, DDNM_E_INVALID, "bad mem_kind");
    if (max_newton < 1 || max_newton > 100 || max_krylov < 1 || max_krylov > 10000)
        return ddnm_fail(ctx, DDNM_E_INVALID, "ddnm_fom_solve: max_newton in 1..100, max_krylov in 1..10000");
    FK(cudaSetDevice(ctx->device));
    FomWork* W = nullptr;
    int rc = fom_reserve(ctx, W, B);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int nx = ctx->nx, ny = ctx->ny, N = nx * ny, Nx = 2 * N;
    const size_t stride = (size_t)NV * Nx;
    double* mu_d = W->mu;
    FK(cudaMemcpyAsync(mu_d, mu, (size_t)B * 16, mem_kind == DDNM_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
    FomDev F;
    F.nx = nx; F.ny = ny; F.N = N; F.Nx = Nx;
    F.hx = ctx->hx; F.hy = ctx->hy; F.nu = ctx->nu; F.bx0 = ctx->box[0]; F.by0 = ctx->box[2];
    F.ihx2 = 1.0 / (2.0 * F.hx); F.ihy2 = 1.0 / (2.0 * F.hy);
    F.lx = F.nu / (F.hx * F.hx); F.ly = F.nu / (F.hy * F.hy);
    F.mu = mu_d;
    F.bnd = W->bnd;
    const int nb = 2 * (nx + ny);
    k_fom_bnd<<<dim3((nb + FT - 1) / FT, B), FT, 0, st>>>(F, B);
    double* X = W->vec + V_X * (size_t)Nx;
    double* R = W->vec + V_R * (size_t)Nx;
    const dim3 gnode((N + FT - 1) / FT, B);
    if (x0) {
        for (int b = 0; b < B; ++b)
            FK(cudaMemcpyAsync(X + (size_t)b * stride, x0 + (size_t)b * Nx, (size_t)Nx * 8,
                               mem_kind == DDNM_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
    } else {
        k_fom_exact<<<gnode, FT, 0, st>>>(F, B, X, stride);
    }
    FK(cudaGetLastError());
    const int G = std::max(1, std::min(MAXG, (Nx + 4 * FT - 1) / (4 * FT)));
    const dim3 gdot(G, B), gvec(std::max(1, std::min(1024, (Nx + FT - 1) / FT)), B);
    const int gfin = (B + 127) / 128;
    // ---- helpers on the instance set `act` (device), all instances' vectors at stride
    auto dots = [&](int a0, int b0, int a1, int b1, const int* act) {
        k_fom_dots<<<gdot, FT, 0, st>>>(W->vec + (size_t)a0 * Nx, W->vec + (size_t)b0 * Nx,
                                        a1 < 0 ? nullptr : W->vec + (size_t)a1 * Nx,
                                        b1 < 0 ? nullptr : W->vec + (size_t)b1 * Nx, nullptr, nullptr, Nx, stride,
                                        W->part, B, act, G);
    };
    // M^{-1}: rows of (instance, component, j) x nx; x-sine transform, tridiagonal y solves, inverse transform
    auto precond = [&](int src, int dst, const int* act) {
        // every instance's Nx values are (2 ny) rows of nx: one batched product per transform
        const dim3 g1((nx + GB_N - 1) / GB_N, (2 * ny + GB_M - 1) / GB_M, B);
        k_fom_gemm<double, float><<<g1, 256, 0, st>>>(W->vec + (size_t)src * Nx, W->S, W->tmp, 2 * ny, nx, nx, 1.f,
                                                     stride, (size_t)Nx, act);
        k_fom_thomas<<<dim3((nx + 127) / 128, 2 * B), 128, 0, st>>>(W->tmp, W->cp, W->inv, B, nx, ny,
                                                                     (float)(ctx->nu / (ctx->hy * ctx->hy)), act);
        k_fom_gemm<float, double><<<g1, 256, 0, st>>>(W->tmp, W->S, W->vec + (size_t)dst * Nx, 2 * ny, nx, nx,
                                                     (float)(2.0 / (nx + 1)), (size_t)Nx, stride, act);
    };
    std::vector<int> newton_act(B, 1), it_newton(B, 0), it_krylov(B, 0), status(B, 1);
    std::vector<double> res0(B, 0.0), res(B, 0.0);
    int* nact_d = W->act;       // Newton-level activity lives on the host; the device flag is per linear solve
    // residual and its norm of every instance
    auto newton_residual = [&](std::vector<double>& out) -> int {
        for (int b = 0; b < B; ++b) W->h_act[b] = newton_act[b];
        FK(cudaMemcpyAsync(nact_d, W->h_act, (size_t)B * 4, cudaMemcpyHostToDevice, st));
        k_fom_res<<<gnode, FT, 0, st>>>(F, B, X, R, stride, nact_d);
        dots(V_R, V_R, -1, -1, nact_d);
        k_fom_fin<<<gfin, 128, 0, st>>>(W->sc, nact_d, W->part, B, G, FIN_INIT, 0.0, 0);
        FK(cudaMemcpyAsync(W->h_sc, W->sc, (size_t)B * NSC * 8, cudaMemcpyDeviceToHost, st));
        FK(cudaStreamSynchronize(st));
        for (int b = 0; b < B; ++b)
            if (newton_act[b]) out[b] = W->h_sc[(size_t)b * NSC + S_BN];
        return DDNM_OK;
    };
    rc = newton_residual(res0);
    if (rc) return rc;
    res = res0;
    std::vector<double> stop(B);
    for (int b = 0; b < B; ++b) {
        stop[b] = 1e-12 * std::max(1.0, res0[b]);
        if (!std::isfinite(res0[b])) { newton_act[b] = 0; status[b] = 2; }
        else if (res0[b] <= stop[b]) { newton_act[b] = 0; status[b] = 0; }
    }
    for (int itn = 0; itn < max_newton; ++itn) {
        int n_act = 0;
        for (int b = 0; b < B; ++b) n_act += newton_act[b];
        if (!n_act) break;
        // linear solve J dx = -r for the active instances (the scalars were set by newton_residual's FIN_INIT)
        for (int b = 0; b < B; ++b) W->h_act[b] = newton_act[b];
        FK(cudaMemcpyAsync(W->act, W->h_act, (size_t)B * 4, cudaMemcpyHostToDevice, st));
        k_fom_neg<<<gvec, FT, 0, st>>>(W->vec, W->act, Nx, B);
        k_fom_vec<<<gvec, FT, 0, st>>>(W->vec, W->sc, W->act, Nx, B, VS_INIT);
        for (int k = 0; k < max_krylov; ++k) {
            dots(V_RH, V_R, -1, -1, W->act);
            k_fom_fin<<<gfin, 128, 0, st>>>(W->sc, W->act, W->part, B, G, FIN_RHO, 0.0, 0);
            k_fom_vec<<<gvec, FT, 0, st>>>(W->vec, W->sc, W->act, Nx, B, VS_P);
            precond(V_P, V_PH, W->act);
            k_fom_jv<<<gnode, FT, 0, st>>>(F, B, X, W->vec + V_PH * (size_t)Nx, W->vec + V_V * (size_t)Nx, stride, W->act);
            dots(V_RH, V_V, -1, -1, W->act);
            k_fom_fin<<<gfin, 128, 0, st>>>(W->sc, W->act, W->part, B, G, FIN_ALPHA, 0.0, 0);
            k_fom_vec<<<gvec, FT, 0, st>>>(W->vec, W->sc, W->act, Nx, B, VS_S);
            precond(V_S, V_SH, W->act);
            k_fom_jv<<<gnode, FT, 0, st>>>(F, B, X, W->vec + V_SH * (size_t)Nx, W->vec + V_T * (size_t)Nx, stride, W->act);
            dots(V_T, V_S, V_T, V_T, W->act);
            k_fom_fin<<<gfin, 128, 0, st>>>(W->sc, W->act, W->part, B, G, FIN_OMEGA, 0.0, 0);
            k_fom_vec<<<gvec, FT, 0, st>>>(W->vec, W->sc, W->act, Nx, B, VS_X);
            dots(V_R, V_R, -1, -1, W->act);
            k_fom_fin<<<gfin, 128, 0, st>>>(W->sc, W->act, W->part, B, G, FIN_RES, 1e-10, max_krylov);
            if (k % 4 == 3 || k == max_krylov - 1) {
                FK(cudaMemcpyAsync(W->h_act, W->act, (size_t)B * 4, cudaMemcpyDeviceToHost, st));
                FK(cudaStreamSynchronize(st));
                int any = 0;
                for (int b = 0; b < B; ++b) any |= W->h_act[b];
                if (!any) break;
            }
        }
        FK(cudaMemcpyAsync(W->h_sc, W->sc, (size_t)B * NSC * 8, cudaMemcpyDeviceToHost, st));
        FK(cudaStreamSynchronize(st));
        for (int b = 0; b < B; ++b) {
            W->h_act[b] = newton_act[b];
            if (newton_act[b]) {
                it_krylov[b] += (int)W->h_sc[(size_t)b * NSC + S_ITERS];
                it_newton[b] += 1;
            }
        }
        FK(cudaMemcpyAsync(W->act, W->h_act, (size_t)B * 4, cudaMemcpyHostToDevice, st));
        k_fom_update<<<gvec, FT, 0, st>>>(W->vec, W->act, Nx, B);
        std::vector<double> prev = res;
        rc = newton_residual(res);
        if (rc) return rc;
        for (int b = 0; b < B; ++b) {
            if (!newton_act[b]) continue;
            if (!std::isfinite(res[b])) { newton_act[b] = 0; status[b] = 2; }
            else if (res[b] <= stop[b]) { newton_act[b] = 0; status[b] = 0; }
            else if (res[b] > 0.5 * prev[b]) {
                // no halving: the rounding floor (converged) if the residual is already tiny, else a stall
                newton_act[b] = 0;
                status[b] = res[b] <= 1e-8 * std::max(1.0, res0[b]) ? 0 : 1;
            }
        }
    }
    FK(cudaGetLastError());
    for (int b = 0; b < B; ++b)
        FK(cudaMemcpyAsync(x_out + (size_t)b * Nx, X + (size_t)b * stride, (size_t)Nx * 8,
                           mem_kind == DDNM_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
    if (stats) {
        for (int b = 0; b < B; ++b) {
            stats[b].newton_iters = it_newton[b];
            stats[b].krylov_iters = it_krylov[b];
            stats[b].status = status[b];
            stats[b].pad = 0;
            stats[b].res0 = res0[b];
            stats[b].res = res[b];
        }
    }
    if (mem_kind == DDNM_MEM_HOST) FK(cudaStreamSynchronize(st));
    return DDNM_OK;
}

// ------------------------------------------------------------------ arithmetic peaks (for roofline fractions)
//
// FP32 and FP64 fused multiply-add throughput of this device, measured: every thread runs 8 independent FMA
// chains (enough to cover the pipe latency) for `iters` steps; 2 flops per FMA.  The grid is 8 CTAs of 256
// threads per SM.  The result is written out so that the loop cannot be removed.
namespace {
template <typename T>
__global__ void __launch_bounds__(256) k_peak(T* out, int iters, T a, T b) {
    T x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == (T)-12345.678) out[threadIdx.x] = s;
}

template <typename T>
int time_peak(ddnm_ctx* ctx, int n_sm, int iters, double* tflops) {
    T* out = nullptr;
    if (cudaMalloc(&out, 256 * sizeof(T)) != cudaSuccess) return ddnm_fail(ctx, DDNM_E_NOMEM, "peak probe buffer");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int grid = 8 * n_sm;
    k_peak<T><<<grid, 256>>>(out, iters / 10, (T)0.999999, (T)1e-7);    // warm-up (clocks up)
    float best = 1e30f;
    for (int r = 0; r < 3; ++r) {
        cudaEventRecord(e0);
        k_peak<T><<<grid, 256>>>(out, iters, (T)0.999999, (T)1e-7);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        best = std::min(best, ms);
    }
    const cudaError_t e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return ffail(ctx, e, "peak probe");
    *tflops = 2.0 * 8.0 * iters * 256.0 * grid / (best * 1e-3) / 1e12;
    return DDNM_OK;
}
}  // namespace

extern "C" int ddnm_fom_residual(ddnm_ctx* ctx, int B, const double* mu, const double* x, double* r_out, int mem_kind,
                                 void* stream) {
    if (!ctx) return DDNM_E_INVALID;
    if (B < 1 || !mu || !x || !r_out) return ddnm_fail(ctx, DDNM_E_INVALID, "ddnm_fom_residual: B >= 1, mu, x, r_out");
    if (mem_kind != DDNM_MEM_HOST && mem_kind != DDNM_MEM_DEVICE) return ddnm_fail(ctx, DDNM_E_INVALID, "bad mem_kind");
    FK(cudaSetDevice(ctx->device));
    FomWork* W = nullptr;
    int rc = fom_reserve(ctx, W, B);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int nx = ctx->nx, ny = ctx->ny, N = nx * ny, Nx = 2 * N;
    const size_t stride = (size_t)NV * Nx;
    const cudaMemcpyKind in = mem_kind == DDNM_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const cudaMemcpyKind out = mem_kind == DDNM_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    FK(cudaMemcpyAsync(W->mu, mu, (size_t)B * 16, in, st));
    FomDev F;
    F.nx = nx; F.ny = ny; F.N = N; F.Nx = Nx;
    F.hx = ctx->hx; F.hy = ctx->hy; F.nu = ctx->nu; F.bx0 = ctx->box[0]; F.by0 = ctx->box[2];
    F.ihx2 = 1.0 / (2.0 * F.hx); F.ihy2 = 1.0 / (2.0 * F.hy);
    F.lx = F.nu / (F.hx * F.hx); F.ly = F.nu / (F.hy * F.hy);
    F.mu = W->mu;
    F.bnd = W->bnd;
    const int nb = 2 * (nx + ny);
    k_fom_bnd<<<dim3((nb + FT - 1) / FT, B), FT, 0, st>>>(F, B);
    double* X = W->vec + V_X * (size_t)Nx;
    double* R = W->vec + V_R * (size_t)Nx;
    for (int b = 0; b < B; ++b) FK(cudaMemcpyAsync(X + (size_t)b * stride, x + (size_t)b * Nx, (size_t)Nx * 8, in, st));
    k_fom_res<<<dim3((N + FT - 1) / FT, B), FT, 0, st>>>(F, B, X, R, stride, nullptr);
    FK(cudaGetLastError());
    for (int b = 0; b < B; ++b) FK(cudaMemcpyAsync(r_out + (size_t)b * Nx, R + (size_t)b * stride, (size_t)Nx * 8, out, st));
    if (mem_kind == DDNM_MEM_HOST) FK(cudaStreamSynchronize(st));
    return DDNM_OK;
}

extern "C" int ddnm_measure_peaks(ddnm_ctx* ctx, double* fp32_tflops, double* fp64_tflops) {
    if (!ctx || !fp32_tflops || !fp64_tflops) return DDNM_E_INVALID;
    FK(cudaSetDevice(ctx->device));
    int n_sm = 0;
    FK(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, ctx->device));
    int rc = time_peak<float>(ctx, n_sm, 1 << 16, fp32_tflops);
    if (!rc) rc = time_peak<double>(ctx, n_sm, 1 << 11, fp64_tflops);
    return rc;
}
