// sm_103a kernels of the batched Lagrange-Gauss-Newton SQP (Sec. 4.1) for the WFPC
// DD-LSPG-ROM with collocation HR (Sec. 3.1, 5.3) on steady 2D Burgers (Sec. 7.1).
//
// One SQP "pass" over the batch (or over one instance group of it inside the solve graph) is:
//   k_eval<T, RO, RG>  one CTA per (instance, subdomain), one launch per width class: the trial point,
//                      HR subnets of both decoders (Eq. subnet) with Jacobians, the collocated Burgers
//                      residual and its stencil partials (Eq. burgers_discretized), the chain rule
//                      R_i = dr/dx dg/dxh (Eq. gauss_newton_hessian b), H_i = R_i^T R_i, R_i^T r_i,
//                      D_i = C A_i dg^G/dxh, rho_i and ||rho_i||^2 (Eq. optimality_residuals_GN).
//   [k_dgemm<T>]       D_i batched over the instances that share a subdomain's decoder.
//   k_constraint<T>    Atil = C (sum_i A_i g_i^G) in FP64 over slices of the constraint rows, and in CTAs
//                      of its own the FP64 L D L^T of every block H_i with the Schur-sum shares.
//   k_kkt              one CTA per instance: merit ||F||_2, Armijo backtracking (Sec. 4.1),
//                      least-squares multiplier start (Sec. 7.2), the border of the Schur complement of
//                      Eq. (sqp_system), its FP64 solve and the update Eq. (sqp_update); in the solve graph
//                      its last CTA also runs the instance group's loop control.
// T is float (MIXED) or double (FP64).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "ddnm_ctx.h"

using namespace ddnm;

namespace {

template <typename T>
__device__ __forceinline__ void activation(int act, T z, T& s, T& ds) {
    if (act == DDNM_ACT_SWISH) {
        const T g = T(1) / (T(1) + exp(-z));
        s = z * g;
        ds = g + z * g * (T(1) - g);
    } else if (act == DDNM_ACT_SIGMOID) {
        const T g = T(1) / (T(1) + exp(-z));
        s = g;
        ds = g * (T(1) - g);
    } else {
        s = z;
        ds = T(1);
    }
}

// exact solution of the steady Burgers problem (Eq. burgers_pde_exact_solution), the Dirichlet data
__device__ void exact_uv(double x, double y, double a, double lam, double nu, double& u, double& v) {
    const double ep = exp(lam * (x - 1.0)), em = exp(-lam * (x - 1.0));
    const double cy = cos(lam * y), sy = sin(lam * y);
    const double psi = a * (1.0 + x) + (ep + em) * cy;
    u = -2.0 * nu * (a + lam * (ep - em) * cy) / psi;
    v = 2.0 * nu * lam * (ep + em) * sy / psi;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// v[0], v[s], ..., v[(n-1)s] summed as a pairwise tree over the values padded with zeros to a power of
// two (adding the zero subtrees is exact, so a slice of the tree computed elsewhere can be passed in as
// one value).  Streaming form: a stack of complete subtrees, merged like a binary counter.
__device__ double tree_sum(const double* v, int n, size_t s) {
    double stk[33];
    int top = 0;
    for (int i0 = 0; i0 < n; i0 += 8) {       // eight loads in flight, then merged in order
        double x8[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) x8[u] = i0 + u < n ? v[(size_t)(i0 + u) * s] : 0.0;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = i0 + u;
            if (i >= n) break;
            double x = x8[u];
            for (int k = i; k & 1; k >>= 1) x = stk[--top] + x;
            stk[top++] = x;
        }
    }
    double acc = top ? stk[--top] : 0.0;
    while (top) acc = stk[--top] + acc;
    return acc;
}

// (row, column) of entry e of a lower triangle stored row by row: e = i (i + 1) / 2 + k, 0 <= k <= i
__device__ __forceinline__ void tri_index(int e, int& i, int& k) {
    int r = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
    while (r * (r + 1) / 2 > e) --r;
    while ((r + 1) * (r + 2) / 2 <= e) ++r;
    i = r;
    k = e - r * (r + 1) / 2;
}

// Barrier over the n threads (a multiple of 32) of a thread range; bar 0 with n = blockDim is __syncthreads.
__device__ __forceinline__ void range_sync(int bar, int n) {
    asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(n) : "memory");
}

// Sum over the threads t < n of a thread range (barrier bar); every thread of the range gets the result.
__device__ double range_sum(double v, double* scratch /* >= 32 */, int t, int n, int bar) {
    v = warp_sum(v);
    range_sync(bar, n);
    if ((t & 31) == 0) scratch[t >> 5] = v;
    range_sync(bar, n);
    const double u = (t & 31) < (n >> 5) ? scratch[t & 31] : 0.0;
    return warp_sum(u);
}

// In-place A = L D L^T of the n x n symmetric row-major matrix A in shared memory (whole CTA): the
// strictly lower part becomes the unit lower factor L, the diagonal keeps D, rd[j] = 1 / D_jj.
// One reciprocal per pivot (no square root), and the next pivot is updated and inverted by thread 0
// while the other threads update the rest of the trailing matrix, so each column costs one barrier.
// Returns false (uniformly) when a pivot is not positive and finite.
__device__ bool block_ldl(double* A, double* rd, int n) {
    const int tid = threadIdx.x, nth = blockDim.x;
    __shared__ int s_ok;
    __syncthreads();
    if (tid == 0) {
        const double d = A[0];
        const int ok = (d > 0.0) && isfinite(d);
        s_ok = ok;
        rd[0] = ok ? 1.0 / d : 0.0;
    }
    __syncthreads();
    if (!s_ok) return false;
    // Warps w with w % 4 == 0 share warp 0's scheduler (and FP64 unit) under the usual warp-to-scheduler
    // assignment; while the trailing triangle fits the other warps in one pass they leave it to them, so that
    // warp 0's pivot chain has its FP64 unit alone.  The column scaling is warp 1's.
    const int w = tid >> 5, nw = nth >> 5;
    const int nwo = nw - (nw + 3) / 4;                       // warps off warp 0's scheduler
    const int wo = w - w / 4 - 1;                            // index among them (w % 4 != 0)
    for (int j = 0; j < n; ++j) {
        const double r = rd[j];
        const int m = n - j - 1;
        if (m > 0) {
            const int ntri = m * (m + 1) / 2;
            if (tid < 32) {          // warp 0: the next pivot and its reciprocal (the critical path)
                if (tid == 0) {
                    const double l = A[(j + 1) * n + j];
                    const double a = A[(j + 1) * n + j + 1] - l * r * l;
                    A[(j + 1) * n + j + 1] = a;
                    const long long ab = __double_as_longlong(a);
                    const int ok = ab > 0 && ab < 0x7FF0000000000000LL;   // positive and finite (integer test)
                    s_ok = ok;
                    rd[j + 1] = ok ? 1.0 / a : 0.0;
                }
            } else if (ntri - 1 <= 32 * nwo) {               // one pass over the warps off warp 0's scheduler
                if (w % 4 != 0) {
                    const int e = 32 * wo + (tid & 31) + 1;     // entry 0 is the pivot
                    if (e < ntri) {
                        int i, k;
                        tri_index(e, i, k);
                        const int ii = j + 1 + i, kk = j + 1 + k;
                        A[ii * n + kk] -= A[ii * n + j] * r * A[kk * n + j];
                    }
                }
            } else {                 // all warps but warp 0
                for (int e = tid - 32 + 1; e < ntri; e += nth - 32) {
                    int i, k;
                    tri_index(e, i, k);
                    const int ii = j + 1 + i, kk = j + 1 + k;
                    A[ii * n + kk] -= A[ii * n + j] * r * A[kk * n + j];
                }
            }
        }
        if (j > 0 && w == 1)
            for (int i = j + (tid & 31); i < n; i += 32) A[i * n + j - 1] *= rd[j - 1];
        __syncthreads();
        if (!s_ok) return false;
    }
    return true;
}

// x <- (L D L^T)^{-1} x with the factors of block_ldl (whole CTA; warp-synchronous when n <= 32).
__device__ void block_ldl_solve(const double* A, const double* rd, int n, double* x) {
    const int tid = threadIdx.x, nth = blockDim.x;
    if (n <= 32) {
        if (tid < 32) {              // lane i holds x_i; x_j of each step comes by a shuffle
            const int lane = tid;
            double xv = lane < n ? x[lane] : 0.0;
            for (int j = 0; j < n; ++j) {
                const double xj = __shfl_sync(0xffffffffu, xv, j);
                if (lane > j && lane < n) xv -= A[lane * n + j] * xj;
            }
            if (lane < n) xv *= rd[lane];
            for (int k = n - 1; k >= 0; --k) {
                const double xk = __shfl_sync(0xffffffffu, xv, k);
                if (lane < k) xv -= A[k * n + lane] * xk;
            }
            if (lane < n) x[lane] = xv;
        }
        __syncthreads();
        return;
    }
    for (int j = 0; j < n; ++j) {
        __syncthreads();
        const double xj = x[j];
        for (int i = j + 1 + tid; i < n; i += nth) x[i] -= A[i * n + j] * xj;
    }
    __syncthreads();
    for (int i = tid; i < n; i += nth) x[i] *= rd[i];
    for (int k = n - 1; k >= 0; --k) {
        __syncthreads();
        const double xk = x[k];
        for (int i = tid; i < k; i += nth) x[i] -= A[k * n + i] * xk;
    }
    __syncthreads();
}

// 4 consecutive values, 16-byte aligned (float4) or 32-byte aligned (two double2)
__device__ __forceinline__ void ld4(const float* p, float* o) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void ld4(const double* p, double* o) {
    const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
__device__ __forceinline__ void st4(float* p, const float* o) {
    *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
}
__device__ __forceinline__ void st4(double* p, const double* o) {
    reinterpret_cast<double2*>(p)[0] = make_double2(o[0], o[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(o[2], o[3]);
}

// One decoder output row of an ELL table in slot-major layout (Kp slots, a multiple of 8; padding slots
// hold column 0, value 0): acc[k] += sum_t val_t * hid[col_t][k] for k < R, i.e. the raw output (k = 0)
// and its Jacobian row (k >= 1) through the hidden records [sigma, sigma' W1].  The column and value loads
// of 8 slots are issued before their gathers so that 16 global loads per thread are in flight.
template <typename T, int R>
__device__ __forceinline__ void ell_accumulate(const int* col, const T* val, int stride, int Kp, const T* hid,
                                               T* acc) {
    for (int t0 = 0; t0 < Kp; t0 += 8) {
        int c[8];
        T v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            c[u] = col[(size_t)(t0 + u) * stride];
            v[u] = val[(size_t)(t0 + u) * stride];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const T* h = hid + (size_t)c[u] * R;
#pragma unroll
            for (int k = 0; k < R; k += 4) {
                T hv[4];
                ld4(h + k, hv);
                acc[k] += v[u] * hv[0];
                acc[k + 1] += v[u] * hv[1];
                acc[k + 2] += v[u] * hv[2];
                acc[k + 3] += v[u] * hv[3];
            }
        }
    }
}

// 32 consecutive decoder output rows of a dense-window tile, lane = row: acc[k] = sum_j val[lane][j] *
// hid[c0 + j][k] over the tile's window.  Every lane reads the same hidden record (one broadcast shared-
// memory wavefront per 16 bytes) and its own 4 window values per vector load (coalesced over the warp);
// three such loads are kept in flight ahead of their use.
template <typename T, int R>
__device__ __forceinline__ void tile_quad(const T* h, const T* v, T* acc) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const T* hr = h + u * R;
#pragma unroll
        for (int k = 0; k < R; k += 4) {
            T hv[4];
            ld4(hr + k, hv);
            acc[k] += v[u] * hv[0];
            acc[k + 1] += v[u] * hv[1];
            acc[k + 2] += v[u] * hv[2];
            acc[k + 3] += v[u] * hv[3];
        }
    }
}

template <typename T, int R>
__device__ __forceinline__ void tile_accumulate(const TileDev& TD, const T* V, const T* hid, int lane, T* acc) {
#pragma unroll
    for (int k = 0; k < R; ++k) acc[k] = T(0);
    const T* vp = V + TD.voff + lane * 4;
    const T* h = hid + (size_t)TD.c0 * R;
    const int tw = TD.tw;
    // three quads of window values in flight: b0, b1, b2 hold columns j, j + 4, j + 8
    T b0[4], b1[4] = {T(0), T(0), T(0), T(0)}, b2[4] = {T(0), T(0), T(0), T(0)};
    ld4(vp, b0);
    if (4 < tw) ld4(vp + 4 * 32, b1);
    if (8 < tw) ld4(vp + 8 * 32, b2);
    for (int j = 0; j < tw; j += 12) {
        tile_quad<T, R>(h + (size_t)j * R, b0, acc);
        if (j + 12 < tw) ld4(vp + (size_t)(j + 12) * 32, b0);
        if (j + 4 < tw) {
            tile_quad<T, R>(h + (size_t)(j + 4) * R, b1, acc);
            if (j + 16 < tw) ld4(vp + (size_t)(j + 16) * 32, b1);
        }
        if (j + 8 < tw) {
            tile_quad<T, R>(h + (size_t)(j + 8) * R, b2, acc);
            if (j + 20 < tw) ld4(vp + (size_t)(j + 20) * 32, b2);
        }
    }
}

// Values only (the first element of each hidden record, records STRIDE apart) of the 32 rows of a tile.
template <typename T, int STRIDE>
__device__ __forceinline__ T tile_values(const TileDev& TD, const T* V, const T* hid, int lane) {
    const T* vp = V + TD.voff + lane * 4;
    const T* h = hid + (size_t)TD.c0 * STRIDE;
    const int tw = TD.tw;
    T acc = T(0);
    for (int j = 0; j < tw; j += 8) {        // two quads of window values in flight
        T v[2][4];
#pragma unroll
        for (int q = 0; q < 2; ++q)
            if (j + 4 * q < tw) ld4(vp + (size_t)(j + 4 * q) * 32, v[q]);
#pragma unroll
        for (int q = 0; q < 2; ++q)
            if (j + 4 * q < tw) {
#pragma unroll
                for (int u = 0; u < 4; ++u) acc += v[q][u] * h[(size_t)(j + 4 * q + u) * STRIDE];
            }
    }
    return acc;
}

// Values only of one ELL row (slot-major, Kp slots), records STRIDE apart.
template <typename T, int STRIDE>
__device__ __forceinline__ T ell_values(const int* col, const T* val, int stride, int Kp, const T* hid) {
    T acc = T(0);
    for (int t0 = 0; t0 < Kp; t0 += 8) {
        int c[8];
        T v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            c[u] = col[(size_t)(t0 + u) * stride];
            v[u] = val[(size_t)(t0 + u) * stride];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) acc += v[u] * hid[(size_t)c[u] * STRIDE];
    }
    return acc;
}

// ------------------------------------------------------------------------ evaluation

// stencil constants 1/(2h_x), 1/(2h_y), nu/h_x^2, nu/h_y^2 in the value type (precomputed on the host)
template <typename T>
__device__ __forceinline__ T cst(const ProbDev& P, int k);
template <>
__device__ __forceinline__ float cst<float>(const ProbDev& P, int k) { return P.cstf[k]; }
template <>
__device__ __forceinline__ double cst<double>(const ProbDev& P, int k) { return P.cst[k]; }

// Barrier of one NT-thread group of an evaluation CTA (named barrier `bar`; the groups of a CTA work on
// different instances and never wait for each other).
template <int NT>
__device__ __forceinline__ void gsync(int bar) {
    asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(NT) : "memory");
}

// Trial point of this subdomain for the coming evaluation (ist[I_XTMODE]).  On a new SQP step the
// subdomain back-substitutes its own piece of the KKT solution of Eq. (sqp_system) from s_lambda, with the
// L D L^T factors of the accepted evaluation: s_i = -L^{-T} D^{-1} (t_i + [0; W_i s_lambda]) when H_i is PD,
// s_O = -L_OO^{-T} (D_O^{-1} t_O + L_GO^T s_G) with s_G from the step kernel when H_i is singular in its G
// block.  Then xt_i = x_i + alpha s_i (Eq. sqp_update); alpha = 1 on a new step.  The whole group stages
// L_i (n_i x n_i doubles) in shared memory (Ls) first, so the solve's warp reads no global memory in its loop.
template <int NT, int NGM>
__device__ void form_trial(const ProbDev& P, const SubDev& S, int b, double* z, double* Ls, int tid, int bar) {
    const int xm = P.ist[(size_t)b * INST_INTS + I_XTMODE];
    if (xm == XT_KEEP) return;
    const int nC = P.n_C, ni = S.ni, nO = S.nO, nG = S.nG;
    const double* x = P.x + (size_t)b * P.n_D + S.xoff;
    double* xt = P.xt + (size_t)b * P.n_D + S.xoff;
    double* s = P.s + (size_t)b * P.n_D + S.xoff;
    if (xm == XT_NEWSTEP) {
        {
            const double* blk = P.blk + (size_t)b * P.blk_stride + S.blk;
            const double* Lg = blk + blk_layout(ni, nG, nC).L;
            for (int e = tid; e < ni * ni; e += NT) Ls[e] = Lg[e];
        }
        gsync<NT>(bar);
        if (tid < 32) {
            const int lane = tid;
            const double* blk = P.blk + (size_t)b * P.blk_stride + S.blk;
            const BlkLayout BL = blk_layout(ni, nG, nC);
            const double* Li = Ls;
            const double* ri = blk + BL.rinv;
            const double* ti = blk + BL.t;
            const double* Wi = blk + BL.W;
            const double* y = P.slam + (size_t)b * nC;
            int nb;
            if (blk[BL.flag] == FLAG_PD) {
                double part[NGM];
#pragma unroll
                for (int k = 0; k < NGM; ++k) part[k] = 0.0;
                for (int c = lane; c < nC; c += 32) {
                    const double yc = y[c];
#pragma unroll
                    for (int k = 0; k < NGM; ++k)
                        if (k < nG) part[k] += Wi[k * nC + c] * yc;
                }
#pragma unroll
                for (int k = 0; k < NGM; ++k)
                    if (k < nG) part[k] = warp_sum(part[k]);
                if (lane < ni) {
                    double v = ti[lane];
#pragma unroll
                    for (int k = 0; k < NGM; ++k)
                        if (k < nG && lane == nO + k) v += part[k];
                    z[lane] = v * ri[lane];
                }
                nb = ni;
            } else {
                if (lane < nO) {
                    double v = ti[lane] * ri[lane];
                    for (int k = 0; k < nG; ++k) v += Li[(nO + k) * ni + lane] * s[nO + k];
                    z[lane] = v;
                }
                nb = nO;
            }
            for (int k = nb - 1; k >= 0; --k) {
                __syncwarp();
                const double zk = z[k];
                if (lane < k) z[lane] -= Li[k * ni + lane] * zk;
            }
            __syncwarp();
            if (lane < nb) s[lane] = -z[lane];
        }
        gsync<NT>(bar);
        if (tid < ni) xt[tid] = x[tid] + s[tid];
        if (tid < 32) {          // ||s_i||^2 and ||x_i||^2 after the merits in the header (the step test)
            const double a = warp_sum(tid < ni ? s[tid] * s[tid] : 0.0);
            const double c = warp_sum(tid < ni ? x[tid] * x[tid] : 0.0);
            if (tid == 0) {
                double* hdr = P.blk + (size_t)b * P.blk_stride + P.n_sub + 2 * S.phio;
                hdr[0] = a;
                hdr[1] = c;
            }
        }
    } else {
        const double alpha = P.dst[(size_t)b * INST_DBLS + D_ALPHA];
        if (tid < ni) xt[tid] = x[tid] + alpha * s[tid];
    }
    gsync<NT>(bar);
}

// One (instance, subdomain) evaluation.  RO = round4(n^O + 1) and RG = round4(n^G + 1) are the padded
// widths of the [value, Jacobian row] records; they are compile-time so that every inner loop has a fixed
// trip count (no predicated-off lanes).  Chunked over the collocation rows so that shared memory stays
// bounded for any subdomain size; every decoder table is read slot-major (consecutive threads ->
// consecutive addresses).
template <typename T, int RO, int RG>
__device__ void eval_item(const ProbDev& P, const SubDev& S, int b, unsigned char* smem, int tid, int bar) {
    constexpr int NT = eval_threads(sizeof(T), RO, RG);
    const EvalSmem L = eval_smem(S, P.n_C, (int)sizeof(T));
    T* sx = (T*)(smem + L.sx);
    T* hidO = (T*)(smem + L.hidO);
    T* hidG = (T*)(smem + L.hidG);
    T* outGn = (T*)(smem + L.outGn);
    T* outO = (T*)(smem + L.outO);
    T* Rr = (T*)(smem + L.Rr);
    double* dH = (double*)(smem + L.dH);
    double* drho = (double*)(smem + L.drho);
    double* dt = (double*)(smem + L.dt);
    double* dD = (double*)(smem + L.dD);
    T* red = (T*)(smem + L.red);
    T* Rt = (T*)(smem + L.Rt);                 // gappy POD: (Z_i Phi_i^r)^+ [R, r], nr x (n_i + 1)

    const T* V = (const T*)P.vpool;
    const int* IP = P.ipool;
    const int nth = NT;
    const int nO = S.nO, nG = S.nG, ni = S.ni, nC = P.n_C, NG = S.NG;
    const int ld = ni + 1;                 // Rr rows: [R row (n_i), r]
    constexpr int WO = RO - 1 > 0 ? ((RO - 1 + 3) & ~3) : 4;   // padded W1 row width of the interior subnet
    constexpr int WG = RG - 1 > 0 ? ((RG - 1 + 3) & ~3) : 4;

    // latent coordinates and multipliers of the trial point
    form_trial<NT, RG - 1>(P, S, b, dt, dH, tid, bar);  // n_i^G <= RG - 1; dH is free until the chunks end
    if (tid < ni) sx[tid] = (T)P.xt[(size_t)b * P.n_D + S.xoff + tid];
    gsync<NT>(bar);

    // hidden layers: rows [sigma(z), sigma'(z) W1[c, :], 0...]; the rows that pad each record array to a
    // multiple of 4 are zero (dense-window tiles may span them with zero values).  The interface subnet's
    // records serve the interface phase; the interior subnet's then take their place for the chunk loop.
    auto hidden_interior = [&]() {
        for (int e = tid; e < (round4(S.hO) - S.hO) * RO; e += nth) hidO[(size_t)S.hO * RO + e] = T(0);
        for (int c = tid; c < S.hO; c += nth) {
            const T* W1 = V + S.w1O + (size_t)c * round4(nO);
            T w[WO];
#pragma unroll
            for (int k = 0; k < WO; k += 4) {
                if (k < round4(nO)) ld4(W1 + k, w + k);
                else w[k] = w[k + 1] = w[k + 2] = w[k + 3] = T(0);
            }
            T z = V[S.b1O + c];
#pragma unroll
            for (int k = 0; k < WO; ++k) z += w[k] * (k < nO ? sx[k] : T(0));
            T s, ds;
            activation<T>(S.actO, z, s, ds);
            T row[RO];
            row[0] = s;
#pragma unroll
            for (int k = 1; k < RO; ++k) row[k] = (k - 1 < WO) ? ds * w[k - 1] : T(0);
#pragma unroll
            for (int k = 0; k < RO; k += 4) st4(hidO + (size_t)c * RO + k, row + k);
        }
    };
    for (int e = tid; e < (round4(S.hG) - S.hG) * RG; e += nth) hidG[(size_t)S.hG * RG + e] = T(0);
    for (int cc = tid; cc < S.hG; cc += nth) {
        const T* W1 = V + S.w1G + (size_t)cc * round4(nG);
        T w[WG];
#pragma unroll
        for (int k = 0; k < WG; k += 4) {
            if (k < round4(nG)) ld4(W1 + k, w + k);
            else w[k] = w[k + 1] = w[k + 2] = w[k + 3] = T(0);
        }
        T z = V[S.b1G + cc];
#pragma unroll
        for (int k = 0; k < WG; ++k) z += w[k] * (k < nG ? sx[nO + k] : T(0));
        T s, ds;
        activation<T>(S.actG, z, s, ds);
        T row[RG];
        row[0] = s;
#pragma unroll
        for (int k = 1; k < RG; ++k) row[k] = (k - 1 < WG) ? ds * w[k - 1] : T(0);
#pragma unroll
        for (int k = 0; k < RG; k += 4) st4(hidG + (size_t)cc * RG + k, row + k);
    }
    gsync<NT>(bar);

    const int nwarp = nth >> 5;
    const int w = tid >> 5, lane = tid & 31;

    // The interface phase (values of every interface output, records of those the stencils use, D_i) and the
    // interior outputs of a chunk, for threads t_ < n_ (warps w_ < nw_) of the group.
    auto interface_phase = [&](int t_, int n_, int w_, int nw_) {
        // interface decoder: values of every output (the constraint residual needs them all: Sec. 5.3's
        // remark, the WFPC constraint is not hyper-reduced), from the first element of the hidden records
        {
            T* gout = (T*)P.gG + (size_t)b * P.sum_NG + S.goff;
            const int tG = S.ntilesG;
            for (int t = w_; t < tG; t += nw_) {
                const T v = tile_values<T, RG>(P.tiles[S.tileG0 + t], V, hidG, lane);
                const int r = t * 32 + lane;
                if (r < NG) gout[r] = V[S.soG + NG + r] + V[S.soG + r] * v;
            }
            if (!tG)
                for (int r = t_; r < NG; r += n_) {
                    const T v = ell_values<T, RG>(IP + S.colG + r, V + S.valG + r, NG, S.Kp, hidG);
                    gout[r] = V[S.soG + NG + r] + V[S.soG + r] * v;
                }
        }
        // interface outputs the collocation stencils use: [y, Jacobian row] records
        for (int r = t_; r < S.NGn; r += n_) {
            T acc[RG];
    #pragma unroll
            for (int k = 0; k < RG; ++k) acc[k] = T(0);
            ell_accumulate<T, RG>(IP + S.colGn + r, V + S.valGn + r, S.NGn, S.Kp, hidG, acc);
            const T sc = V[S.soGn + r], off = V[S.soGn + S.NGn + r];
            acc[0] = off + sc * acc[0];
    #pragma unroll
            for (int k = 1; k < RG; ++k) acc[k] *= sc;
    #pragma unroll
            for (int k = 0; k < RG; k += 4) st4(outGn + (size_t)r * RG + k, acc + k);
        }
        // D_i = C A_i dg^G/dxh = Q_i P_G with Q_i = C A_i diag(scale) W2~ (n_C x h_G, precomputed, stored
        // transposed with rows of qld = round4(n_C) values) and P_G[h] = sigma'(z_h) W1~[h, :] (from the hidden
        // records).  Either here, thread (group, c) summing the hidden units h = group, group + n_grp, ... for
        // row c (eight Q loads in flight) and the groups added in order afterwards, or batched over the
        // instances that share the decoder (k_dgemm), for which P_G is written out.
        if (P.srpc) {                          // SRPC: D_i = A^_i, constant (Sec. 3.2)
            for (int o = t_; o < nC * nG; o += n_) dD[o] = P.Ahat[S.ahat + o];
            gsync<NT>(bar);
        } else if (P.d_gemm) {
            T* pg = (T*)P.PG + (size_t)b * P.pg_stride + S.pgoff;
            for (int e = t_; e < S.hG * nG; e += n_) {
                const int h = e / nG, k = e - h * nG;
                pg[e] = hidG[(size_t)h * RG + 1 + k];
            }
        } else {
            const int ngrp = n_ / nC;
            const int c = t_ % nC, grp = t_ / nC;
            if (grp < ngrp) {
                T acc[RG - 1];
    #pragma unroll
                for (int k = 0; k < RG - 1; ++k) acc[k] = T(0);
                const T* Qt = V + S.Qt;
                constexpr int U = 8;                               // loads in flight
                int h = grp;
                for (; h + (U - 1) * ngrp < S.hG; h += U * ngrp) {
                    T q[U];
    #pragma unroll
                    for (int u = 0; u < U; ++u) q[u] = Qt[(size_t)(h + u * ngrp) * P.qld + c];
    #pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const T* pr = hidG + (size_t)(h + u * ngrp) * RG + 1;
    #pragma unroll
                        for (int k = 0; k < RG - 1; ++k) acc[k] += q[u] * pr[k];
                    }
                }
                for (; h < S.hG; h += ngrp) {
                    const T q = Qt[(size_t)h * P.qld + c];
                    const T* pr = hidG + (size_t)h * RG + 1;
    #pragma unroll
                    for (int k = 0; k < RG - 1; ++k) acc[k] += q * pr[k];
                }
    #pragma unroll
                for (int k = 0; k < RG - 1; ++k)
                    if (k < nG) red[((size_t)grp * nC + c) * nG + k] = acc[k];
            }
            gsync<NT>(bar);
            for (int o = t_; o < nC * nG; o += n_) {
                T a = T(0);
                for (int g = 0; g < ngrp; ++g) a += red[(size_t)g * nC * nG + o];
                dD[o] = (double)a;
            }
        }
    };
    auto interior_outputs = [&](const ChunkDev& Cq, int t_, int n_, int w_, int nw_) {
    // interior decoder outputs of this chunk's collocation rows: dense-window tiles, warp per tile,
    // where the host built them; the ELL table otherwise
    {
        const int tO = Cq.ntiles;
        for (int t = w_; t < tO; t += nw_) {
            T acc[RO];
            tile_accumulate<T, RO>(P.tiles[Cq.tile0 + t], V, hidO, lane, acc);
            const int r = t * 32 + lane;
            if (r < Cq.m) {
                const T sc = V[Cq.so + r], off = V[Cq.so + Cq.m + r];
                acc[0] = off + sc * acc[0];
#pragma unroll
                for (int k = 1; k < RO; ++k) acc[k] *= sc;
#pragma unroll
                for (int k = 0; k < RO; k += 4) st4(outO + (size_t)r * RO + k, acc + k);
            }
        }
        const int mO = tO ? 0 : Cq.m;                 // rows left to the ELL table
        for (int r = t_; r < mO; r += n_) {
            T acc[RO];
#pragma unroll
            for (int k = 0; k < RO; ++k) acc[k] = T(0);
            ell_accumulate<T, RO>(IP + Cq.col + r, V + Cq.val + r, Cq.m, S.Kp, hidO, acc);
            const T sc = V[Cq.so + r], off = V[Cq.so + Cq.m + r];
            acc[0] = off + sc * acc[0];
#pragma unroll
            for (int k = 1; k < RO; ++k) acc[k] *= sc;
#pragma unroll
            for (int k = 0; k < RO; k += 4) st4(outO + (size_t)r * RO + k, acc + k);
        }
    }
    };
    // H_i = R^T R and R^T r.  Entry e < npair is the pair (a <= c) of H_i, entry npair + a is (R^T r)_a: the
    // product of columns a and c of the [R, r] rows.  Warp w sums the chunk rows w, w + nwarp, ... for the
    // entries lane, lane + 32, ... into its own running sums in shared memory (hp); after the chunks the
    // warps' sums are added in warp order, thread e taking entry e (gappy HR: thread e forms entry e from the
    // projected rows instead).
    const int npair = ni * (ni + 1) / 2, nent = npair + ni;
    auto entry_pair = [&](int e, int& a, int& c) {
        a = 0;
        c = 0;
        if (e < npair) {
            int rem = e;
            while (rem >= ni - a) {
                rem -= ni - a;
                ++a;
            }
            c = a + rem;
        } else if (e < nent) {
            a = e - npair;
            c = ni;
        }
    };
    int pa, pc;
    entry_pair(tid, pa, pc);
    T* hp = (T*)(smem + L.hp);
    int* hpair = (int*)(smem + L.hpair);
    for (int e = tid; e < nent; e += nth) {
        int a, c;
        entry_pair(e, a, c);
        hpair[e] = a | c << 16;
    }
    for (int e = tid; e < nwarp * nent; e += nth) hp[e] = T(0);   // read after the chunk's barriers
    T hacc = T(0);
    const int* hr = P.hr + (size_t)S.hr_off * HR_INTS;
    for (int e = tid; e < S.nr * ld; e += nth) Rt[e] = T(0);
    interface_phase(tid, nth, w, nwarp);
    gsync<NT>(bar);                              // the interface records are no longer read
    hidden_interior();
    gsync<NT>(bar);
    for (int q = 0; q < S.n_chunks; ++q) {
        const ChunkDev Cq = P.chunk[S.chunk0 + q];
        interior_outputs(Cq, tid, nth, w, nwarp);
        gsync<NT>(bar);
        // collocation rows of the chunk: tpr threads per row, thread `sub` of a row forming entries sub,
        // sub + tpr, ... of its [R row, r] (each entry sums the row's operands in the same order whatever tpr)
        const T* bnd = (const T*)P.bnd + (size_t)b * P.n_bnd * 2;
        const T ax = cst<T>(P, 0), ay = cst<T>(P, 1), cx = cst<T>(P, 2), cy = cst<T>(P, 3);
        const int tpr = S.hr_chunk < nth ? nth / S.hr_chunk : 1;
        const int sub = tid % tpr;
        for (int it = tid / tpr; it < Cq.nq; it += nth / tpr) {
            const int qq = Cq.q0 + it;
            const int comp = hr[qq];
            int code[6];
#pragma unroll
            for (int o = 0; o < 6; ++o) code[o] = hr[(size_t)(o + 1) * S.NB + qq];
            T f[6];
#pragma unroll
            for (int o = 0; o < 6; ++o) {
                const int kind = code[o] >> OP_SHIFT, idx = code[o] & OP_MASK;
                f[o] = kind == OP_INTERIOR ? outO[(size_t)idx * RO]
                                           : (kind == OP_INTERFACE ? outGn[(size_t)idx * RG] : bnd[idx]);
            }
            const T up = comp == 0 ? f[0] : f[5];
            const T vp = comp == 0 ? f[5] : f[0];
            const T dxf = f[1] - f[2], dyf = f[3] - f[4];
            const T r = -up * dxf * ax - vp * dyf * ay + cx * (f[1] - T(2) * f[0] + f[2]) +
                        cy * (f[3] - T(2) * f[0] + f[4]);
            T d[6];
            d[0] = -T(2) * cx - T(2) * cy - (comp == 0 ? dxf * ax : dyf * ay);
            d[1] = -up * ax + cx;
            d[2] = up * ax + cx;
            d[3] = -vp * ay + cy;
            d[4] = vp * ay + cy;
            d[5] = -(comp == 0 ? dyf * ay : dxf * ax);
            T* row = Rr + (size_t)it * ld;
            for (int k = sub; k <= ni; k += tpr) {
                // interior latents take the interior operands' Jacobian rows, interface latents the interface
                // operands'; entry n_i is the residual
                if (k == ni) {
                    row[k] = r;
                    continue;
                }
                const bool inner = k < nO;
                const int want = inner ? OP_INTERIOR : OP_INTERFACE;
                const T* base = inner ? outO + 1 + k : outGn + 1 + (k - nO);
                const int rs = inner ? RO : RG;
                T v = T(0);
#pragma unroll
                for (int o = 0; o < 6; ++o)
                    if ((code[o] >> OP_SHIFT) == want) v += d[o] * base[(size_t)(code[o] & OP_MASK) * rs];
                row[k] = v;
            }
            if (sub == 0 && P.r_hr) P.r_hr[(size_t)b * P.sum_NB + S.hr_off + qq] = (double)r;
        }
        gsync<NT>(bar);
        if (S.nr) {
            // gappy-POD HR (B_i = (Z_i Phi_i^r)^+ Z_i, Sec. 3.1): the projector's columns of this chunk's rows
            // applied to [R, r], summed over the chunks; entry e of Rt is one thread's
            const T* Pg = V + S.gp + Cq.q0;
            for (int e = tid; e < S.nr * ld; e += nth) {
                const int a = e / ld, j = e - a * ld;
                const T* pr = Pg + (size_t)a * S.NB;
                T acc = T(0);
                for (int ql = 0; ql < Cq.nq; ++ql) acc += pr[ql] * Rr[(size_t)ql * ld + j];
                Rt[e] += acc;
            }
        } else {
            for (int e = lane; e < nent; e += 32) {
                const int pk = hpair[e], a = pk & 0xFFFF, c = pk >> 16;
                T h0 = T(0), h1 = T(0);
                int ql = w;
                for (; ql + nwarp < Cq.nq; ql += 2 * nwarp) {
                    h0 += Rr[(size_t)ql * ld + a] * Rr[(size_t)ql * ld + c];
                    h1 += Rr[(size_t)(ql + nwarp) * ld + a] * Rr[(size_t)(ql + nwarp) * ld + c];
                }
                if (ql < Cq.nq) h0 += Rr[(size_t)ql * ld + a] * Rr[(size_t)ql * ld + c];
                hp[(size_t)w * nent + e] += h0 + h1;
            }
        }
        if (q + 1 < S.n_chunks) gsync<NT>(bar);   // outO / Rr reused by the next chunk
    }
    if (S.nr) {                                  // H_i and R_i^T r_i from the projected rows
        gsync<NT>(bar);
        if (tid < nent) {
            T h0 = T(0);
            for (int a = 0; a < S.nr; ++a) h0 += Rt[(size_t)a * ld + pa] * Rt[(size_t)a * ld + pc];
            hacc = h0;
        }
    } else {                                     // the warps' sums, added in warp order
        gsync<NT>(bar);
        if (tid < nent) {
            T h0 = T(0);
            for (int v = 0; v < nwarp; ++v) h0 += hp[(size_t)v * nent + tid];
            hacc = h0;
        }
    }
    if (tid < npair) {
        dH[pa * ni + pc] = (double)hacc;
        dH[pc * ni + pa] = (double)hacc;
    } else if (tid < npair + ni) {
        drho[pa] = (double)hacc;
    }
    gsync<NT>(bar);

    // H_i and rho_i = R_i^T r + E_i^T lambda (E_i = [0, D_i]) with phi_i = ||rho_i||^2 (in FP64: warp k forms
    // entry n^O + k, lanes over the multipliers), or R_i^T r alone when k_dgemm forms D_i and the rest
    double* blk = P.blk + (size_t)b * P.blk_stride + S.blk;
    const BlkLayout BL = blk_layout(ni, nG, nC);
    if (!P.d_gemm) {
        const int w2 = tid >> 5, l2 = tid & 31;
        const double* lam = P.lamt + (size_t)b * nC;
        for (int k = w2; k < nG; k += nwarp) {
            double v = 0.0;
            for (int c = l2; c < nC; c += 32) v += dD[c * nG + k] * lam[c];
            v = warp_sum(v);
            if (l2 == 0) drho[nO + k] += v;
        }
        gsync<NT>(bar);
        if (tid < 32) {
            const double r = tid < ni ? drho[tid] : 0.0;
            const double ph = warp_sum(r * r);
            if (tid == 0) P.blk[(size_t)b * P.blk_stride + S.phio] = ph;
        }
        for (int e = tid; e < nC * nG; e += nth) blk[BL.D + e] = dD[e];
    }
    for (int e = tid; e < ni * ni; e += nth) blk[BL.H + e] = dH[e];
    if (tid < ni) blk[BL.rho + tid] = drho[tid];
}

// One launch per class of subdomains sharing the padded record widths (RO, RG).  Items are (instance,
// subdomain of the class); item k is instance k % B of subdomain subs[k / B] (subs: the class's subdomains,
// largest first).  A CTA holds G = blockDim / NT independent groups (NT = eval_threads) (each with its own named
// barrier and shared-memory area of `stride` bytes) that take consecutive items, i.e. neighbouring
// instances of one subdomain, whose decoder tables they then share through L1.  With ctr == NULL group g of
// CTA c takes item c G + g; otherwise the grid is persistent and every group claims items from *ctr (zero
// before the launch) until none are left.
template <typename T, int RO, int RG>
__global__ void __launch_bounds__(eval_reg_threads(sizeof(T), RO, RG), 1)
    k_eval(ProbDev P, int B, const int* subs, int nsub, int* ctr, int stride) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int NT = eval_threads(sizeof(T), RO, RG);
    const int G = blockDim.x / NT, g = threadIdx.x / NT;
    const int tid = threadIdx.x - g * NT, bar = g + 1;
    unsigned char* gsm = smem + (size_t)g * stride;
    const int items = B * nsub;
    if (!ctr) {
        const int k = blockIdx.x * G + g;
        if (k >= items) return;
        const int b = k % B;
        if (P.ist[(size_t)b * INST_INTS + I_STATUS] != ST_RUNNING) return;
        eval_item<T, RO, RG>(P, P.sub[subs[k / B]], b, gsm, tid, bar);
        return;
    }
    __shared__ int s_item[4];
    for (;;) {
        if (tid == 0) s_item[g] = atomicAdd(ctr, 1);
        gsync<NT>(bar);
        const int k = s_item[g];
        gsync<NT>(bar);                       // every thread has its item before s_item is claimed again
        if (k >= items) return;
        const int b = k % B;
        if (P.ist[(size_t)b * INST_INTS + I_STATUS] != ST_RUNNING) continue;
        eval_item<T, RO, RG>(P, P.sub[subs[k / B]], b, gsm, tid, bar);
        gsync<NT>(bar);                       // shared memory is reused by the next item
    }
}

// host side: the kernel of a width class
template <typename T>
using EvalKernel = void (*)(ProbDev, int, const int*, int, int*, int);

template <typename T>
EvalKernel<T> eval_kernel(int ro, int rg) {
#define DDNM_EVAL_CASE(A, G) \
    if (ro == A && rg == G) return k_eval<T, A, G>;
    DDNM_EVAL_CASE(4, 4) DDNM_EVAL_CASE(4, 8) DDNM_EVAL_CASE(4, 12)
    DDNM_EVAL_CASE(8, 4) DDNM_EVAL_CASE(8, 8) DDNM_EVAL_CASE(8, 12)
    DDNM_EVAL_CASE(12, 4) DDNM_EVAL_CASE(12, 8) DDNM_EVAL_CASE(12, 12)
    DDNM_EVAL_CASE(16, 4) DDNM_EVAL_CASE(16, 8) DDNM_EVAL_CASE(16, 12)
#undef DDNM_EVAL_CASE
    return nullptr;
}

// k_dgemm shared memory: the staging area (also the reduction area afterwards), then TB x n_C multipliers
template <typename T, int CPT>
__host__ __device__ constexpr int dg_smem_main(int ncp) {
    return ((DG_KT * (ncp + (DG_THREADS / ncp) * CPT) > DG_THREADS * CPT ? DG_KT * (ncp + (DG_THREADS / ncp) * CPT)
                                                                           : DG_THREADS * CPT) *
                (int)sizeof(T) + 15) & ~15;
}

// D_i = C A_i dg_i^G/dxh = Q_i P_G (Eq. sqp_block_matrices) for the instances of one subdomain at once:
// Q_i (n_C x h_G, stored transposed) is shared by every instance, so the product over a tile of TB instances
// is a GEMM [n_C x h_G] x [h_G x (TB n^G)].  CTA (subdomain, instance tile); thread (c, g) owns row c of C;
// the thread groups g are split into column groups (CPT consecutive columns (instance, k) each) and, when
// the tile has few columns, into hidden-unit groups whose partial sums are added in order at the end.  h_G
// is walked in chunks of DG_KT staged in shared memory (Q rows coalesced, each instance's P_G slice
// contiguous).  Epilogue in FP64: D_i into the block, rho_i^G += D_i^T lambda (E_i = [0, D_i], Eq.
// optimality_residuals_GN) and phi_i = ||rho_i||^2.
template <typename T, int CPT>
__global__ void __launch_bounds__(DG_THREADS) k_dgemm(ProbDev P, int B, int TB) {
    extern __shared__ __align__(16) unsigned char dsm[];
    const int si = blockIdx.x, tid = threadIdx.x;
    const SubDev& S = P.sub[si];
    const int nC = P.n_C, nG = S.nG, nO = S.nO, ni = S.ni, hG = S.hG;
    const int ncp = (nC + 31) & ~31, ngrp = DG_THREADS / ncp;
    const int cols = TB * nG;
    const int cg = (cols + CPT - 1) / CPT;      // column groups (the host keeps cg <= ngrp)
    const int kg = ngrp / cg;                   // hidden-unit groups
    const int ncolp = cg * CPT;
    const int b0 = blockIdx.y * TB;
    if (b0 >= B) return;
    T* Qs = (T*)dsm;                            // DG_KT x ncp
    T* Ps = Qs + DG_KT * ncp;                   // DG_KT x ncolp
    __shared__ unsigned char run[DG_THREADS];
    for (int bl = tid; bl < TB; bl += DG_THREADS) {
        const int b = b0 + bl;
        run[bl] = b < B && P.ist[(size_t)b * INST_INTS + I_STATUS] == ST_RUNNING;
    }
    const int c = tid % ncp, g = tid / ncp;
    const int colg = g % cg, kgr = g / cg;
    const bool active = g < cg * kg;
    T acc[CPT];
#pragma unroll
    for (int j = 0; j < CPT; ++j) acc[j] = T(0);
    const T* Qt = (const T*)P.vpool + S.Qt;
    for (int h0 = 0; h0 < hG; h0 += DG_KT) {
        __syncthreads();
        for (int e = tid; e < DG_KT * ncp; e += DG_THREADS) {
            const int hh = e / ncp, cc = e - hh * ncp;
            Qs[e] = (h0 + hh < hG && cc < nC) ? Qt[(size_t)(h0 + hh) * P.qld + cc] : T(0);
        }
        for (int e = tid; e < TB * DG_KT * nG; e += DG_THREADS) {
            const int bl = e / (DG_KT * nG), rem = e - bl * DG_KT * nG;
            const int hh = rem / nG, k = rem - hh * nG;
            T v = T(0);
            if (h0 + hh < hG && run[bl])
                v = ((const T*)P.PG)[(size_t)(b0 + bl) * P.pg_stride + S.pgoff + (size_t)(h0 + hh) * nG + k];
            Ps[hh * ncolp + bl * nG + k] = v;
        }
        for (int e = tid; e < DG_KT * (ncolp - cols); e += DG_THREADS) {   // padding columns
            const int hh = e / (ncolp - cols), cc = e - hh * (ncolp - cols);
            Ps[hh * ncolp + cols + cc] = T(0);
        }
        __syncthreads();
        if (active) {
            const T* pr = Ps + colg * CPT;
            for (int hh = kgr; hh < DG_KT; hh += kg) {
                const T q = Qs[hh * ncp + c];
#pragma unroll
                for (int j = 0; j < CPT; j += 4) {
                    T pv[4];
                    ld4(pr + hh * ncolp + j, pv);
                    acc[j] += q * pv[0];
                    acc[j + 1] += q * pv[1];
                    acc[j + 2] += q * pv[2];
                    acc[j + 3] += q * pv[3];
                }
            }
        }
    }
    // partial sums of the hidden-unit groups, added in group order; multipliers of the tile's instances
    __syncthreads();
    T* red = (T*)dsm;                                            // kg x ncp x ncolp
    double* lam_s = (double*)(dsm + dg_smem_main<T, CPT>(ncp));  // TB x nC
    if (active)
#pragma unroll
        for (int j = 0; j < CPT; ++j) red[((size_t)kgr * ncp + c) * ncolp + colg * CPT + j] = acc[j];
    for (int e = tid; e < TB * nC; e += DG_THREADS) {
        const int b = b0 + e / nC;
        lam_s[e] = b < B ? P.lamt[(size_t)b * nC + e % nC] : 0.0;
    }
    __syncthreads();
    const BlkLayout BL = blk_layout(ni, nG, nC);
    for (int e = tid; e < nC * cols; e += DG_THREADS) {
        const int cc = e / cols, col = e - cc * cols;
        T v = T(0);
        for (int k = 0; k < kg; ++k) v += red[((size_t)k * ncp + cc) * ncolp + col];
        red[(size_t)cc * ncolp + col] = v;                       // this (c, col) is read by this thread only
        const int bl = col / nG, kk = col - bl * nG;
        if (run[bl]) P.blk[(size_t)(b0 + bl) * P.blk_stride + S.blk + BL.D + cc * nG + kk] = (double)v;
    }
    __syncthreads();
    for (int col = tid; col < cols; col += DG_THREADS) {
        const int bl = col / nG, k = col - bl * nG;
        if (!run[bl]) continue;
        double v = 0.0;
        for (int cc = 0; cc < nC; ++cc) v += (double)red[(size_t)cc * ncolp + col] * lam_s[bl * nC + cc];
        P.blk[(size_t)(b0 + bl) * P.blk_stride + S.blk + BL.rho + nO + k] += v;
    }
    __syncthreads();
    for (int bl = tid; bl < TB; bl += DG_THREADS) {
        if (!run[bl]) continue;
        double* blk = P.blk + (size_t)(b0 + bl) * P.blk_stride;
        double ph = 0.0;
        for (int jj = 0; jj < ni; ++jj) ph += blk[S.blk + BL.rho + jj] * blk[S.blk + BL.rho + jj];
        blk[S.phio] = ph;
    }
}

template <int NGM>
__device__ void factor_cta(const ProbDev& P, int b, int f, double* scr);

// Partial Atil over one slice of the constraint rows: jump_r = g_lo - g_hi (FP64, once per row), then
// Atil_c += sum_r C[c][r] jump_r, one warp per row c of C; partials per (instance, slice).  The rows c of C
// are split over nrg CTAs (the same sums, more SMs, when the batch alone gives too few CTAs).  CTA (x, b):
// x < n_split nrg takes slice x % n_split, row group x / n_split; the CTAs after them factor the
// Gauss-Newton blocks of the evaluated point for the step kernel (factor_cta), side by side in one launch.
template <typename T, int NGM>
__global__ void __launch_bounds__(CON_THREADS) k_constraint(ProbDev P, int B, int nrg) {
    extern __shared__ double jump[];      // con_split doubles (or the factorisation scratch)
    const int b = blockIdx.y, xi = blockIdx.x, ncon = P.n_split * nrg;
    if (b >= B) return;
    if (P.ist[(size_t)b * INST_INTS + I_STATUS] != ST_RUNNING) return;
    if (xi >= ncon) {
        factor_cta<NGM>(P, b, xi - ncon, jump);
        return;
    }
    const int sp = xi % P.n_split, rg = xi / P.n_split;
    if (P.srpc) {               // SRPC: Atil = sum_i A^_i xh_i^G (Sec. 3.2) into slice 0, the other slices zero
        const int rpg0 = (P.n_C + nrg - 1) / nrg;
        double* o0 = P.Atil + ((size_t)b * P.n_split + sp) * P.n_C;
        for (int c = rg * rpg0 + threadIdx.x; c < min(P.n_C, (rg + 1) * rpg0); c += blockDim.x) {
            double a = 0.0;
            if (sp == 0)
                for (int i = 0; i < P.n_sub; ++i) {
                    const SubDev& S = P.sub[i];
                    const double* Ai = P.Ahat + S.ahat + (size_t)c * S.nG;
                    const double* xg = P.xt + (size_t)b * P.n_D + S.xoff + S.nO;
                    for (int k = 0; k < S.nG; ++k) a += Ai[k] * xg[k];
                }
            o0[c] = a;
        }
        return;
    }
    const int r0 = sp * P.con_split, nr = min(P.con_split, P.N_A - r0);
    const T* g = (const T*)P.gG + (size_t)b * P.sum_NG;
    for (int r = threadIdx.x; r < nr; r += blockDim.x)
        jump[r] = (double)g[P.con_lo[r0 + r]] - (double)g[P.con_hi[r0 + r]];
    __syncthreads();
    // one warp per row c of C; the slice is cut into CON_BLOCK-row blocks (lane l sums rows l, l+32, ...
    // of a block, then a warp sum), and the blocks are combined as a pairwise tree.  With the step kernel
    // combining the slices the same way, Atil is one fixed pairwise tree over the blocks whatever the
    // slice size (a power of two times CON_BLOCK): the result does not depend on the launch plan.
    __shared__ double part[CON_THREADS / 32][MAX_CON_SPLIT / CON_BLOCK];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int nb = P.con_split / CON_BLOCK;
    double* out = P.Atil + ((size_t)b * P.n_split + sp) * P.n_C;
    const int rpg = (P.n_C + nrg - 1) / nrg;
    const int c1 = min(P.n_C, (rg + 1) * rpg);
    for (int c = rg * rpg + w; c < c1; c += nw) {
        const double* Cr = P.C + (size_t)c * P.N_A + r0;
        for (int k = 0; k < nb; ++k) {
            const int hi = min(nr, (k + 1) * CON_BLOCK);
            double acc = 0.0;
            for (int r = k * CON_BLOCK + lane; r < hi; r += 32) acc += Cr[r] * jump[r];
            acc = warp_sum(acc);
            if (lane == 0) part[w][k] = acc;
        }
        __syncwarp();
        if (lane == 0) out[c] = tree_sum(part[w], nb, 1);
        __syncwarp();
    }
}

// ------------------------------------------------------------------------ Atil in double-float (mixed path)

// a + b = s + e exactly (Knuth's TwoSum; the _rn intrinsics keep the compiler from contracting or reordering)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Atil partials of one slice of the constraint rows for a tile of instances, on the FP32 pipe, accurate to
// about 2^-48 of sum_l |C_kl jump_l| (Sec. 3.1: Atil = C sum_i A_i g_i^G = C jump).  C is shared by every
// instance, so a CTA stages a chunk of it once for TBI instances.  C is held split, C = C_hi + C_lo (two
// floats, transposed: Ct[l][c]); jump_l = g_lo - g_hi, the difference of two FP32 interface outputs, is held
// exactly as j_hi + j_lo (TwoSum).  A term C_kl jump_l is C_hi j_hi, exact as p + e with e from an FMA, plus
// the cross terms C_hi j_lo + C_lo j_hi (C_lo j_lo, below 2^-48 of the term, is left out).  p joins a running
// FP32 sum s through TwoSum, whose error, e and the cross terms join a second FP32 sum c: the accumulation of
// Ogita, Rump and Oishi's Dot2.  Every ATIL_FOLD rows s + c is added to an FP64 accumulator, which bounds the
// second-order error of Dot2 by that block length (about (64 u)^2 = 2^-36 in the worst case, u = 2^-24,
// typically near u^2).  CTA (slice, instance tile, row tile); thread: RM consecutive rows of C (by lane) x IM
// instances (by warp).  The partial of (instance, slice) goes where the FP64 slices put theirs.
template <int RM, int IM>
__global__ void __launch_bounds__(256) k_atil_df(ProbDev P, int B) {
    constexpr int RT = 32 * RM, TBI = 8 * IM, KC = ATIL_KC, JS = TBI + 1;
    __shared__ __align__(16) float Ch[KC * RT];
    __shared__ __align__(16) float Cl[KC * RT];
    __shared__ float Jh[KC * JS], Jl[KC * JS];
    __shared__ int s_run[TBI];
    __shared__ int s_any;
    const int tid = threadIdx.x, lane = tid & 31, wq = tid >> 5;
    const int sl = blockIdx.x, b0 = blockIdx.y * TBI, c0 = blockIdx.z * RT;
    const int k0 = sl * P.con_split, k1 = min(P.N_A, k0 + P.con_split);
    if (tid == 0) s_any = 0;
    __syncthreads();
    if (tid < TBI) {
        const int b = b0 + tid;
        const int r = b < B && P.ist[(size_t)b * INST_INTS + I_STATUS] == ST_RUNNING;
        s_run[tid] = r;
        if (r) s_any = 1;
    }
    __syncthreads();
    if (!s_any) return;
    const float* g = (const float*)P.gG;
    float s[RM][IM], c[RM][IM];
    double acc[RM][IM];
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < IM; ++j) {
            s[i][j] = c[i][j] = 0.f;
            acc[i][j] = 0.0;
        }
    for (int k = k0; k < k1; k += KC) {
        __syncthreads();
        for (int e = tid; e < KC * RT / 4; e += 256) {          // C chunk: KC rows of Ct, RT values each
            const int kk = e / (RT / 4), q = e - kk * (RT / 4);
            float4 h = make_float4(0.f, 0.f, 0.f, 0.f), l = h;
            if (k + kk < k1) {
                const size_t o = (size_t)(k + kk) * P.ldct + c0 + 4 * q;
                h = *reinterpret_cast<const float4*>(P.Cthi + o);
                l = *reinterpret_cast<const float4*>(P.Ctlo + o);
            }
            reinterpret_cast<float4*>(Ch)[e] = h;
            reinterpret_cast<float4*>(Cl)[e] = l;
        }
        for (int e = tid; e < KC * TBI; e += 256) {             // jumps of the tile's instances, exact
            const int inst = e / KC, kk = e - inst * KC;
            float hi = 0.f, lo = 0.f;
            if (k + kk < k1 && s_run[inst]) {
                const float* gb = g + (size_t)(b0 + inst) * P.sum_NG;
                two_sum(gb[P.con_lo[k + kk]], -gb[P.con_hi[k + kk]], hi, lo);
            }
            Jh[kk * JS + inst] = hi;
            Jl[kk * JS + inst] = lo;
        }
        __syncthreads();
#pragma unroll 2
        for (int kk = 0; kk < KC; ++kk) {
            float ch[RM], cl[RM], jh[IM], jl[IM];
            if constexpr (RM == 4) {
                const float4 a = reinterpret_cast<const float4*>(Ch + kk * RT)[lane];
                const float4 b = reinterpret_cast<const float4*>(Cl + kk * RT)[lane];
                ch[0] = a.x; ch[1] = a.y; ch[2] = a.z; ch[3] = a.w;
                cl[0] = b.x; cl[1] = b.y; cl[2] = b.z; cl[3] = b.w;
            } else if constexpr (RM == 2) {
                const float2 a = reinterpret_cast<const float2*>(Ch + kk * RT)[lane];
                const float2 b = reinterpret_cast<const float2*>(Cl + kk * RT)[lane];
                ch[0] = a.x; ch[1] = a.y;
                cl[0] = b.x; cl[1] = b.y;
            } else {
                ch[0] = Ch[kk * RT + lane];
                cl[0] = Cl[kk * RT + lane];
            }
#pragma unroll
            for (int j = 0; j < IM; ++j) {
                jh[j] = Jh[kk * JS + wq * IM + j];
                jl[j] = Jl[kk * JS + wq * IM + j];
            }
#pragma unroll
            for (int i = 0; i < RM; ++i)
#pragma unroll
                for (int j = 0; j < IM; ++j) {
                    const float p = __fmul_rn(ch[i], jh[j]);
                    const float e = __fmaf_rn(ch[i], jh[j], -p);        // ch jh - p, exactly
                    float t, q;
                    two_sum(s[i][j], p, t, q);
                    s[i][j] = t;
                    float cc = __fadd_rn(c[i][j], __fadd_rn(q, e));
                    cc = __fmaf_rn(ch[i], jl[j], cc);
                    c[i][j] = __fmaf_rn(cl[i], jh[j], cc);
                }
        }
        if ((k - k0 + KC) % ATIL_FOLD == 0 || k + KC >= k1) {
#pragma unroll
            for (int i = 0; i < RM; ++i)
#pragma unroll
                for (int j = 0; j < IM; ++j) {
                    acc[i][j] += (double)s[i][j] + (double)c[i][j];
                    s[i][j] = c[i][j] = 0.f;
                }
        }
    }
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < IM; ++j) {
            const int cr = c0 + RM * lane + i, inst = wq * IM + j;
            if (cr < P.n_C && s_run[inst]) P.Atil[((size_t)(b0 + inst) * P.n_split + sl) * P.n_C + cr] = acc[i][j];
        }
}

// the double-float Atil launch of a pass: instance tiles of 32, 16 or 8 (by batch), row tiles of ldct rows up to
// 128; the summation order of an entry does not depend on either, so the result does not depend on the plan
cudaError_t launch_atil(ddnm_ctx* ctx, const ProbDev& P, int B, cudaStream_t st) {
    const int RT = std::min(P.ldct, 128), IM = B >= 32 ? 4 : (B >= 16 ? 2 : 1), TBI = 8 * IM;
    const dim3 grid(P.n_split, (B + TBI - 1) / TBI, P.ldct / RT);
#define DDNM_ATIL(R, I) \
    if (RT == 32 * R && IM == I) k_atil_df<R, I><<<grid, 256, 0, st>>>(P, B);
    DDNM_ATIL(1, 1) DDNM_ATIL(1, 2) DDNM_ATIL(1, 4) DDNM_ATIL(2, 1) DDNM_ATIL(2, 2) DDNM_ATIL(2, 4)
    DDNM_ATIL(4, 1) DDNM_ATIL(4, 2) DDNM_ATIL(4, 4)
#undef DDNM_ATIL
    (void)ctx;
    return cudaGetLastError();
}

// CTAs per (slice, instance) of k_constraint over the rows of C: about two CTAs per SM in all, at least one
// row of C per warp
int con_row_groups(const ddnm_ctx* ctx, const ProbDev& P, int B) {
    const int base = std::max(1, B * P.n_split);
    const int want = (2 * (ctx->n_sm > 0 ? ctx->n_sm : 148) + base - 1) / base;
    const int most = (P.n_C + CON_THREADS / 32 - 1) / (CON_THREADS / 32);
    return std::max(1, std::min(want, most));
}

// ------------------------------------------------------------------------ SQP step

// FP64 factorisation of the Gauss-Newton blocks of 32 / LG subdomains of one instance at an accepted point, one
// warp, LG lanes for each (n_i <= 16): every FP64 instruction, the pivot reciprocals included, serves all of
// them.  H_i = L D L^T (unit lower L, one reciprocal per pivot), t = L^{-1} rho_i, W = L_GG^{-1} D_i^T (the
// Omega rows of L^{-1} E_i^T vanish), u_i = W^T D_G^{-1} t_G.  Lemma 1 only needs H_i PD on null(E_i): when the
// collocation rows miss an interface direction, H_i is singular in its G block while H_i^{OO} is PD; the
// factorisation of that subdomain then stops after the O columns and it is handled through
// G = H_GG - L_GO D_O L_GO^T (snapshot after the O columns).  Subdomains i_first .. i_first + 32/LG - 1 below
// ns; scratch (32 / LG) fs doubles; flags (FLAG_PD, FLAG_OMEGA_FAIL, FLAG_GAMMA_SING as 0, 1, 2) to fl[] and
// the blocks.  A pivot is accepted when its bits are those of a positive finite double (integer tests) and it
// exceeds P.piv_eps times the block's largest diagonal entry (below that it is the rounding remainder of a
// direction the collocation rows miss, and the block takes the second Schur level).
// Columns are taken two at a time where the lane groups allow (one reciprocal per pair), else one at a time.
template <int LG, int NGM>
__device__ void factor_group(const ProbDev& P, double* blk, const int* s_blk, const unsigned char* s_nO,
                             const unsigned char* s_nG, int i_first, int ns, double* scr, int fs, unsigned char* fl,
                             const unsigned short* tri) {
    const int lane = threadIdx.x & 31, half = lane / LG, hl = lane % LG, nC = P.n_C;
    const int i = i_first + half < ns ? i_first + half : -1;
    const bool on = i >= 0;
    const int nO = on ? s_nO[i] : 0, nG = on ? s_nG[i] : 0, ni = nO + nG;
    const BlkLayout BL = blk_layout(ni, nG, nC);
    double* bi = on ? blk + s_blk[i] : nullptr;
    double* L = scr + (size_t)half * fs;
    double* t = L + ni * ni;
    double* rinv = t + ni;
    double* ucol = rinv + ni;                   // column j before its scaling
    double* ucol2 = ucol + ni;                  // column j + 1 of a paired step, updated by column j, unscaled
    double* G = ucol2 + ni;
    int nmax = 0;
    for (int q = 0; q < 32 / LG && i_first + q < ns; ++q) nmax = max(nmax, (int)s_nO[i_first + q] + s_nG[i_first + q]);
    double dpre[2][NGM];                        // D_i[c][:] for c = hl, hl + LG, loaded ahead of the pivots
#pragma unroll
    for (int q = 0; q < NGM; ++q) dpre[0][q] = dpre[1][q] = 0.0;
    if (on) {
        for (int e = hl; e < ni * ni; e += LG) L[e] = bi[BL.H + e];
        for (int e = hl; e < ni; e += LG) t[e] = bi[BL.rho + e];
#pragma unroll
        for (int u = 0; u < 2; ++u)
            if (hl + u * LG < nC) {
#pragma unroll
                for (int q = 0; q < NGM; ++q)
                    if (q < nG) dpre[u][q] = bi[BL.D + (hl + u * LG) * nG + q];
            }
    }
    __syncwarp();
    int flag = 0, nf = 0;                       // this half's subdomain: flag and factored columns
    bool act = on;
    auto posfin = [](double v) {                // positive and finite (integer test)
        const long long vb = __double_as_longlong(v);
        return vb > 0 && vb < 0x7FF0000000000000LL;
    };
    // pivots at or below thr are rounding remainders (a direction no collocation row sees): rank test
    double thr = 0.0;
    if (on) {
        for (int j = 0; j < ni; ++j) thr = fmax(thr, L[j * ni + j]);
        thr *= P.piv_eps;
    }
    for (int j = 0; j < nmax;) {
        if (act && j == nO)
            for (int e = hl; e < nG * nG; e += LG) G[e] = L[(nO + e / nG) * ni + nO + e % nG];
        __syncwarp();
        // Two columns at once where every live lane group can: the 2 x 2 block [a b; b c] of columns j, j + 1
        // (both in the O block or both in the G block) has a > 0 and det = a c - b^2 > 0.  One reciprocal
        // q = 1 / (a det) gives both pivots' reciprocals: 1 / d_j = det q and 1 / d_{j+1} = a / det = a (a q).
        const bool live = act && j < ni;
        double pa = 0.0, pb = 0.0, pdet = 0.0;
        bool pair_ok = false;
        if (live && j + 1 < ni && !(j < nO && j + 1 >= nO)) {
            pa = L[j * ni + j];
            pb = L[(j + 1) * ni + j];
            const double pc = L[(j + 1) * ni + j + 1];
            pdet = fma(pa, pc, -(pb * pb));
            pair_ok = posfin(pa) && posfin(pdet) && pa > thr && pdet > thr * pa;
        }
        if (__all_sync(0xffffffffu, !live || pair_ok)) {
            if (live) {
                const double q = 1.0 / (pa * pdet);
                const double ra = pdet * q, rdet = pa * q, r1 = pa * rdet;
                for (int ii = j + 2 + hl; ii < ni; ii += LG) {   // columns j and j + 1 below the block
                    const double u = L[ii * ni + j], v = L[ii * ni + j + 1];
                    const double l0 = u * ra;
                    const double v1 = v - l0 * pb;              // column j + 1 updated by column j
                    ucol[ii] = u;
                    ucol2[ii] = v1;
                    L[ii * ni + j] = l0;
                    L[ii * ni + j + 1] = v1 * r1;
                }
                if (hl == 0) {
                    L[(j + 1) * ni + j] = pb * ra;
                    L[(j + 1) * ni + j + 1] = pdet * ra;         // d_{j+1}
                    rinv[j] = ra;
                    rinv[j + 1] = r1;
                }
                nf = j + 2;
            }
            __syncwarp();
            const int m = ni - j - 2;
            if (live && m > 0) {
                for (int e = hl; e < m * (m + 1) / 2; e += LG) {   // trailing triangle: columns j, then j + 1
                    const int ta = tri[e] >> 8, tc = tri[e] & 255;
                    const int ii = j + 2 + ta, kk = j + 2 + tc;
                    double x = L[ii * ni + kk];
                    x -= L[ii * ni + j] * ucol[kk];
                    x -= L[ii * ni + j + 1] * ucol2[kk];
                    L[ii * ni + kk] = x;
                }
            }
            __syncwarp();
            j += 2;
            continue;
        }
        double r = 0.0;
        bool piv = false;
        if (live) {
            const double d = L[j * ni + j];
            if (!posfin(d) || d <= thr) {       // not positive and finite, or numerically zero
                flag = j < nO ? 1 : 2;
                act = false;
            } else {
                r = 1.0 / d;
                nf = j + 1;
                piv = true;
            }
        }
        const int m = ni - j - 1;
        if (piv) {                                           // column j of L, keeping the unscaled one
            for (int ii = j + 1 + hl; ii < ni; ii += LG) {
                const double a = L[ii * ni + j];
                ucol[ii] = a;
                L[ii * ni + j] = a * r;
            }
            if (hl == 0) rinv[j] = r;
        }
        __syncwarp();
        if (piv && m > 0) {
            for (int e = hl; e < m * (m + 1) / 2; e += LG) {     // trailing lower triangle: (a_ij / d_j) a_kj
                const int a = tri[e] >> 8, c = tri[e] & 255;
                const int ii = j + 1 + a, kk = j + 1 + c;
                L[ii * ni + kk] -= L[ii * ni + j] * ucol[kk];
            }
        }
        __syncwarp();
        ++j;
    }
    // t = L^{-1} rho over the factored columns (n_f = n_i when PD, n^O when G-singular)
    const int nft = flag == 0 ? ni : (flag == 2 ? nO : 0);
    for (int j = 0; j < nmax; ++j) {
        const double tj = j < nft ? t[j] : 0.0;
        if (j < nft)
            for (int ii = j + 1 + hl; ii < ni; ii += LG) t[ii] -= L[ii * ni + j] * tj;
        __syncwarp();
    }
    (void)nf;
    if (on) {
        if (flag != 1) {
            for (int e = hl; e < ni * ni; e += LG) bi[BL.L + e] = L[e];
            for (int e = hl; e < ni; e += LG) {
                bi[BL.t + e] = t[e];
                bi[BL.rinv + e] = rinv[e];
            }
        }
        if (flag == 2)
            for (int e = hl; e < nG * nG; e += LG) bi[BL.G + e] = G[e];
        if (flag == 0) {
            for (int c = hl; c < nC; c += LG) {
                double wv[NGM];
                double uc = 0.0;
#pragma unroll
                for (int q = 0; q < NGM; ++q) {
                    if (q < nG) {
                        double v = c == hl ? dpre[0][q] : (c == hl + LG ? dpre[1][q] : bi[BL.D + c * nG + q]);
#pragma unroll
                        for (int mm = 0; mm < q; ++mm) v -= L[(nO + q) * ni + nO + mm] * wv[mm];
                        wv[q] = v;
                        bi[BL.W + q * nC + c] = v;
                        uc += v * rinv[nO + q] * t[nO + q];
                    }
                }
                bi[BL.u + c] = uc;
            }
        }
        if (hl == 0) {
            bi[BL.flag] = (double)flag;
            fl[i] = (unsigned char)flag;
        }
    }
    __syncwarp();
}

// Factor CTA f of instance b (a role of k_constraint): the Gauss-Newton blocks of subdomains 8f .. 8f + 7 of
// the evaluated point, FP64, one warp per pair (a half-warp each) on warps 0-3, i.e. one per scheduler and FP64
// unit under the usual warp-to-scheduler assignment; the other warps idle.  The CTAs of an instance spread
// over SMs, where the step kernel's one CTA would take the blocks on one SM's four FP64 units.  Every
// evaluation is factored (the step kernel decides afterwards whether the point is accepted; a rejected
// trial's factors are never read: a backtrack forms its trial point from s).  Then, when the staging fits
// (P.Spart set), the CTA's share of the Schur sums of the KKT step.  scr: ctx->fac_smem bytes, i.e.
// 8 fac_stride doubles, or (2 fac_rows + 8) n_C doubles with the shares.
template <int NGM>
__device__ void factor_cta(const ProbDev& P, int b, int f, double* scr) {
    constexpr int SPC = 2 * FAC_WARPS;                          // subdomains per CTA
    __shared__ int s_blk[SPC];
    __shared__ unsigned char s_nO[SPC], s_nG[SPC], s_fl[SPC];
    __shared__ unsigned short tri[MAX_TRI];                     // (row << 8 | column) of triangle entry e
    __shared__ int s_skip;
    const int i0 = f * SPC, tid = threadIdx.x, w = tid >> 5;
    if (i0 >= P.n_sub) return;
    const int nrel = min(SPC, P.n_sub - i0);
    // A trial the step kernel is bound to reject needs no factors: phi^2 = ||F||^2 >= sum_i ||rho_i||^2, so
    // when the subdomain residuals alone exceed the Armijo bound (with a relative margin of 1e-12 for the
    // order of summation) the trial fails; so does the start-up pass, which only forms the multiplier.
    if (w == 0) {
        const int* ist = P.ist + (size_t)b * INST_INTS;
        const double* dst = P.dst + (size_t)b * INST_DBLS;
        const int mode = ist[I_MODE], nbt = ist[I_NBT];
        const double alpha = dst[D_ALPHA], phi0 = dst[D_PHI0];
        const double* hdr = P.blk + (size_t)b * P.blk_stride;   // the merits ||rho_i||^2, subdomain i at index i
        double sphi = 0.0;
        for (int i = tid; i < P.n_sub; i += 32) sphi += hdr[i];
        sphi = warp_sum(sphi);
        if (tid == 0)
            s_skip = mode == MODE_INIT0 ||
                     (mode == MODE_LS && nbt < P.max_bt &&
                      sphi > (1.0 - 2.0 * P.c1 * alpha) * phi0 * phi0 * (1.0 + 1e-12));
    }
    for (int e = tid; e < MAX_TRI; e += blockDim.x) {
        int a, c;
        tri_index(e, a, c);
        tri[e] = (unsigned short)(a << 8 | c);
    }
    if (tid < nrel) {
        const SubDev& S = P.sub[i0 + tid];
        s_blk[tid] = S.blk;
        s_nO[tid] = (unsigned char)S.nO;
        s_nG[tid] = (unsigned char)S.nG;
    }
    __syncthreads();
    if (s_skip) return;
    double* blk = P.blk + (size_t)b * P.blk_stride;
    if (w < FAC_WARPS && 2 * w < nrel)
        factor_group<16, NGM>(P, blk, s_blk, s_nO, s_nG, 2 * w, nrel, scr + (size_t)w * 2 * P.fac_stride, P.fac_stride,
                         s_fl, tri);
    if (!P.Spart) return;          // the KKT step forms the Schur sums itself
    __syncthreads();               // the CTA's blocks factored: W_i, 1 / D_jj, u_i and the flags written
    // the CTA's share of the border of the Schur complement of Eq. (sqp_system): over its subdomains with H_i
    // PD, sum W_i^T D_G,i^{-1} W_i (lower triangle) and sum u_i, rows in subdomain order (k ascending in one);
    // the KKT step adds the shares of an instance in CTA order
    const int nC = P.n_C, ntri = nC * (nC + 1) / 2;
    int rows = 0;
    for (int q = 0; q < nrel; ++q) rows += s_nG[q];
    double* Wsh = scr;                          // rows x nC
    double* Wr = Wsh + (size_t)rows * nC;       // rows x nC, row k scaled by 1 / D_kk
    double* Us = Wr + (size_t)rows * nC;        // nrel x nC
    for (int e = tid; e < (rows + nrel) * nC; e += blockDim.x) {
        if (e < rows * nC) {
            int q = 0, off = e;
            while (off >= s_nG[q] * nC) off -= s_nG[q++] * nC;
            const int nG = s_nG[q], nO = s_nO[q];
            const BlkLayout BL = blk_layout(nO + nG, nG, nC);
            const double* bi = blk + s_blk[q];
            const bool pd = s_fl[q] == 0;
            const double wv = pd ? bi[BL.W + off] : 0.0;
            Wsh[e] = wv;
            Wr[e] = wv * (pd ? bi[BL.rinv + nO + off / nC] : 0.0);
        } else {
            const int g = e - rows * nC, q = g / nC, c = g % nC;
            const int nG = s_nG[q];
            Us[g] = s_fl[q] == 0 ? blk[s_blk[q] + blk_layout(s_nO[q] + nG, nG, nC).u + c] : 0.0;
        }
    }
    __syncthreads();
    double* out = P.Spart + ((size_t)b * P.nfc + f) * (ntri + nC);
    for (int e = tid; e < ntri + nC; e += blockDim.x) {
        double v = 0.0;
        if (e < ntri) {
            int c1, c2;
            tri_index(e, c1, c2);
            for (int r = 0; r < rows; ++r) v += Wr[r * nC + c1] * Wsh[r * nC + c2];
        } else {
            for (int q = 0; q < nrel; ++q) v += Us[q * nC + e - ntri];
        }
        out[e] = v;
    }
}

// Step 3 of k_kkt by the threads t < n of a thread range (barrier bar): the border of the Schur complement of
// Eq. (sqp_system) over the subdomains with H_i PD (flag s_fl[i] == 0),
//   S = sum_i E_i H_i^{-1} E_i^T = sum_i W_i^T D_G,i^{-1} W_i (lower triangle)   and   us = sum_i u_i,
// each entry summed over the subdomains in index order (rows k ascending inside one), W_i, D_G^{-1} W_i and u_i
// staged in shared memory a chunk of subdomains at a time (work: 2 ss_rows n_C + (chunk subdomains) n_C).
__device__ __forceinline__ void kkt_schur_sums(const ProbDev& P, const double* blk, const int* s_blk,
                                               const unsigned char* s_nO, const unsigned char* s_nG,
                                               const unsigned char* s_fl, double* Sm, double* us, double* work,
                                               int t, int n, int bar) {
    const int nC = P.n_C;
    for (int e = t; e < nC * nC; e += n) Sm[e] = 0.0;
    for (int c = t; c < nC; c += n) us[c] = 0.0;
    double* Wsh = work;                                  // ss_rows x nC
    double* Wr = work + (size_t)P.ss_rows * nC;          // ss_rows x nC, row k scaled by 1 / D_kk
    const int ntri = nC * (nC + 1) / 2, NE = ntri + nC;
    for (int ch = 0; ch < P.n_ss_chunks; ++ch) {
        const int i0 = P.ss_chunk[ch], i1 = P.ss_chunk[ch + 1];
        // stage W_i, D_G^{-1} W_i and u_i of the chunk: thread e takes entry e of the chunk's rows
        int tot = 0;
        for (int i = i0; i < i1; ++i) tot += s_nG[i] * nC;
        double* Us = Wr + (size_t)P.ss_rows * nC;          // (i1 - i0) x nC
        for (int e = t; e < tot + (i1 - i0) * nC; e += n) {
            if (e < tot) {
                int i = i0, off = e;
                while (off >= s_nG[i] * nC) off -= s_nG[i++] * nC;
                const int nG = s_nG[i], nO = s_nO[i];
                const BlkLayout BL = blk_layout(nO + nG, nG, nC);
                const double* bi = blk + s_blk[i];
                const bool pd = s_fl[i] == 0;
                const double wv = pd ? bi[BL.W + off] : 0.0;
                const double r = pd ? bi[BL.rinv + nO + off / nC] : 0.0;
                Wsh[e] = wv;
                Wr[e] = wv * r;
            } else {
                const int f = e - tot, i = i0 + f / nC, c = f % nC;
                const int nG = s_nG[i];
                Us[f] = s_fl[i] == 0 ? blk[s_blk[i] + blk_layout(s_nO[i] + nG, nG, nC).u + c] : 0.0;
            }
        }
        const int rows = tot / nC;
        range_sync(bar, n);
        for (int e = t; e < NE; e += n) {
            if (e < ntri) {
                int c1, c2;
                tri_index(e, c1, c2);
                double v = Sm[c1 * nC + c2];
                for (int r = 0; r < rows; ++r) v += Wr[r * nC + c1] * Wsh[r * nC + c2];
                Sm[c1 * nC + c2] = v;
            } else {
                const int c = e - ntri;
                double v = us[c];
                for (int i = 0; i < i1 - i0; ++i) v += Us[i * nC + c];
                us[c] = v;
            }
        }
        range_sync(bar, n);
    }
}

enum { DEC_STEP = 0, DEC_DONE = 1, DEC_INIT0 = 2 };

// Step 1 of k_kkt for one instance, by the threads t < n of a thread range (barrier bar): merit
// phi = ||F||_2 with F = [rho_1 .. rho_n; Atil] (Sec. 4.1) from the merits ||rho_i||^2 (the header of the block
// area, subdomain i's at index i) and the constraint partials (Atil to At), Armijo backtracking test, update and
// stopping rule (Eq. sqp_update, Sec. 7.1).  Returns, the same to every thread of the range, DEC_DONE (a
// rejected trial, whose backtrack is set up here, or a stop), DEC_INIT0 (the start-up pass: the least-squares
// multiplier follows) or DEC_STEP (an accepted point that does not stop).  The accepted point's lambda <- lamt
// is copied here, and x <- xt too when copy_x is set or the instance stops.
__device__ __forceinline__ int kkt_decide(const ProbDev& P, int b, const double* blk, double* At, double* scratch, int t, int n,
                          int bar, bool copy_x) {
    int* ist = P.ist + (size_t)b * INST_INTS;
    double* dst = P.dst + (size_t)b * INST_DBLS;
    const int nC = P.n_C, ns = P.n_sub, nD = P.n_D;
    // one round of independent loads: the instance state, the merits and the constraint partial sums
    const int mode = ist[I_MODE];
    const int iters0 = ist[I_ITERS], nbt = ist[I_NBT];
    const double alpha = dst[D_ALPHA], phi0 = dst[D_PHI0];
    double acc = 0.0, ss = 0.0, xx = 0.0;
    for (int i = t; i < ns; i += n) {
        acc += blk[i];
        ss += blk[ns + 2 * i];
        xx += blk[ns + 2 * i + 1];
    }
    for (int c = t; c < nC; c += n) {
        const double a = tree_sum(P.Atil + (size_t)b * P.n_split * nC + c, P.n_split, nC);
        At[c] = a;
        acc += a * a;
    }
    const double phi2 = range_sum(acc, scratch, t, n, bar);   // barriers inside: the range has read ist and dst
    const double phi = sqrt(phi2);
    // the step test (mixed path with step_tol > 0): the first trial of a step whose Gauss-Newton step is below
    // step_tol of the iterate is accepted and ends the solve (near the solution the FP32 evaluation's merit
    // stalls at its rounding level, where an Armijo comparison would only compare rounding noise)
    bool small = false;
    if (P.step_tol > 0.0 && mode == MODE_LS && nbt == 0) {
        const double s2 = range_sum(ss, scratch, t, n, bar), x2 = range_sum(xx, scratch, t, n, bar);
        small = s2 <= P.step_tol * P.step_tol * x2 && x2 > 0.0;
    }
    if (mode == MODE_INIT0) {
        if (t == 0) ist[I_NEVALS] += 1;
        return DEC_INIT0;
    }
    bool accept = true, lsfail = false;
    if (mode == MODE_LS && !(phi2 <= (1.0 - 2.0 * P.c1 * alpha) * phi0 * phi0) && !small) {
        if (nbt < P.max_bt) accept = false;
        else lsfail = true;
    }
    double* lam = P.lam + (size_t)b * nC;
    double* lamt = P.lamt + (size_t)b * nC;
    if (!accept) {
        const double a = alpha * P.beta;
        const double* slam = P.slam + (size_t)b * nC;
        for (int c = t; c < nC; c += n) lamt[c] = lam[c] + a * slam[c];
        if (t == 0) {
            ist[I_NEVALS] += 1;
            dst[D_ALPHA] = a;
            ist[I_NBT] = nbt + 1;
            ist[I_XTMODE] = XT_BACKTRACK;
            atomicAdd(P.active, 1);
        }
        return DEC_DONE;
    }
    for (int c = t; c < nC; c += n) lam[c] = lamt[c];
    const int iters = iters0 + (mode == MODE_LS ? 1 : 0);
    int status = ST_RUNNING;
    if (!isfinite(phi)) status = DDNM_NONFINITE;
    else if (phi < P.tol) status = DDNM_CONVERGED;
    else if (small) status = DDNM_CONVERGED;
    else if (iters >= P.max_iter) status = DDNM_MAX_ITER;
    if (copy_x || status != ST_RUNNING) {
        double* x = P.x + (size_t)b * nD;
        const double* xt = P.xt + (size_t)b * nD;
        for (int k = t; k < nD; k += n) x[k] = xt[k];
    }
    if (t == 0) {
        ist[I_NEVALS] += 1;
        ist[I_ITERS] = iters;
        dst[D_PHI0] = phi;
        dst[D_PHI] = phi;
        if (mode == MODE_LS) dst[D_ALPHA_LAST] = alpha;
        if (lsfail) ist[I_FLAGS] |= DDNM_FLAG_LS_FAIL;
        if (small && !(phi < P.tol)) ist[I_FLAGS] |= DDNM_FLAG_STEP;
        if (status != ST_RUNNING) ist[I_STATUS] = status;
    }
    return status == ST_RUNNING ? DEC_STEP : DEC_DONE;
}

// One SQP pass's work after the evaluation, the constraint residual and the factorisation of the blocks
// (both in k_constraint), one CTA per instance:
//  1. judge the evaluation: merit phi = ||F||_2 with F = [rho_1 .. rho_n; Atil] (Sec. 4.1), Armijo
//     backtracking test, update and stopping rule (Eq. sqp_update, Sec. 7.1).  A rejected trial becomes
//     the next backtrack (the evaluation forms xt = x + alpha beta s); the start-up pass solves for the
//     least-squares multiplier (Sec. 7.2);
//  3. (beside step 1) the border of the Schur complement of Eq. (sqp_system) over the subdomains with H_i PD,
//       S = sum_i E_i H_i^{-1} E_i^T = sum_i W_i^T D_G,i^{-1} W_i,   r = Atil - sum_i u_i;
//  4. S = L_S D_S L_S^T and s_lambda; the subdomains F whose H_i is singular in the G block keep their
//     interface steps s_F as unknowns: with Z = L_S^{-1} D_F, q = L_S^{-1} r and G_F their Schur
//     complements, (G_F + Z^T D_S^{-1} Z) s_F = -(rho_G - L_GO t_O)_F - Z^T D_S^{-1} q and
//     s_lambda = L_S^{-T} D_S^{-1} (q + Z s_F).  Every other piece of s is back-substituted by the
//     evaluation of its subdomain (form_trial).
__device__ __forceinline__ void kkt_body(const ProbDev& P, int B) {
    extern __shared__ __align__(16) double ksm[];
    __shared__ double scratch[32];
    __shared__ int s_mF, s_over, s_fail;
    __shared__ int fcol_sub[MAX_MF], fcol_k[MAX_MF];
    __shared__ unsigned char s_fl[MAX_SUB];
    const int b = blockIdx.x, tid = threadIdx.x, nth = blockDim.x;
    const int w = tid >> 5, lane = tid & 31, nw = nth >> 5;
    if (b >= B) return;
    int* ist = P.ist + (size_t)b * INST_INTS;
    double* dst = P.dst + (size_t)b * INST_DBLS;
    if (ist[I_STATUS] != ST_RUNNING) return;
    const int nC = P.n_C, ns = P.n_sub, nD = P.n_D;
    double* blk = P.blk + (size_t)b * P.blk_stride;
    double* Sm = ksm;                 // nC x nC (lower triangle used)
    double* rhs = Sm + nC * nC;       // nC
    double* At = rhs + nC;            // nC: Atil
    double* rv = At + nC;             // nC: reciprocal pivots
    double* us = rv + nC;             // nC: sum_i u_i
    double* work = us + nC;           // union: W staging (when summed here) | Z, T of the border solve
    double* lam = P.lam + (size_t)b * nC;
    double* lamt = P.lamt + (size_t)b * nC;
    double* slam = P.slam + (size_t)b * nC;

    // per-subdomain fields used below, in shared memory (one round of loads instead of a chain per use)
    __shared__ int s_blk[MAX_SUB];
    __shared__ unsigned char s_nO[MAX_SUB], s_nG[MAX_SUB];
    __shared__ int s_dec;

    // ---- 1 and 3: judge the trial point (the last KKT_DW warps) while the others add up the Schur sums of step 3
    // from the shares k_constraint left (sums formed beside a rejected trial or a stop are simply not used).  A
    // border too wide for the shares is summed here from the blocks, after the judgement: only at an accepted
    // point, for those sums are the bulk of the step's FP64 work.
    {
        const int nst = nth - 32 * KKT_DW;                   // threads of the Schur sums
        if (tid < nst) {
            for (int i = tid; i < ns; i += nst) {
                const SubDev& S = P.sub[i];
                const int bo = S.blk, nO = S.nO, nG = S.nG;
                s_blk[i] = bo;
                s_nO[i] = (unsigned char)nO;
                s_nG[i] = (unsigned char)nG;
                s_fl[i] = (unsigned char)blk[bo + blk_layout(nO + nG, nG, nC).flag];
            }
            if (P.Spart) {
                // S (lower triangle) and sum_i u_i: the shares of the factorisation CTAs added in CTA order
                const int ntri = nC * (nC + 1) / 2;
                const double* sp = P.Spart + (size_t)b * P.nfc * (ntri + nC);
                for (int e = tid; e < ntri + nC; e += nst) {
                    double v = 0.0;
                    for (int f = 0; f < P.nfc; ++f) v += sp[(size_t)f * (ntri + nC) + e];
                    if (e < ntri) {
                        int c1, c2;
                        tri_index(e, c1, c2);
                        Sm[c1 * nC + c2] = v;
                    } else {
                        us[e - ntri] = v;
                    }
                }
            }
        } else {
            const int dec = kkt_decide(P, b, blk, At, scratch, tid - nst, 32 * KKT_DW, 1, true);
            if (tid == nst) s_dec = dec;
        }
    }
    __syncthreads();
    const int dec = s_dec;
    if (dec == DEC_DONE) return;
    if (dec == DEC_INIT0) {
        // least-squares multiplier (Sec. 7.2): min_l sum_i ||rho_i^G + D_i^T l||^2 at lambda = 0,
        // normal equations (sum_i D_i D_i^T) l = -sum_i D_i rho_i^G
        for (int e = tid; e < nC * nC; e += nth) {
            const int c1 = e / nC, c2 = e % nC;
            double v = 0.0;
            for (int i = 0; i < ns; ++i) {
                const SubDev& S = P.sub[i];
                const double* D = blk + S.blk + blk_layout(S.ni, S.nG, nC).D;
                for (int k = 0; k < S.nG; ++k) v += D[c1 * S.nG + k] * D[c2 * S.nG + k];
            }
            Sm[e] = v;
        }
        for (int c = tid; c < nC; c += nth) {
            double v = 0.0;
            for (int i = 0; i < ns; ++i) {
                const SubDev& S = P.sub[i];
                const BlkLayout BL = blk_layout(S.ni, S.nG, nC);
                const double* D = blk + S.blk + BL.D;
                const double* rho = blk + S.blk + BL.rho;
                for (int k = 0; k < S.nG; ++k) v -= D[c * S.nG + k] * rho[S.nO + k];
            }
            rhs[c] = v;
        }
        if (!block_ldl(Sm, rv, nC)) {
            if (tid == 0) ist[I_STATUS] = DDNM_KKT_FAIL;
            return;
        }
        block_ldl_solve(Sm, rv, nC, rhs);
        for (int c = tid; c < nC; c += nth) lamt[c] = rhs[c];
        if (tid == 0) {
            ist[I_MODE] = MODE_INIT1;
            ist[I_XTMODE] = XT_KEEP;
            atomicAdd(P.active, 1);
        }
        return;
    }
    if (!P.Spart) kkt_schur_sums(P, blk, s_blk, s_nO, s_nG, s_fl, Sm, us, work, tid, nth, 0);
    if (w == 0) {                // flags: a vote first, the scan only when some block is not PD
        int bad = 0;
        for (int i = lane; i < ns; i += 32) bad |= s_fl[i];
        if (!__any_sync(0xffffffffu, bad != 0)) {
            if (lane == 0) s_mF = s_over = s_fail = 0;
        } else if (lane == 0) {
            int mF = 0, over = 0, fail = 0;
            for (int i = 0; i < ns; ++i) {
                const int fl = s_fl[i];
                if (fl == 1) fail = 1;
                if (fl == 2) {
                    const int nG = P.sub[i].nG;
                    if (mF + nG > MAX_MF) {
                        over = 1;
                        continue;
                    }
                    for (int k = 0; k < nG; ++k) {
                        fcol_sub[mF] = i;
                        fcol_k[mF] = k;
                        ++mF;
                    }
                }
            }
            s_mF = mF;
            s_over = over;
            s_fail = fail;
        }
    }
    __syncthreads();
    const int mF = s_mF;
    if (s_fail || s_over) {      // H_i^{OO} not PD somewhere, or too many singular interface blocks
        if (tid == 0) ist[I_STATUS] = DDNM_KKT_FAIL;
        return;
    }

    for (int c = tid; c < nC; c += nth) rhs[c] = At[c] - us[c];

    // ---- 4. the border system
    if (!block_ldl(Sm, rv, nC)) {
        if (tid == 0) ist[I_STATUS] = DDNM_KKT_FAIL;
        return;
    }
    double* Z = work;                     // nC x (mF + 1), row-major (last column: q)
    double* T = Z + nC * (MAX_MF + 1);    // MAX_MF x MAX_MF
    double* rT = T + MAX_MF * MAX_MF;     // MAX_MF reciprocal pivots of T
    double* sF = rT + MAX_MF;             // MAX_MF
    if (mF == 0) {
        block_ldl_solve(Sm, rv, nC, rhs);
    } else {
        const int ldz = mF + 1;
        for (int e = tid; e < nC * ldz; e += nth) {
            const int c = e / ldz, a = e % ldz;
            double v;
            if (a == mF) {
                v = rhs[c];
            } else {
                const SubDev& S = P.sub[fcol_sub[a]];
                v = blk[S.blk + blk_layout(S.ni, S.nG, nC).D + c * S.nG + fcol_k[a]];
            }
            Z[e] = v;
        }
        // [Z q] <- L_S^{-1} [D_F r]   (unit lower)
        for (int j = 0; j < nC; ++j) {
            __syncthreads();
            const int m = nC - j - 1;
            for (int e = tid; e < m * ldz; e += nth) {
                const int i = j + 1 + e / ldz, a = e % ldz;
                Z[i * ldz + a] -= Sm[i * nC + j] * Z[j * ldz + a];
            }
        }
        __syncthreads();
        // T = G_F + Z^T D_S^{-1} Z, right-hand side -(t~_G)_F - Z^T D_S^{-1} q
        for (int e = tid; e < mF * mF; e += nth) {
            const int a = e / mF, c2 = e % mF;
            double v = 0.0;
            for (int c = 0; c < nC; ++c) v += Z[c * ldz + a] * rv[c] * Z[c * ldz + c2];
            if (fcol_sub[a] == fcol_sub[c2]) {
                const SubDev& S = P.sub[fcol_sub[a]];
                v += blk[S.blk + blk_layout(S.ni, S.nG, nC).G + fcol_k[a] * S.nG + fcol_k[c2]];
            }
            T[e] = v;
        }
        for (int a = tid; a < mF; a += nth) {
            const SubDev& S = P.sub[fcol_sub[a]];
            double v = -blk[S.blk + blk_layout(S.ni, S.nG, nC).t + S.nO + fcol_k[a]];
            for (int c = 0; c < nC; ++c) v -= Z[c * ldz + a] * rv[c] * Z[c * ldz + mF];
            sF[a] = v;
        }
        if (!block_ldl(T, rT, mF)) {
            if (tid == 0) ist[I_STATUS] = DDNM_KKT_FAIL;
            return;
        }
        block_ldl_solve(T, rT, mF, sF);
        for (int c = tid; c < nC; c += nth) {
            double v = Z[c * ldz + mF];
            for (int a = 0; a < mF; ++a) v += Z[c * ldz + a] * sF[a];
            rhs[c] = v * rv[c];
        }
        // rhs <- L_S^{-T} rhs  (unit upper)
        for (int k = nC - 1; k >= 0; --k) {
            __syncthreads();
            const double xk = rhs[k];
            for (int i = tid; i < k; i += nth) rhs[i] -= Sm[k * nC + i] * xk;
        }
        __syncthreads();
        double* s_ = P.s + (size_t)b * nD;
        for (int a = tid; a < mF; a += nth) {
            const SubDev& S = P.sub[fcol_sub[a]];
            s_[S.xoff + S.nO + fcol_k[a]] = sF[a];
        }
        __syncthreads();
    }
    for (int c = tid; c < nC; c += nth) {
        slam[c] = rhs[c];
        lamt[c] = lam[c] + rhs[c];
    }
    if (tid == 0) {
        dst[D_ALPHA] = 1.0;
        ist[I_NBT] = 0;
        ist[I_MODE] = MODE_LS;
        ist[I_XTMODE] = XT_NEWSTEP;
        atomicAdd(P.active, 1);
    }
}

// The step kernel: kkt_body for every instance, then, inside the solve graph (loop > 0), the loop control of
// the instance group by the CTA that finishes last: count the pass, clear the running count, the arrival
// count and the persistent evaluation's work counters, and (loop = 2, the last pass of the loop body) end
// the group's device-side while loop when no instance is running or the pass bound is reached.  (Every
// return of kkt_body is taken by a whole CTA.)
__global__ void __maxnreg__(64) k_kkt(ProbDev P, int B, int loop, int p0, int max_passes,
                                      cudaGraphConditionalHandle h) {
    kkt_body(P, B);
    if (!loop) return;
    __shared__ int s_last;
    __threadfence();                       // this CTA's running-count update before its arrival
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(P.arrive, 1) == (int)gridDim.x - 1;
    __syncthreads();
    if (!s_last || threadIdx.x != 0) return;
    __threadfence();
    const int a = atomicAdd(P.active, 0);
    const int p = *P.pass + 1;
    *P.pass = p;
    *P.active = 0;
    *P.arrive = 0;
    for (int k = 0; k < MAX_CLASSES; ++k) P.ctr[k] = 0;
    if (loop == 2 && (a == 0 || p0 + p >= max_passes)) cudaGraphSetConditional(h, 0);
}

// ------------------------------------------------------------------------ set-up / outputs

// start state of every instance and its Dirichlet data
__global__ void k_init(ProbDev P, int B, int has_x0, int has_lam0, int mode, int fp64) {
    const int b = blockIdx.x, tid = threadIdx.x, nth = blockDim.x;
    if (b >= B) return;
    for (int k = tid; k < P.n_D; k += nth) {
        const double v = has_x0 ? P.x[(size_t)b * P.n_D + k] : 0.0;
        P.x[(size_t)b * P.n_D + k] = v;
        P.xt[(size_t)b * P.n_D + k] = v;
        P.s[(size_t)b * P.n_D + k] = 0.0;
    }
    for (int c = tid; c < P.n_C; c += nth) {
        const double v = has_lam0 ? P.lam[(size_t)b * P.n_C + c] : 0.0;
        P.lam[(size_t)b * P.n_C + c] = v;
        P.lamt[(size_t)b * P.n_C + c] = v;
        P.slam[(size_t)b * P.n_C + c] = 0.0;
    }
    const double a = P.mu[2 * b], lm = P.mu[2 * b + 1];
    for (int p = tid; p < P.n_bnd; p += nth) {
        const double x = P.bx0 + P.bnd_ij[2 * p] * P.hx, y = P.by0 + P.bnd_ij[2 * p + 1] * P.hy;
        double u, v;
        exact_uv(x, y, a, lm, P.nu, u, v);
        const size_t o = ((size_t)b * P.n_bnd + p) * 2;
        if (fp64) {
            ((double*)P.bnd)[o] = u;
            ((double*)P.bnd)[o + 1] = v;
        } else {
            ((float*)P.bnd)[o] = (float)u;
            ((float*)P.bnd)[o + 1] = (float)v;
        }
    }
    if (tid == 0) {
        int* ist = P.ist + (size_t)b * INST_INTS;
        ist[I_STATUS] = ST_RUNNING;
        ist[I_MODE] = mode;
        ist[I_ITERS] = 0;
        ist[I_NBT] = 0;
        ist[I_FLAGS] = 0;
        ist[I_NEVALS] = 0;
        ist[I_XTMODE] = XT_KEEP;
        double* dst = P.dst + (size_t)b * INST_DBLS;
        dst[D_PHI0] = 0.0;
        dst[D_ALPHA] = 1.0;
        dst[D_PHI] = 0.0;
        dst[D_ALPHA_LAST] = 0.0;
    }
}

__global__ void k_stats(ProbDev P, int B, ddnm_stats* out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const int* ist = P.ist + (size_t)b * INST_INTS;
    const double* dst = P.dst + (size_t)b * INST_DBLS;
    ddnm_stats s;
    s.iters = ist[I_ITERS];
    s.status = ist[I_STATUS];
    s.flags = ist[I_FLAGS];
    s.n_evals = ist[I_NEVALS];
    s.merit = dst[D_PHI];
    s.alpha_last = dst[D_ALPHA_LAST];
    out[b] = s;
}

// F = [rho_0; ...; rho_{n-1}; Atil] of the last evaluation, plus the blocks for ddnm_linearize
__global__ void k_gather(ProbDev P, int B, double* F, double* H, double* D, double* At) {
    const int b = blockIdx.x, tid = threadIdx.x, nth = blockDim.x;
    if (b >= B) return;
    const int nC = P.n_C;
    const double* blk = P.blk + (size_t)b * P.blk_stride;
    int hoff = 0, doff = 0, hsum = 0, dsum = 0;
    for (int i = 0; i < P.n_sub; ++i) {
        hsum += P.sub[i].ni * P.sub[i].ni;
        dsum += nC * P.sub[i].nG;
    }
    for (int i = 0; i < P.n_sub; ++i) {
        const SubDev& S = P.sub[i];
        const BlkLayout BL = blk_layout(S.ni, S.nG, nC);
        if (F)
            for (int k = tid; k < S.ni; k += nth) F[(size_t)b * (P.n_D + nC) + S.xoff + k] = blk[S.blk + BL.rho + k];
        if (H)
            for (int e = tid; e < S.ni * S.ni; e += nth) H[(size_t)b * hsum + hoff + e] = blk[S.blk + BL.H + e];
        if (D)
            for (int e = tid; e < nC * S.nG; e += nth) D[(size_t)b * dsum + doff + e] = blk[S.blk + BL.D + e];
        hoff += S.ni * S.ni;
        doff += nC * S.nG;
    }
    for (int c = tid; c < nC; c += nth) {
        const double a = tree_sum(P.Atil + (size_t)b * P.n_split * nC + c, P.n_split, nC);
        if (F) F[(size_t)b * (P.n_D + nC) + P.n_D + c] = a;
        if (At) At[(size_t)b * nC + c] = a;
    }
}

// full decoders (all outputs) for the reconstructed state; each variable from its owner
template <typename T>
__global__ void k_reconstruct(ProbDev P, int B, const double* xh, double* state) {
    extern __shared__ __align__(16) unsigned char smem[];
    T* hid = (T*)smem;
    const int b = blockIdx.x / P.n_sub, si = blockIdx.x % P.n_sub;
    if (b >= B) return;
    const SubDev& S = P.sub[si];
    const T* V = (const T*)P.vpool;
    const int* IP = P.ipool;
    const int tid = threadIdx.x, nth = blockDim.x;
    for (int pass = 0; pass < 2; ++pass) {
        const bool g = pass == 1;
        const int n = g ? S.nG : S.nO, w = g ? S.wG_full : S.wO_full, N = g ? S.NG : S.NO_full;
        const double* x = xh + (size_t)b * P.n_D + S.xoff + (g ? S.nO : 0);
        const T* W1 = V + (g ? S.fw1G : S.fw1O);
        const T* b1 = V + (g ? S.fb1G : S.fb1O);
        __syncthreads();
        for (int c = tid; c < w; c += nth) {
            T z = b1[c];
            for (int k = 0; k < n; ++k) z += W1[(size_t)c * n + k] * (T)x[k];
            T s, ds;
            activation<T>(g ? S.actG : S.actO, z, s, ds);
            hid[c] = s;
        }
        __syncthreads();
        const int* cols = IP + (g ? S.fcolG : S.fcolO);
        const T* vals = V + (g ? S.fw2G : S.fw2O);
        const T* so = V + (g ? S.foutG : S.foutO);
        const int* own = IP + S.own + (g ? S.NO_full : 0);
        const int* ids = IP + S.ids + (g ? S.NO_full : 0);
        for (int r = tid; r < N; r += nth) {
            if (!own[r]) continue;
            T y = T(0);
            for (int t = 0; t < S.K; ++t) {
                const int c = cols[(size_t)r * S.K + t];
                if (c < 0) break;
                y += vals[(size_t)r * S.K + t] * hid[c];
            }
            state[(size_t)b * P.N_x + ids[r]] = (double)(so[N + r] + so[r] * y);
        }
    }
}

// FOM residual r(x; mu) of Eq. (burgers_discretized) at every node, Dirichlet data from mu
__global__ void k_fom_residual(ProbDev P, int B, const double* state, double* res) {
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int N = P.nx * P.ny;
    if (gid >= (long long)B * N) return;
    const int b = (int)(gid / N), p = (int)(gid % N);
    const int i = p % P.nx, j = p / P.nx;
    const double* u = state + (size_t)b * P.N_x;
    const double* v = u + N;
    const double a = P.mu[2 * b], lm = P.mu[2 * b + 1];
    double U[5], Vv[5];   // centre, E, W, N, S
    const int I[5] = {i, i + 1, i - 1, i, i}, J[5] = {j, j, j, j + 1, j - 1};
    for (int o = 0; o < 5; ++o) {
        if (I[o] >= 0 && I[o] < P.nx && J[o] >= 0 && J[o] < P.ny) {
            U[o] = u[J[o] * P.nx + I[o]];
            Vv[o] = v[J[o] * P.nx + I[o]];
        } else {
            exact_uv(P.bx0 + (I[o] + 1) * P.hx, P.by0 + (J[o] + 1) * P.hy, a, lm, P.nu, U[o], Vv[o]);
        }
    }
    const double ax = 0.5 / P.hx, ay = 0.5 / P.hy, cx = P.nu / (P.hx * P.hx), cy = P.nu / (P.hy * P.hy);
    const double ru = -U[0] * (U[1] - U[2]) * ax - Vv[0] * (U[3] - U[4]) * ay + cx * (U[1] - 2 * U[0] + U[2]) +
                      cy * (U[3] - 2 * U[0] + U[4]);
    const double rv = -U[0] * (Vv[1] - Vv[2]) * ax - Vv[0] * (Vv[3] - Vv[4]) * ay + cx * (Vv[1] - 2 * Vv[0] + Vv[2]) +
                      cy * (Vv[3] - 2 * Vv[0] + Vv[4]);
    res[(size_t)b * P.N_x + p] = ru;
    res[(size_t)b * P.N_x + N + p] = rv;
}

// Warm-start screening: instance b started from the learned prediction, instance B + b from the default
// start xh0 = 0.  After both start-up passes the one with the smaller merit (a finite one; the default
// start wins ties and failures of the prediction) continues in slot b.  Both screenings count as evaluations.
__global__ void k_ws_select(ProbDev P, int B) {
    const int b = blockIdx.x, tid = threadIdx.x, nth = blockDim.x;
    if (b >= B) return;
    int* iw = P.ist + (size_t)b * INST_INTS;
    int* iz = P.ist + (size_t)(B + b) * INST_INTS;
    double* dw = P.dst + (size_t)b * INST_DBLS;
    double* dz = P.dst + (size_t)(B + b) * INST_DBLS;
    auto valid = [](const int* is, const double* ds) {
        return (is[I_STATUS] == ST_RUNNING || is[I_STATUS] == DDNM_CONVERGED) && isfinite(ds[D_PHI0]);
    };
    const bool vw = valid(iw, dw), vz = valid(iz, dz);
    const bool use_zero = !vw || (vz && !(dw[D_PHI0] < dz[D_PHI0]));
    const int evals = iw[I_NEVALS] + iz[I_NEVALS];
    __syncthreads();
    if (use_zero) {
        const size_t nD = P.n_D, nC = P.n_C;
        for (size_t k = tid; k < nD; k += nth) {
            P.x[b * nD + k] = P.x[(B + b) * nD + k];
            P.xt[b * nD + k] = P.xt[(B + b) * nD + k];
            P.s[b * nD + k] = P.s[(B + b) * nD + k];
        }
        for (size_t c = tid; c < nC; c += nth) {
            P.lam[b * nC + c] = P.lam[(B + b) * nC + c];
            P.lamt[b * nC + c] = P.lamt[(B + b) * nC + c];
            P.slam[b * nC + c] = P.slam[(B + b) * nC + c];
        }
        const double* bz = P.blk + (size_t)(B + b) * P.blk_stride;
        double* bw = P.blk + (size_t)b * P.blk_stride;
        for (int k = tid; k < P.blk_stride; k += nth) bw[k] = bz[k];
        if (tid < INST_DBLS) dw[tid] = dz[tid];
        if (tid < INST_INTS) iw[tid] = iz[tid];
    }
    __syncthreads();
    if (tid == 0) {
        iw[I_NEVALS] = evals;
        if (use_zero) iw[I_FLAGS] |= DDNM_FLAG_WS_FALLBACK;
    }
}

// ------------------------------------------------------------------------ host drivers

struct Launch {
    ddnm_ctx* ctx;
    cudaStream_t st;
};

int cfail(ddnm_ctx* ctx, cudaError_t e, const char* what) {
    return ddnm_fail(ctx, DDNM_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cfail(ctx, e_, #call);       \
    } while (0)

// per-kernel timing: a pair of events around a launch when timing is on
int tstart(ddnm_ctx* ctx, int kind, cudaStream_t st) {
    if (!ctx->timing) return -1;
    const size_t k = ctx->n_events;
    while (ctx->events.size() < 2 * (k + 1)) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return -1;
        ctx->events.push_back(e);
    }
    if (ctx->event_kind.size() < k + 1) ctx->event_kind.resize(k + 1);
    ctx->event_kind[k] = kind;
    cudaEventRecord(ctx->events[2 * k], st);
    ctx->n_events = k + 1;
    return (int)k;
}

void tstop(ddnm_ctx* ctx, int k, cudaStream_t st) {
    if (k >= 0) cudaEventRecord(ctx->events[2 * k + 1], st);
}

int tflush(ddnm_ctx* ctx, cudaStream_t st) {
    if (!ctx->timing || ctx->n_events == 0) return DDNM_OK;
    CK(cudaStreamSynchronize(st));
    for (size_t k = 0; k < ctx->n_events; ++k) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, ctx->events[2 * k], ctx->events[2 * k + 1]));
        if (ctx->event_kind[k] == 0) ctx->tm.eval_ms += ms;
        else if (ctx->event_kind[k] == 1) ctx->tm.constraint_ms += ms;
        else ctx->tm.step_ms += ms;
    }
    ctx->n_events = 0;
    return DDNM_OK;
}

template <typename T>
int set_smem_attrs(ddnm_ctx* ctx) {
    for (const auto& g : ctx->eval_classes)
        CK(cudaFuncSetAttribute(eval_kernel<T>(g.ro, g.rg), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                std::max(g.smem, g.groups * g.stride)));
    CK(cudaFuncSetAttribute(k_kkt, cudaFuncAttributeMaxDynamicSharedMemorySize, ctx->kkt_smem));
    CK(cudaFuncSetAttribute(k_constraint<T, NG_SMALL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            std::max(MAX_CON_SPLIT * 8, ctx->fac_smem)));
    CK(cudaFuncSetAttribute(k_constraint<T, MAX_NG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            std::max(MAX_CON_SPLIT * 8, ctx->fac_smem)));
    {
        constexpr int CPT = sizeof(T) == 8 ? 16 : 32;
        const int ncp = (ctx->n_C + 31) & ~31;
        const int tb_max = std::max(1, (DG_THREADS / ncp) * CPT / ctx->max_nG);
        const int smem = dg_smem_main<T, CPT>(ncp) + tb_max * ctx->n_C * 8;
        CK(cudaFuncSetAttribute(k_dgemm<T, CPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    }
    CK(cudaFuncSetAttribute(k_reconstruct<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, std::max(ctx->rec_smem, 16)));
    return DDNM_OK;
}

// the batched D_i GEMM of one pass (after the evaluation launches): instance tiles of about
// B n_sub / (2 SMs) instances, at most as many as the CTA's columns hold
template <typename T>
cudaError_t launch_dgemm(ddnm_ctx* ctx, const ProbDev& P, int B, cudaStream_t st) {
    constexpr int CPT = sizeof(T) == 8 ? 16 : 32;
    const int ncp = (P.n_C + 31) & ~31, ncol = (DG_THREADS / ncp) * CPT;
    const int tb_max = std::max(1, ncol / ctx->max_nG);
    const int n_sm = ctx->n_sm > 0 ? ctx->n_sm : 148;
    const long long want = ((long long)B * P.n_sub + 2LL * n_sm - 1) / (2LL * n_sm);
    const int TB = (int)std::max(1LL, std::min<long long>(want, tb_max));
    const size_t smem = (size_t)dg_smem_main<T, CPT>(ncp) + (size_t)TB * P.n_C * 8;
    k_dgemm<T, CPT><<<dim3(P.n_sub, (B + TB - 1) / TB), DG_THREADS, smem, st>>>(P, B, TB);
    return cudaGetLastError();
}

// One pass's evaluation (one launch per width class, then the batched D_i GEMM) and constraint launches for
// the B instances of P.
// persist: the evaluation launches are persistent; zero_ctr: clear their work counters first (the loop
// kernel of the solve graph clears them otherwise).
template <typename T>
int launch_eval(ddnm_ctx* ctx, const ProbDev& P, int B, cudaStream_t st, bool persist = false, bool zero_ctr = true,
                bool factor = false) {
    int k = tstart(ctx, 0, st);
    if (persist && zero_ctr) CK(cudaMemsetAsync(P.ctr, 0, MAX_CLASSES * sizeof(int), st));
    for (size_t ci = 0; ci < ctx->eval_classes.size(); ++ci) {
        const EvalClass& g = ctx->eval_classes[ci];
        const int G = ctx->tune.eval_groups == 1 ? 1 : g.groups;
        const int items = B * g.n;
        int grid = (items + G - 1) / G;
        int* ctr = nullptr;
        if (persist) {
            grid = std::min(grid, std::max(1, ctx->n_sm * ctx->tune.eval_persist / G));
            ctr = P.ctr + ci;
        }
        eval_kernel<T>(g.ro, g.rg)<<<grid, g.nt * G, G == 1 ? g.smem : G * g.stride, st>>>(
            P, B, ctx->d_classes + g.off, g.n, ctr, g.stride);
        CK(cudaGetLastError());
        ctx->tm.eval_launches++;
    }
    if (P.d_gemm == 2) {
        if constexpr (sizeof(T) == 4) CK(ddnm_launch_dgemm_tc(ctx, P, B, st));
        ctx->tm.eval_launches++;
    } else if (P.d_gemm) {
        CK(launch_dgemm<T>(ctx, P, B, st));
        ctx->tm.eval_launches++;
    }
    tstop(ctx, k, st);
    k = tstart(ctx, 1, st);
    {
        // with the factorisation CTAs of the step (8 subdomains each) when the pass goes on to a KKT step; the
        // double-float Atil (mixed path) in a launch of its own, the constraint launch then only factorises
        const int nfc = factor ? (P.n_sub + 2 * FAC_WARPS - 1) / (2 * FAC_WARPS) : 0;
        const int nrg = P.atil_df ? 0 : con_row_groups(ctx, P, B);
        if constexpr (sizeof(T) == 4) {
            if (P.atil_df) CK(launch_atil(ctx, P, B, st));
        }
        const size_t smem = std::max((size_t)P.con_split * 8, nfc ? (size_t)ctx->fac_smem : 0);
        if (smem > (size_t)std::max(MAX_CON_SPLIT * 8, ctx->fac_smem))     // beyond what set_smem_attrs allowed
            return ddnm_fail(ctx, DDNM_E_UNSUPPORTED, "constraint launch: shared memory above its limit");
        if (P.n_split * nrg + nfc > 0) {
            // the factorisation's register arrays sized for the largest n_i^G
            auto kern = ctx->max_nG <= NG_SMALL ? k_constraint<T, NG_SMALL> : k_constraint<T, MAX_NG>;
            kern<<<dim3(P.n_split * nrg + nfc, B), CON_THREADS, smem, st>>>(P, B, nrg);
        }
    }
    CK(cudaGetLastError());
    tstop(ctx, k, st);
    ctx->tm.constraint_launches++;
    return DDNM_OK;
}

// The device-side loop control of an instance group's pass inside the solve graph (k_kkt's last CTA):
// on = 1 counts the pass and clears the counters, on = 2 (the last pass of the loop body) also decides
// whether the loop goes on.
struct LoopCtl {
    int on = 0;
    int p0 = 0, max_passes = 0;
    cudaGraphConditionalHandle h = 0;
};

// One SQP pass (evaluation, constraint residual, KKT step) of the B instances of P.  host_style: clear the
// running count before the step (the step's loop control in the solve graph does it otherwise).
template <typename T>
int run_pass(ddnm_ctx* ctx, const ProbDev& P, int B, cudaStream_t st, bool persist, bool host_style,
             const LoopCtl& lc = LoopCtl{}) {
    int rc = launch_eval<T>(ctx, P, B, st, persist, host_style, true);
    if (rc) return rc;
    if (host_style) CK(cudaMemsetAsync(P.active, 0, sizeof(int), st));
    const int k = tstart(ctx, 2, st);
    k_kkt<<<B, KKT_THREADS, ctx->kkt_smem, st>>>(P, B, lc.on, lc.p0, lc.max_passes, lc.h);
    CK(cudaGetLastError());
    tstop(ctx, k, st);
    ctx->tm.step_launches++;
    return DDNM_OK;
}

// The instances [b0, b0 + n) of P as a batch of their own, with instance group c's control counters.
ProbDev group_view(const ProbDev& P, int b0, int c, size_t tsize) {
    ProbDev Q = P;
    const size_t b = (size_t)b0, nD = P.n_D, nC = P.n_C;
    Q.mu += 2 * b;
    Q.x += b * nD;
    Q.lam += b * nC;
    Q.xt += b * nD;
    Q.lamt += b * nC;
    Q.s += b * nD;
    Q.slam += b * nC;
    Q.Atil += b * P.n_split * nC;
    if (Q.Spart) Q.Spart += b * P.nfc * (nC * (nC + 1) / 2 + nC);
    Q.dst += b * INST_DBLS;
    Q.ist += b * INST_INTS;
    Q.bnd = (char*)P.bnd + b * P.n_bnd * 2 * tsize;
    Q.gG = (char*)P.gG + b * P.sum_NG * tsize;
    Q.PG = (char*)P.PG + b * P.pg_stride * tsize;
    Q.blk += b * P.blk_stride;
    if (Q.r_hr) Q.r_hr += b * P.sum_NB;
    Q.active = P.active + c;
    Q.pass = P.pass + c;
    Q.ctr = P.ctr + (size_t)c * MAX_CLASSES;
    Q.arrive = P.arrive + c;
    return Q;
}

// copy n doubles from the caller (host or device memory) into device memory
int copy_in(ddnm_ctx* ctx, double* dst, const double* src, size_t n, int mem_kind, cudaStream_t st) {
    if (!n) return DDNM_OK;
    CK(cudaMemcpyAsync(dst, src, n * 8, mem_kind == DDNM_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
    return DDNM_OK;
}

int copy_out(ddnm_ctx* ctx, void* dst, const void* src, size_t bytes, int mem_kind, cudaStream_t st) {
    if (!bytes) return DDNM_OK;
    CK(cudaMemcpyAsync(dst, src, bytes, mem_kind == DDNM_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
    return DDNM_OK;
}

int prepare(ddnm_ctx* ctx, int B, int mem_kind) {
    if (!ctx) return DDNM_E_INVALID;
    if (B < 1) return ddnm_fail(ctx, DDNM_E_INVALID, "B must be >= 1");
    if (mem_kind != DDNM_MEM_HOST && mem_kind != DDNM_MEM_DEVICE) return ddnm_fail(ctx, DDNM_E_INVALID, "bad mem_kind");
    int rc = ddnm_finalize(ctx);   // checks the call order first, then touches the device
    if (rc) return rc;
    CK(cudaSetDevice(ctx->device));
    rc = ddnm_reserve(ctx, B);
    if (rc) return rc;
    if (!ctx->n_sm) CK(cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, ctx->device));
    rc = ctx->precision == DDNM_FP64 ? set_smem_attrs<double>(ctx) : set_smem_attrs<float>(ctx);
    return rc;
}

template <typename T>
int reconstruct(ddnm_ctx* ctx, const ProbDev& P, int B, const double* xh_dev, double* state_dev, cudaStream_t st) {
    CK(cudaMemsetAsync(state_dev, 0, (size_t)B * P.N_x * 8, st));
    k_reconstruct<T><<<B * P.n_sub, 256, std::max(ctx->rec_smem, 16), st>>>(P, B, xh_dev, state_dev);
    CK(cudaGetLastError());
    ctx->tm.other_launches++;
    return DDNM_OK;
}

// Temporary device buffer for outputs whose caller pointer is host memory.
struct Tmp {
    void* p = nullptr;
    ~Tmp() { cudaFree(p); }
};

// ------------------------------------------------------------------ solve graph (launch plan)

// Launch counts of the last graph solve: the loop passes per instance group are read back with the
// results and folded into the counters when next needed.
void fold_pending(ddnm_ctx* ctx) {
    if (!ctx->pass_pending) return;
    ctx->pass_pending = false;
    if (cudaEventSynchronize(ctx->pass_ev) != cudaSuccess) return;
    long long passes = 0;
    for (int c = 0; c < ctx->pending_chains; ++c) passes += ctx->h_pass[c];
    ctx->tm.eval_launches += passes * ctx->pending_classes;   // with the D_i GEMM when it is used
    ctx->tm.constraint_launches += passes;
    ctx->tm.step_launches += passes;           // k_kkt
}

// the D_i form: 0 in the evaluation, 1 the batched FP32 GEMM, 2 the tensor-core GEMM (mixed path only; the
// FP64 path and sizes it does not take fall back to 1)
int resolved_dgemm(const ddnm_ctx* ctx) {
    if (ctx->srpc) return 0;                    // SRPC: D_i is the constant A^_i
    int d = ctx->tune.d_gemm;
    if (d < 0) d = ctx->dgemm_auto && ddnm_dgemm_tc_ok(ctx) ? 2 : ctx->dgemm_auto;
    return d == 2 && !ddnm_dgemm_tc_ok(ctx) ? 1 : d;
}

// the Atil form of the plan (double-float instance tiles only in the mixed path, with the split C uploaded);
// sets the slices of the constraint rows that the Atil partials cover
void resolve_atil(const ddnm_ctx* ctx, ProbDev& P) {
    const int want = ctx->tune.atil < 0 ? ctx->atil_auto : ctx->tune.atil;
    P.atil_df = (ctx->precision == DDNM_MIXED && want == 1 && P.Cthi && !ctx->srpc) ? 1 : 0;
    if (P.atil_df) {
        P.con_split = ATIL_KS;
        P.n_split = (P.N_A + ATIL_KS - 1) / ATIL_KS;
    }
}

void drop_graph(ddnm_ctx* ctx) {
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    if (ctx->graph) cudaGraphDestroy(ctx->graph);
    ctx->gexec = nullptr;
    ctx->graph = nullptr;
    ctx->gkey.clear();
}

int n_groups(const ddnm_ctx* ctx, int B) { return std::max(1, std::min(ctx->tune.chains, B)); }

// Capture the solve of B instances (Bw with the warm-start shadow copies) as one graph:
//   clear the control area -> k_init -> [warm start: two screening passes over Bw, k_ws_select]
//   -> per instance group, a conditional while node whose body is PASSES_PER_BODY passes (each KKT step ends
//      its pass with the loop control; the last one decides whether the loop goes on).  A body's later
//      passes after the group has finished launch kernels that find no running instance and return: one
//      loop turn (the conditional node's relaunch) per PASSES_PER_BODY passes instead of per pass.
template <typename T>
int build_graph(ddnm_ctx* ctx, const ProbDev& P, int B, int Bw, bool ws, bool has_x0, bool has_lam0,
                int max_passes) {
    drop_graph(ctx);
    if (!ctx->cap_main) CK(cudaStreamCreateWithFlags(&ctx->cap_main, cudaStreamNonBlocking));
    if (!ctx->cap_body) CK(cudaStreamCreateWithFlags(&ctx->cap_body, cudaStreamNonBlocking));
    const ddnm_timing tm_saved = ctx->tm;      // capturing is not launching
    const bool persist = ctx->tune.eval_persist > 0;
    const size_t tsize = sizeof(T);
    cudaGraph_t G = nullptr;
    CK(cudaGraphCreate(&G, 0));
    cudaStream_t cs = ctx->cap_main, cb = ctx->cap_body;
    auto abort_capture = [&](int rc) {
        cudaStreamCaptureStatus status;
        cudaGraph_t t = nullptr;
        if (cudaStreamIsCapturing(cb, &status) == cudaSuccess && status != cudaStreamCaptureStatusNone)
            cudaStreamEndCapture(cb, &t);
        t = nullptr;
        if (cudaStreamIsCapturing(cs, &status) == cudaSuccess && status != cudaStreamCaptureStatusNone)
            cudaStreamEndCapture(cs, &t);
        cudaGraphDestroy(G);
        cudaGetLastError();
        ctx->tm = tm_saved;
        return rc;
    };
    cudaError_t e = cudaStreamBeginCaptureToGraph(cs, G, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return abort_capture(cfail(ctx, e, "cudaStreamBeginCaptureToGraph"));
    e = cudaMemsetAsync(P.active, 0, CTL_INTS * sizeof(int), cs);
    if (e != cudaSuccess) return abort_capture(cfail(ctx, e, "capture: clear control area"));
    k_init<<<Bw, 128, 0, cs>>>(P, Bw, has_x0 || ws, has_lam0, has_lam0 ? MODE_INIT1 : MODE_INIT0, (int)(tsize == 8));
    int p0 = 0;
    if (ws) {
        for (int pass = 0; pass < 2; ++pass) {
            const int rc = run_pass<T>(ctx, P, Bw, cs, persist, true);
            if (rc) return abort_capture(rc);
        }
        k_ws_select<<<B, 128, 0, cs>>>(P, B);
        e = cudaMemsetAsync(P.active, 0, CTL_INTS * sizeof(int), cs);
        if (e != cudaSuccess) return abort_capture(cfail(ctx, e, "capture: clear control area"));
        p0 = 2;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return abort_capture(cfail(ctx, e, "capture: start-up launches"));
    cudaStreamCaptureStatus status;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    e = cudaStreamGetCaptureInfo(cs, &status, nullptr, nullptr, &deps, nullptr, &ndeps);
    if (e != cudaSuccess) return abort_capture(cfail(ctx, e, "cudaStreamGetCaptureInfo"));
    const std::vector<cudaGraphNode_t> start(deps, deps + ndeps);
    const int K = n_groups(ctx, B);
    std::vector<cudaGraphNode_t> loops;
    for (int c = 0; c < K; ++c) {
        const int b0 = (int)((long long)B * c / K), b1 = (int)((long long)B * (c + 1) / K);
        const ProbDev Q = group_view(P, b0, c, tsize);
        cudaGraphConditionalHandle h;
        e = cudaGraphConditionalHandleCreate(&h, G, 1, cudaGraphCondAssignDefault);
        if (e != cudaSuccess) return abort_capture(cfail(ctx, e, "cudaGraphConditionalHandleCreate"));
        cudaGraphNodeParams np{};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        e = cudaGraphAddNode(&node, G, start.data(), nullptr, start.size(), &np);
        if (e != cudaSuccess) return abort_capture(cfail(ctx, e, "cudaGraphAddNode(while)"));
        loops.push_back(node);
        e = cudaStreamBeginCaptureToGraph(cb, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                          cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) return abort_capture(cfail(ctx, e, "cudaStreamBeginCaptureToGraph(body)"));
        for (int u = 0; u < PASSES_PER_BODY; ++u) {
            LoopCtl lc;
            lc.on = u + 1 < PASSES_PER_BODY ? 1 : 2;
            lc.p0 = p0;
            lc.max_passes = max_passes;
            lc.h = h;
            const int rc = run_pass<T>(ctx, Q, b1 - b0, cb, persist, false, lc);
            if (rc) return abort_capture(rc);
        }
        cudaGraph_t body = nullptr;
        e = cudaStreamEndCapture(cb, &body);
        if (e != cudaSuccess) return abort_capture(cfail(ctx, e, "cudaStreamEndCapture(body)"));
    }
    e = cudaStreamUpdateCaptureDependencies(cs, loops.data(), nullptr, loops.size(), cudaStreamSetCaptureDependencies);
    if (e != cudaSuccess) return abort_capture(cfail(ctx, e, "cudaStreamUpdateCaptureDependencies"));
    cudaGraph_t done = nullptr;
    e = cudaStreamEndCapture(cs, &done);
    if (e != cudaSuccess) return abort_capture(cfail(ctx, e, "cudaStreamEndCapture"));
    ctx->tm = tm_saved;
    e = cudaGraphInstantiate(&ctx->gexec, G, 0);
    if (e != cudaSuccess) {
        ctx->gexec = nullptr;
        cudaGraphDestroy(G);
        return cfail(ctx, e, "cudaGraphInstantiate");
    }
    ctx->graph = G;
    return DDNM_OK;
}

template <typename T>
int solve_graph(ddnm_ctx* ctx, const ProbDev& P, int B, int Bw, bool ws, bool has_x0, bool has_lam0, int max_passes,
                cudaStream_t st) {
    fold_pending(ctx);
    auto bits = [](double v) {
        long long b;
        std::memcpy(&b, &v, 8);
        return b;
    };
    const ddnm_options& o = ctx->opt;
    const std::vector<long long> key{ctx->gen, B, Bw, ws, has_x0, has_lam0, (long long)sizeof(T), max_passes,
                                     bits(o.tol), bits(o.armijo_c1), bits(o.beta), o.max_iter, o.max_backtracks, bits(P.step_tol),
                                     ctx->tune.chains, ctx->tune.con_split, ctx->tune.eval_persist, ctx->n_sm,
                                     P.d_gemm, ctx->tune.eval_groups, P.atil_df};
    if (!ctx->gexec || key != ctx->gkey) {
        const int rc = build_graph<T>(ctx, P, B, Bw, ws, has_x0, has_lam0, max_passes);
        if (rc) return rc;
        ctx->gkey = key;
    }
    if (!ctx->h_pass) CK(cudaMallocHost(&ctx->h_pass, MAX_CHAINS * sizeof(int)));
    if (!ctx->pass_ev) CK(cudaEventCreateWithFlags(&ctx->pass_ev, cudaEventDisableTiming));
    CK(cudaGraphLaunch(ctx->gexec, st));
    const int cls = (int)ctx->eval_classes.size() + (P.d_gemm ? 1 : 0);
    ctx->tm.other_launches += 1 + (ws ? 1 : 0);                // k_init, k_ws_select
    if (ws) {
        ctx->tm.eval_launches += 2 * cls;
        ctx->tm.constraint_launches += 2;
        ctx->tm.step_launches += 2;
    }
    CK(cudaMemcpyAsync(ctx->h_pass, P.pass, MAX_CHAINS * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaEventRecord(ctx->pass_ev, st));
    ctx->pass_pending = true;
    ctx->pending_chains = n_groups(ctx, B);
    ctx->pending_classes = cls;
    return DDNM_OK;
}

}  // namespace

extern "C" int ddnm_solve_batch(ddnm_ctx* ctx, int B, const double* mu, const double* x0, const double* lam0,
                                double* x_out, double* lam_out, double* state_out, ddnm_stats* stats, int mem_kind,
                                void* stream) {
    // learned warm start: instances [0, B) start from the MLP prediction, a shadow copy [B, 2B) from the
    // default start; after the two start-up passes each instance keeps the start with the smaller merit
    const bool ws = ctx && ctx->ws.enabled && !x0 && !lam0;
    const int Bw = ws ? 2 * B : B;
    int rc = prepare(ctx, Bw, mem_kind);
    if (rc) return rc;
    if (!mu) return ddnm_fail(ctx, DDNM_E_INVALID, "mu is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    ProbDev P = ctx->pd;
    P.r_hr = nullptr;
    const bool fp64 = ctx->precision == DDNM_FP64;
    if ((rc = copy_in(ctx, P.mu, mu, (size_t)B * 2, mem_kind, st))) return rc;
    if (x0 && (rc = copy_in(ctx, P.x, x0, (size_t)B * P.n_D, mem_kind, st))) return rc;
    if (lam0 && (rc = copy_in(ctx, P.lam, lam0, (size_t)B * P.n_C, mem_kind, st))) return rc;
    if (ws) {
        CK(cudaMemcpyAsync(P.mu + (size_t)B * 2, P.mu, (size_t)B * 2 * 8, cudaMemcpyDeviceToDevice, st));
        if ((rc = ddnm_ws_predict_dev(ctx, B, P.mu, P.x, nullptr, st))) return rc;
        CK(cudaMemsetAsync(P.x + (size_t)B * P.n_D, 0, (size_t)B * P.n_D * 8, st));
    }
    const int max_passes = 3 + ctx->opt.max_iter * (ctx->opt.max_backtracks + 1);
    P.tol = ctx->opt.tol;
    P.c1 = ctx->opt.armijo_c1;
    P.beta = ctx->opt.beta;
    P.max_iter = ctx->opt.max_iter;
    P.max_bt = ctx->opt.max_backtracks;
    P.step_tol = fp64 ? 0.0 : ctx->opt.step_tol;
    P.con_split = ctx->tune.con_split;
    P.n_split = (P.N_A + P.con_split - 1) / P.con_split;
    P.d_gemm = resolved_dgemm(ctx);
    resolve_atil(ctx, P);
    if (ctx->tune.graph && !ctx->timing) {
        rc = fp64 ? solve_graph<double>(ctx, P, B, Bw, ws, x0 != nullptr, lam0 != nullptr, max_passes, st)
                  : solve_graph<float>(ctx, P, B, Bw, ws, x0 != nullptr, lam0 != nullptr, max_passes, st);
        if (rc) return rc;
    } else {
        // host-driven passes: the running count is read back every few passes
        k_init<<<Bw, 128, 0, st>>>(P, Bw, x0 != nullptr || ws, lam0 != nullptr, lam0 ? MODE_INIT1 : MODE_INIT0, fp64);
        CK(cudaGetLastError());
        ctx->tm.other_launches++;
        const bool persist = ctx->tune.eval_persist > 0;
        const int check_every = 4;
        int Bp = Bw;                      // instances in the passes (2B during the warm-start screening)
        for (int pass = 0; pass < max_passes; ++pass) {
            rc = fp64 ? run_pass<double>(ctx, P, Bp, st, persist, true) : run_pass<float>(ctx, P, Bp, st, persist, true);
            if (rc) return rc;
            if (ws && pass == 1) {        // both starts linearised: keep the better one per instance
                k_ws_select<<<B, 128, 0, st>>>(P, B);
                CK(cudaGetLastError());
                ctx->tm.other_launches++;
                Bp = B;
                continue;
            }
            if (pass % check_every == check_every - 1 || pass == max_passes - 1) {
                CK(cudaMemcpyAsync(ctx->h_active, P.active, sizeof(int), cudaMemcpyDeviceToHost, st));
                CK(cudaStreamSynchronize(st));
                if (*ctx->h_active == 0) break;
            }
        }
    }
    if (x_out && (rc = copy_out(ctx, x_out, P.x, (size_t)B * P.n_D * 8, mem_kind, st))) return rc;
    if (lam_out && (rc = copy_out(ctx, lam_out, P.lam, (size_t)B * P.n_C * 8, mem_kind, st))) return rc;
    if (stats) {
        Tmp t;
        ddnm_stats* dstats = stats;
        if (mem_kind == DDNM_MEM_HOST) {
            CK(cudaMalloc(&t.p, (size_t)B * sizeof(ddnm_stats)));
            dstats = (ddnm_stats*)t.p;
        }
        k_stats<<<(B + 127) / 128, 128, 0, st>>>(P, B, dstats);
        CK(cudaGetLastError());
        ctx->tm.other_launches++;
        if (mem_kind == DDNM_MEM_HOST) {
            CK(cudaMemcpyAsync(stats, dstats, (size_t)B * sizeof(ddnm_stats), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
        }
    }
    if (state_out) {
        Tmp t;
        double* dstate = state_out;
        if (mem_kind == DDNM_MEM_HOST) {
            CK(cudaMalloc(&t.p, (size_t)B * P.N_x * 8));
            dstate = (double*)t.p;
        }
        rc = fp64 ? reconstruct<double>(ctx, P, B, P.x, dstate, st) : reconstruct<float>(ctx, P, B, P.x, dstate, st);
        if (rc) return rc;
        if (mem_kind == DDNM_MEM_HOST) {
            CK(cudaMemcpyAsync(state_out, dstate, (size_t)B * P.N_x * 8, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
        }
    }
    if (mem_kind == DDNM_MEM_HOST) CK(cudaStreamSynchronize(st));
    return tflush(ctx, st);
}

namespace {
// One evaluation at (x, lam) for B instances (no iteration).
template <typename T>
int eval_once(ddnm_ctx* ctx, ProbDev& P, int B, const double* mu, const double* x, const double* lam, int mem_kind,
              cudaStream_t st, double* r_hr_dev) {
    int rc;
    if ((rc = copy_in(ctx, P.mu, mu, (size_t)B * 2, mem_kind, st))) return rc;
    if ((rc = copy_in(ctx, P.x, x, (size_t)B * P.n_D, mem_kind, st))) return rc;
    if (lam && (rc = copy_in(ctx, P.lam, lam, (size_t)B * P.n_C, mem_kind, st))) return rc;
    k_init<<<B, 128, 0, st>>>(P, B, 1, lam != nullptr, MODE_INIT1, (int)(sizeof(T) == 8));
    CK(cudaGetLastError());
    ctx->tm.other_launches++;
    P.r_hr = r_hr_dev;
    P.d_gemm = resolved_dgemm(ctx);
    resolve_atil(ctx, P);
    return launch_eval<T>(ctx, P, B, st);
}
}  // namespace

extern "C" int ddnm_residual(ddnm_ctx* ctx, int B, const double* mu, const double* x, const double* lam, double* F_out,
                             double* r_hr_out, double* r_full_out, int mem_kind, void* stream) {
    int rc = prepare(ctx, B, mem_kind);
    if (rc) return rc;
    if (!mu || !x) return ddnm_fail(ctx, DDNM_E_INVALID, "mu and x are required");
    cudaStream_t st = (cudaStream_t)stream;
    ProbDev P = ctx->pd;
    const bool fp64 = ctx->precision == DDNM_FP64;
    const bool host = mem_kind == DDNM_MEM_HOST;
    Tmp tF, tR, tS, tRF;
    double* dF = F_out;
    double* dR = r_hr_out;
    if (host && F_out) { CK(cudaMalloc(&tF.p, (size_t)B * (P.n_D + P.n_C) * 8)); dF = (double*)tF.p; }
    if (host && r_hr_out) { CK(cudaMalloc(&tR.p, (size_t)B * P.sum_NB * 8)); dR = (double*)tR.p; }
    rc = fp64 ? eval_once<double>(ctx, P, B, mu, x, lam, mem_kind, st, dR) : eval_once<float>(ctx, P, B, mu, x, lam, mem_kind, st, dR);
    if (rc) return rc;
    if (dF) {
        k_gather<<<B, 128, 0, st>>>(P, B, dF, nullptr, nullptr, nullptr);
        CK(cudaGetLastError());
        ctx->tm.other_launches++;
    }
    if (r_full_out) {
        CK(cudaMalloc(&tS.p, (size_t)B * P.N_x * 8));
        double* dstate = (double*)tS.p;
        rc = fp64 ? reconstruct<double>(ctx, P, B, P.x, dstate, st) : reconstruct<float>(ctx, P, B, P.x, dstate, st);
        if (rc) return rc;
        double* dRF = r_full_out;
        if (host) { CK(cudaMalloc(&tRF.p, (size_t)B * P.N_x * 8)); dRF = (double*)tRF.p; }
        const long long tot = (long long)B * P.nx * P.ny;
        k_fom_residual<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(P, B, dstate, dRF);
        CK(cudaGetLastError());
        ctx->tm.other_launches++;
        if (host) CK(cudaMemcpyAsync(r_full_out, dRF, (size_t)B * P.N_x * 8, cudaMemcpyDeviceToHost, st));
    }
    if (host && F_out) CK(cudaMemcpyAsync(F_out, dF, (size_t)B * (P.n_D + P.n_C) * 8, cudaMemcpyDeviceToHost, st));
    if (host && r_hr_out) CK(cudaMemcpyAsync(r_hr_out, dR, (size_t)B * P.sum_NB * 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));   // temporaries are freed on return
    return tflush(ctx, st);
}

extern "C" int ddnm_reconstruct(ddnm_ctx* ctx, int B, const double* x, double* state_out, int mem_kind, void* stream) {
    int rc = prepare(ctx, B, mem_kind);
    if (rc) return rc;
    if (!x || !state_out) return ddnm_fail(ctx, DDNM_E_INVALID, "x and state_out are required");
    cudaStream_t st = (cudaStream_t)stream;
    const ProbDev& P = ctx->pd;
    const bool host = mem_kind == DDNM_MEM_HOST;
    Tmp tS;
    const double* dx = x;
    double* dS = state_out;
    if (host) {
        if ((rc = copy_in(ctx, P.x, x, (size_t)B * P.n_D, mem_kind, st))) return rc;
        dx = P.x;
        CK(cudaMalloc(&tS.p, (size_t)B * P.N_x * 8));
        dS = (double*)tS.p;
    }
    rc = ctx->precision == DDNM_FP64 ? reconstruct<double>(ctx, P, B, dx, dS, st)
                                     : reconstruct<float>(ctx, P, B, dx, dS, st);
    if (rc) return rc;
    if (host) {
        CK(cudaMemcpyAsync(state_out, dS, (size_t)B * P.N_x * 8, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));   // the temporary is freed on return
    }
    return DDNM_OK;
}

extern "C" int ddnm_linearize(ddnm_ctx* ctx, int B, const double* mu, const double* x, const double* lam, double* H_out,
                              double* D_out, double* Atil_out, int mem_kind, void* stream) {
    int rc = prepare(ctx, B, mem_kind);
    if (rc) return rc;
    if (!mu || !x) return ddnm_fail(ctx, DDNM_E_INVALID, "mu and x are required");
    cudaStream_t st = (cudaStream_t)stream;
    ProbDev P = ctx->pd;
    const bool fp64 = ctx->precision == DDNM_FP64;
    const bool host = mem_kind == DDNM_MEM_HOST;
    size_t hsum = 0, dsum = 0;
    for (const SubDev& S : ctx->hsub) {
        hsum += (size_t)S.ni * S.ni;
        dsum += (size_t)P.n_C * S.nG;
    }
    Tmp tH, tD, tA;
    double *dH = H_out, *dD = D_out, *dA = Atil_out;
    if (host && H_out) { CK(cudaMalloc(&tH.p, B * hsum * 8)); dH = (double*)tH.p; }
    if (host && D_out) { CK(cudaMalloc(&tD.p, B * dsum * 8)); dD = (double*)tD.p; }
    if (host && Atil_out) { CK(cudaMalloc(&tA.p, (size_t)B * P.n_C * 8)); dA = (double*)tA.p; }
    rc = fp64 ? eval_once<double>(ctx, P, B, mu, x, lam, mem_kind, st, nullptr)
              : eval_once<float>(ctx, P, B, mu, x, lam, mem_kind, st, nullptr);
    if (rc) return rc;
    k_gather<<<B, 128, 0, st>>>(P, B, nullptr, dH, dD, dA);
    CK(cudaGetLastError());
    ctx->tm.other_launches++;
    if (host && H_out) CK(cudaMemcpyAsync(H_out, dH, B * hsum * 8, cudaMemcpyDeviceToHost, st));
    if (host && D_out) CK(cudaMemcpyAsync(D_out, dD, B * dsum * 8, cudaMemcpyDeviceToHost, st));
    if (host && Atil_out) CK(cudaMemcpyAsync(Atil_out, dA, (size_t)B * P.n_C * 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return tflush(ctx, st);
}

extern "C" int ddnm_timing_enable(ddnm_ctx* ctx, int on) {
    if (!ctx) return DDNM_E_INVALID;
    fold_pending(ctx);
    ctx->timing = on != 0;
    ctx->n_events = 0;
    if (on) ctx->tm = ddnm_timing{};
    return DDNM_OK;
}

extern "C" int ddnm_get_timing(const ddnm_ctx* ctx, ddnm_timing* out) {
    if (!ctx || !out) return DDNM_E_INVALID;
    fold_pending(const_cast<ddnm_ctx*>(ctx));
    *out = ctx->tm;
    return DDNM_OK;
}

void ddnm_release_graph(ddnm_ctx* ctx) {
    fold_pending(ctx);
    drop_graph(ctx);
    if (ctx->cap_main) cudaStreamDestroy(ctx->cap_main);
    if (ctx->cap_body) cudaStreamDestroy(ctx->cap_body);
    if (ctx->pass_ev) cudaEventDestroy(ctx->pass_ev);
    if (ctx->h_pass) cudaFreeHost(ctx->h_pass);
    ctx->cap_main = ctx->cap_body = nullptr;
    ctx->pass_ev = nullptr;
    ctx->h_pass = nullptr;
}

extern "C" int ddnm_set_tune(ddnm_ctx* ctx, const ddnm_tune* t) {
    if (!ctx || !t) return DDNM_E_INVALID;
    const bool pow2 = t->con_split > 0 && (t->con_split & (t->con_split - 1)) == 0;
    if (t->graph < 0 || t->graph > 1 || t->chains < 1 || t->chains > MAX_CHAINS || !pow2 ||
        t->con_split < MIN_CON_SPLIT || t->con_split > MAX_CON_SPLIT || t->eval_persist < 0 || t->eval_persist > 8 ||
        t->d_gemm < -1 || t->d_gemm > 2 || t->eval_groups < 0 || t->eval_groups > 1 || t->atil < -1 || t->atil > 1)
        return ddnm_fail(ctx, DDNM_E_INVALID, "tune: graph 0/1, chains 1..64, con_split 512, 1024 or 2048, "
                                              "eval_persist 0..8, d_gemm -1..2, eval_groups 0/1, atil -1..1");
    ctx->tune = *t;
    return DDNM_OK;
}

extern "C" int ddnm_get_tune(const ddnm_ctx* ctx, ddnm_tune* t) {
    if (!ctx || !t) return DDNM_E_INVALID;
    *t = ctx->tune;
    return DDNM_OK;
}

extern "C" int ddnm_autotune(ddnm_ctx* ctx, int B, const double* mu, int mem_kind, void* stream, int max_iter,
                             int reps, ddnm_tune* best, float* best_ms) {
    if (!ctx) return DDNM_E_INVALID;
    if (B < 1 || !mu || max_iter < 0) return ddnm_fail(ctx, DDNM_E_INVALID, "autotune: B >= 1, mu and max_iter >= 0");
    cudaStream_t st = (cudaStream_t)stream;
    const ddnm_options opt_saved = ctx->opt;
    const bool timing_saved = ctx->timing;
    if (max_iter > 0) ctx->opt.max_iter = max_iter;
    ctx->timing = false;
    reps = std::max(1, std::min(reps, 64));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = DDNM_OK;
    auto finish = [&](int r) {
        ctx->opt = opt_saved;
        ctx->timing = timing_saved;
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        return r;
    };
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return finish(ddnm_fail(ctx, DDNM_E_CUDA, "autotune: event creation failed"));
    auto time_plan = [&](const ddnm_tune& t, float* ms) -> int {
        ctx->tune = t;
        int r = ddnm_solve_batch(ctx, B, mu, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, mem_kind, stream);
        if (r) return r;
        std::vector<float> v;
        for (int k = 0; k < reps; ++k) {
            if (cudaEventRecord(e0, st) != cudaSuccess) return ddnm_fail(ctx, DDNM_E_CUDA, "autotune: event record");
            r = ddnm_solve_batch(ctx, B, mu, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, mem_kind, stream);
            if (r) return r;
            float m = 0.f;
            if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&m, e0, e1) != cudaSuccess)
                return ddnm_fail(ctx, DDNM_E_CUDA, "autotune: event timing");
            v.push_back(m);
        }
        std::sort(v.begin(), v.end());
        *ms = v[v.size() / 2];
        return DDNM_OK;
    };
    ddnm_tune cur = ctx->tune;
    cur.graph = 1;
    float cur_ms = 0.f;
    if ((rc = time_plan(cur, &cur_ms))) return finish(rc);
    auto sweep = [&](int ddnm_tune::*knob, std::initializer_list<int> values) -> int {
        for (int v : values) {
            if (v == cur.*knob) continue;
            if (knob == &ddnm_tune::chains && v > B) continue;
            ddnm_tune t = cur;
            t.*knob = v;
            float ms = 0.f;
            const int r = time_plan(t, &ms);
            if (r) return r;
            if (ms < cur_ms) {
                cur = t;
                cur_ms = ms;
            }
        }
        return DDNM_OK;
    };
    if ((rc = sweep(&ddnm_tune::chains, {1, 2, 4, 8, 16, 32, 64}))) return finish(rc);
    if ((rc = sweep(&ddnm_tune::eval_persist, {0, 1, 2, 4}))) return finish(rc);
    if ((rc = sweep(&ddnm_tune::con_split, {512, 1024, 2048}))) return finish(rc);
    if (cur.d_gemm < 0) cur.d_gemm = resolved_dgemm(ctx);
    if (ddnm_dgemm_tc_ok(ctx)) {
        if ((rc = sweep(&ddnm_tune::d_gemm, {0, 1, 2}))) return finish(rc);
    } else if ((rc = sweep(&ddnm_tune::d_gemm, {0, 1}))) {
        return finish(rc);
    }
    if ((rc = sweep(&ddnm_tune::eval_groups, {0, 1}))) return finish(rc);
    if (ctx->precision == DDNM_MIXED) {
        if (cur.atil < 0) cur.atil = ctx->atil_auto;
        if ((rc = sweep(&ddnm_tune::atil, {0, 1}))) return finish(rc);
    }
    ctx->tune = cur;
    if (best) *best = cur;
    if (best_ms) *best_ms = cur_ms;
    return finish(DDNM_OK);
}

void ddnm_release_events(ddnm_ctx* ctx) {
    for (cudaEvent_t e : ctx->events) cudaEventDestroy(e);
    ctx->events.clear();
}

// ------------------------------------------------------------------ evaluation without allocation
//
// ddnm_residual_noalloc: the evaluation of ddnm_residual (F only) for callers that cannot allocate
// device memory (see include/ddnm.h).  Its scratch -- per-instance solver state, Dirichlet data,
// interface outputs, per-subdomain Gauss-Newton / Schur blocks, Atil -- lives in the file-scope array
// below instead of the context's workspace.  Each GPU that loads this library holds the array until
// the process exits.  All calls share it: calls that overlap on the GPU race on it.

#define DDNM_NOALLOC_SCRATCH_BYTES (16u << 20)   /* 16 MiB */

static __device__ __align__(256) unsigned char g_noalloc_scratch[DDNM_NOALLOC_SCRATCH_BYTES];

namespace {

// Device address of g_noalloc_scratch, looked up with cudaGetSymbolAddress once per device and CUDA context
// (with that device current), on the first no-allocation call there.  The host-side name of the array is only
// a stand-in.  The cache is keyed by the context's unique id (cuCtxGetId, reached through the runtime's
// driver entry points, so the library does not link libcuda): after the application resets the device
// (cudaDeviceReset) the primary context, and with it the array's address, is new, and the next call looks
// the address up again.
std::mutex g_noalloc_mu;
struct NoallocAddr {
    void* p = nullptr;
    unsigned long long ctx_id = 0;
};
NoallocAddr g_noalloc_addr[128];

typedef int (*ctx_get_current_fn)(void** pctx);                    // cuCtxGetCurrent(CUcontext*)
typedef int (*ctx_get_id_fn)(void* ctx, unsigned long long* id);   // cuCtxGetId(CUcontext, unsigned long long*)

// unique id of the CUDA context current on this thread (0 if it cannot be read)
unsigned long long current_ctx_id() {
    static ctx_get_current_fn get_cur = nullptr;
    static ctx_get_id_fn get_id = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        cudaDriverEntryPointQueryResult q;
        void* f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_cur = (ctx_get_current_fn)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (ctx_get_id_fn)f;
    }
    void* c = nullptr;
    unsigned long long id = 0;
    if (get_cur && get_id && get_cur(&c) == 0 && c && get_id(c, &id) == 0) return id;
    return 0;
}

int noalloc_scratch(ddnm_ctx* ctx, void** out) {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (ctx->device < 0 || ctx->device >= 128) return ddnm_fail(ctx, DDNM_E_INVALID, "device ordinal out of range");
    NoallocAddr& a = g_noalloc_addr[ctx->device];
    const unsigned long long id = current_ctx_id();
    if (!a.p || id == 0 || id != a.ctx_id) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return ddnm_fail(ctx, DDNM_E_CUDA, std::string("cudaGetSymbolAddress(no-allocation scratch): ") +
                                                   cudaGetErrorString(e));
        a.p = p;
        a.ctx_id = id;
    }
    *out = a.p;
    return DDNM_OK;
}

// A caller's pointer must be device (or managed) memory of ctx's device: the kernels dereference it.
int check_device_ptr(ddnm_ctx* ctx, const void* p, const char* what) {
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return ddnm_fail(ctx, DDNM_E_INVALID, std::string("ddnm_residual_noalloc: ") + what +
                                                  " is not a pointer the CUDA runtime knows");
    }
    if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) ||
        (at.type == cudaMemoryTypeDevice && at.device != ctx->device))
        return ddnm_fail(ctx, DDNM_E_INVALID, std::string("ddnm_residual_noalloc: ") + what +
                                                  " must be device memory on device " + std::to_string(ctx->device));
    return DDNM_OK;
}

// per-instance state and Dirichlet data for one evaluation (no copies of the caller's inputs)
__global__ void k_noalloc_init(ProbDev P, int B, int fp64) {
    const int b = blockIdx.x, tid = threadIdx.x, nth = blockDim.x;
    if (b >= B) return;
    const double a = P.mu[2 * b], lm = P.mu[2 * b + 1];
    for (int p = tid; p < P.n_bnd; p += nth) {
        const double x = P.bx0 + P.bnd_ij[2 * p] * P.hx, y = P.by0 + P.bnd_ij[2 * p + 1] * P.hy;
        double u, v;
        exact_uv(x, y, a, lm, P.nu, u, v);
        const size_t o = ((size_t)b * P.n_bnd + p) * 2;
        if (fp64) {
            ((double*)P.bnd)[o] = u;
            ((double*)P.bnd)[o + 1] = v;
        } else {
            ((float*)P.bnd)[o] = (float)u;
            ((float*)P.bnd)[o + 1] = (float)v;
        }
    }
    if (tid == 0) {
        int* ist = P.ist + (size_t)b * INST_INTS;
        for (int k = 0; k < INST_INTS; ++k) ist[k] = 0;
        ist[I_STATUS] = ST_RUNNING;
        ist[I_MODE] = MODE_INIT1;
    }
}

template <typename T>
int noalloc_eval(ddnm_ctx* ctx, ProbDev& P, int B, double* F_out, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    for (const auto& g : ctx->eval_classes) {
        e = cudaFuncSetAttribute(eval_kernel<T>(g.ro, g.rg), cudaFuncAttributeMaxDynamicSharedMemorySize, g.smem);
        if (e != cudaSuccess) return cfail(ctx, e, "cudaFuncSetAttribute(k_eval)");
    }
    k_noalloc_init<<<B, 128, 0, st>>>(P, B, (int)(sizeof(T) == 8));
    for (const auto& g : ctx->eval_classes)
        eval_kernel<T>(g.ro, g.rg)<<<B * g.n, g.nt, g.smem, st>>>(P, B, ctx->d_classes + g.off, g.n, nullptr,
                                                                           g.stride);
    if (P.d_gemm) {
        e = launch_dgemm<T>(ctx, P, B, st);
        if (e != cudaSuccess) return cfail(ctx, e, "no-allocation D_i product launch");
    }
    {
        const int nrg = con_row_groups(ctx, P, B);
        k_constraint<T, NG_SMALL><<<dim3(P.n_split * nrg, B), CON_THREADS, P.con_split * sizeof(double), st>>>(
            P, B, nrg);        // no factorisation CTAs here
    }
    k_gather<<<B, 128, 0, st>>>(P, B, F_out, nullptr, nullptr, nullptr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cfail(ctx, e, "no-allocation evaluation launch");
    return DDNM_OK;
}

}  // namespace

extern "C" int ddnm_residual_noalloc(ddnm_ctx* ctx, int B, const double* mu, const double* x, const double* lam,
                                     double* F_out, void* stream) {
    if (!ctx) return DDNM_E_INVALID;
    if (B < 1 || !mu || !x || !F_out) return ddnm_fail(ctx, DDNM_E_INVALID, "B >= 1 and device mu, x, F_out are required");
    if (!ctx->finalized)
        return ddnm_fail(ctx, DDNM_E_STATE,
                         "the decoder and constraint tables are not on the device yet: make one allocating call "
                         "(ddnm_residual, ddnm_linearize or ddnm_solve_batch) first");
    ProbDev P = ctx->pd;
    P.d_gemm = resolved_dgemm(ctx);
    const size_t tsize = ctx->precision == DDNM_FP64 ? 8 : 4;
    auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
    size_t o = 0;
    const size_t o_ist = o; o = al(o + (size_t)B * INST_INTS * 4);
    const size_t o_dst = o; o = al(o + (size_t)B * INST_DBLS * 8);
    const size_t o_bnd = o; o = al(o + (size_t)B * std::max(P.n_bnd, 1) * 2 * 8);
    const size_t o_gG = o; o = al(o + (size_t)B * P.sum_NG * tsize);
    const size_t o_PG = o; o = al(o + (P.d_gemm ? (size_t)B * P.pg_stride * tsize : 0));
    const size_t o_blk = o; o = al(o + (size_t)B * P.blk_stride * 8);
    const size_t o_At = o; o = al(o + (size_t)B * P.n_split * P.n_C * 8);
    const size_t o_lz = o; o = al(o + (size_t)B * P.n_C * 8);
    if (o > DDNM_NOALLOC_SCRATCH_BYTES) {
        const size_t per = o / B + 1;
        return ddnm_fail(ctx, DDNM_E_UNSUPPORTED,
                         "ddnm_residual_noalloc: " + std::to_string(B) + " instances need " + std::to_string(o) +
                             " bytes of scratch, the static array holds " + std::to_string(DDNM_NOALLOC_SCRATCH_BYTES) +
                             " (about " + std::to_string(DDNM_NOALLOC_SCRATCH_BYTES / per) + " instances of this problem)");
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cfail(ctx, e, "cudaSetDevice");
    int rc = check_device_ptr(ctx, mu, "mu");
    if (!rc) rc = check_device_ptr(ctx, x, "x");
    if (!rc && lam) rc = check_device_ptr(ctx, lam, "lam");
    if (!rc) rc = check_device_ptr(ctx, F_out, "F_out");
    if (rc) return rc;
    void* base = nullptr;
    rc = noalloc_scratch(ctx, &base);
    if (rc) return rc;
    char* s = (char*)base;
    cudaStream_t st = (cudaStream_t)stream;
    P.mu = const_cast<double*>(mu);        // read only by the kernels below
    P.xt = const_cast<double*>(x);         // read only by k_eval
    P.ist = (int*)(s + o_ist);
    P.dst = (double*)(s + o_dst);
    P.bnd = (void*)(s + o_bnd);
    P.gG = (void*)(s + o_gG);
    P.PG = (void*)(s + o_PG);
    P.blk = (double*)(s + o_blk);
    P.Atil = (double*)(s + o_At);
    P.Spart = nullptr;                     // no KKT step here
    P.r_hr = nullptr;
    if (lam) {
        P.lamt = const_cast<double*>(lam);  // read only by k_eval
    } else {
        // the array keeps the previous call's contents: the zero multiplier must be cleared each call
        P.lamt = (double*)(s + o_lz);
        e = cudaMemsetAsync(P.lamt, 0, (size_t)B * P.n_C * 8, st);
        if (e != cudaSuccess) return cfail(ctx, e, "cudaMemsetAsync(zero multipliers)");
    }
    return ctx->precision == DDNM_FP64 ? noalloc_eval<double>(ctx, P, B, F_out, st)
                                       : noalloc_eval<float>(ctx, P, B, F_out, st);
}
