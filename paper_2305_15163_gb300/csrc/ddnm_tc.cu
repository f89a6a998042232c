// sm_103a tensor-core (tcgen05) form of the batched D_i GEMM of the mixed path.
//
// D_i = C A_i dg_i^G/dxh = Q_i P_G (Eq. sqp_block_matrices, with Q_i = C A_i diag(scale) W2~ precomputed):
// Q_i (n_C x h_G) is shared by every instance of subdomain i, so the product over a tile of instances is one
// GEMM [n_C x h_G] x [h_G x (instances x n^G)].  k_dgemm_tc runs it on the 5th-generation tensor cores:
//   - CTA = (subdomain, tile of instances); M = 128 rows of C (n_C <= 128, zero rows above n_C),
//     N = instances x n^G columns (padded to a multiple of 16, at most 256), K = h_G in chunks of 32;
//   - FP32 accuracy from TF32 operands by splitting each operand x = hi + lo (hi = tf32(x), lo = tf32(x - hi))
//     and accumulating hi*hi + hi*lo + lo*hi in the FP32 accumulator (the lo*lo term is below 2^-22 of the
//     product): three tcgen05.mma.kind::tf32 per K step, the accumulator in tensor memory;
//   - Q_i is split and laid out on the host in the tensor core's shared-memory order (K-major, no swizzle:
//     8-row x 16-byte core matrices, K-adjacent ones 128 bytes apart, M-adjacent ones 1024 bytes apart), so a
//     chunk is one contiguous 16 KB block per part, copied by the TMA engine (cp.async.bulk) with completion
//     on an mbarrier; P_G of the tile's instances is split and written in the same order by the threads;
//   - two stages: while the tensor core works on chunk c, the threads stage chunk c + 1;
//   - epilogue: tcgen05.ld of the accumulator rows, D_i into the blocks (FP64), rho_i^G += D_i^T lambda and
//     phi_i = ||rho_i||^2 in FP64 (Eq. optimality_residuals_GN).
// Every wait on an mbarrier is bounded; on a timeout the kernel records DDNM_TC_TIMEOUT in P.err, waits (again
// bounded) for what it issued, frees its tensor memory and returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ddnm_ctx.h"

using namespace ddnm;

namespace {

constexpr int TC_THREADS = 256;
constexpr int TC_KC = 32;                       // hidden units per K chunk (4 MMA K steps of 8)
constexpr int TC_M = 128;
constexpr int TC_MAXN = 256;
constexpr int TC_ABYTES = TC_M * TC_KC * 4;     // one part (hi or lo) of a Q chunk
constexpr int PG_BATCH = 8;                     // P_G loads a staging thread has in flight
constexpr long long TC_SPIN = 1LL << 22;        // bounded mbarrier waits (try_wait polls)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start address, leading (K-direction) and stride (M/N-direction) byte offsets
// between core matrices, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both K-major, M x N
__device__ __forceinline__ uint32_t umma_idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
                 "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

// true once the phase with parity `parity` of the mbarrier has completed; false after TC_SPIN polls
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (long long it = 0; it < TC_SPIN; ++it) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

// TMA bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) from global to shared memory,
// counted on the mbarrier's transaction count
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// row-group / K-block layout of a K-major operand with 32 K values per chunk: element (row, k) of the chunk
__device__ __forceinline__ int kmajor_index(int row, int k) {
    return ((row >> 3) * (TC_KC / 4) + (k >> 2)) * 32 + (row & 7) * 4 + (k & 3);
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// CTA (subdomain blockIdx.x, instances b0 .. b0 + TB - 1); Np = TB n^G rounded up to 16 (<= 256).
__global__ void __launch_bounds__(TC_THREADS, 1) k_dgemm_tc(ProbDev P, int B, int TB, int Np) {
    extern __shared__ __align__(1024) unsigned char tsm[];
    __shared__ __align__(8) uint64_t bar_full[2], bar_done[2];
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    __shared__ unsigned char s_run[TC_MAXN];
    const int si = blockIdx.x, tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const SubDev& S = P.sub[si];
    const int nC = P.n_C, nG = S.nG, nO = S.nO, ni = S.ni, hG = S.hG;
    const int b0 = blockIdx.y * TB, cols = TB * nG;
    const int nch = S.hGp / TC_KC;
    const uint32_t BBYTES = (uint32_t)Np * TC_KC * 4;
    // stage s: Q hi, Q lo (16 KB each), then P_G hi, P_G lo (BBYTES each)
    auto Ahi = [&](int st) { return (float*)(tsm + st * TC_ABYTES); };
    auto Alo = [&](int st) { return (float*)(tsm + (2 + st) * TC_ABYTES); };
    auto Bhi = [&](int st) { return (float*)(tsm + 4 * TC_ABYTES + st * BBYTES); };
    auto Blo = [&](int st) { return (float*)(tsm + 4 * TC_ABYTES + (2 + st) * BBYTES); };
    int any = 0;
    for (int t = tid; t < TB; t += TC_THREADS) {
        const int b = b0 + t;
        const int r = b < B && P.ist[(size_t)b * INST_INTS + I_STATUS] == ST_RUNNING;
        s_run[t] = (unsigned char)r;
    }
    if (tid == 0) {
        s_fail = 0;
        for (int s = 0; s < 2; ++s) {
            mbar_init(smem_u32(&bar_full[s]), 1);
            mbar_init(smem_u32(&bar_done[s]), 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    for (int t = 0; t < TB; ++t) any |= s_run[t];
    if (!any) return;                                   // uniform: no instance of the tile is running
    if (w == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(TC_MAXN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    const uint32_t idesc = umma_idesc_tf32(TC_M, Np);
    const float* Qhi = P.Qtc + S.qtc;
    const float* Qlo = Qhi + (size_t)S.hGp * TC_M;
    const float* PG = (const float*)P.PG;
    int issued = 0;                                     // chunks whose MMAs thread 0 committed
    for (int c = 0; c < nch; ++c) {
        const int s = c & 1;
        if (c >= 2 && !mbar_wait(smem_u32(&bar_done[s]), ((c >> 1) - 1) & 1)) s_fail = 1;
        __syncthreads();
        if (s_fail) break;
        if (tid == 0) {                                 // Q chunk c: two contiguous 16 KB blocks
            const uint32_t bf = smem_u32(&bar_full[s]);
            mbar_expect_tx(bf, 2 * TC_ABYTES);
            bulk_g2s(smem_u32(Ahi(s)), Qhi + (size_t)c * TC_M * TC_KC, TC_ABYTES, bf);
            bulk_g2s(smem_u32(Alo(s)), Qlo + (size_t)c * TC_M * TC_KC, TC_ABYTES, bf);
        }
        // P_G chunk: column n = t n^G + k of the tile, K = hidden units h0 .. h0 + 31; split into hi + lo.  Each
        // thread issues PG_BATCH loads before it splits and stores any (P_G is read-only here), so the chunk's
        // loads are in flight together instead of one memory latency per element.
        const int h0 = c * TC_KC, tot = TB * TC_KC * nG;
        for (int e0 = tid; e0 < tot; e0 += PG_BATCH * TC_THREADS) {
            float v[PG_BATCH];
#pragma unroll
            for (int u = 0; u < PG_BATCH; ++u) {
                const int e = e0 + u * TC_THREADS;
                v[u] = 0.f;
                if (e < tot) {
                    const int t = e / (TC_KC * nG), rem = e - t * TC_KC * nG;
                    if (h0 + rem / nG < hG && s_run[t])
                        v[u] = __ldg(PG + (size_t)(b0 + t) * P.pg_stride + S.pgoff + (size_t)h0 * nG + rem);
                }
            }
#pragma unroll
            for (int u = 0; u < PG_BATCH; ++u) {
                const int e = e0 + u * TC_THREADS;
                if (e < tot) {
                    const int t = e / (TC_KC * nG), rem = e - t * TC_KC * nG;
                    const int hh = rem / nG, k = rem - hh * nG;
                    const float hi = tf32_rna(v[u]), lo = tf32_rna(v[u] - hi);
                    const int idx = kmajor_index(t * nG + k, hh);
                    Bhi(s)[idx] = hi;
                    Blo(s)[idx] = lo;
                }
            }
        }
        for (int e = tid; e < (Np - cols) * TC_KC; e += TC_THREADS) {   // padding columns
            const int n = cols + e / TC_KC, hh = e % TC_KC;
            Bhi(s)[kmajor_index(n, hh)] = 0.f;
            Blo(s)[kmajor_index(n, hh)] = 0.f;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            if (!mbar_wait(smem_u32(&bar_full[s]), (c >> 1) & 1)) {
                s_fail = 1;
            } else {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                for (int ks = 0; ks < TC_KC / 8; ++ks) {
                    const uint32_t off = ks * 2 * 128;          // two K-adjacent core matrices per K step
                    const uint64_t ah = umma_desc(smem_u32(Ahi(s)) + off, 128, 1024);
                    const uint64_t al = umma_desc(smem_u32(Alo(s)) + off, 128, 1024);
                    const uint64_t bh = umma_desc(smem_u32(Bhi(s)) + off, 128, 1024);
                    const uint64_t bl = umma_desc(smem_u32(Blo(s)) + off, 128, 1024);
                    mma_tf32(tmem, ah, bh, idesc, (c > 0 || ks > 0) ? 1u : 0u);
                    mma_tf32(tmem, ah, bl, idesc, 1u);
                    mma_tf32(tmem, al, bh, idesc, 1u);
                }
                mma_commit(smem_u32(&bar_done[s]));
                issued = c + 1;
            }
        }
    }
    // the last committed chunk's MMAs (the commit tracks every earlier MMA of the thread)
    __shared__ int s_issued;
    if (tid == 0) s_issued = issued;
    __syncthreads();
    const int last = s_issued - 1;
    bool ok = !s_fail && s_issued == nch;
    if (last >= 0 && !mbar_wait(smem_u32(&bar_done[last & 1]), (last >> 1) & 1)) ok = false;
    if (tid == 0 && s_fail && last + 1 < nch) {        // a Q copy may still be in flight: let it land
        const int c = last + 1;
        mbar_wait(smem_u32(&bar_full[c & 1]), (c >> 1) & 1);
    }
    __syncthreads();
    if (!ok) {
        if (tid == 0) atomicExch(P.err, DDNM_TC_TIMEOUT);
    } else {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // epilogue: warp w reads accumulator lanes 32 (w % 4) .. + 31 (rows c of D), columns half w / 4
        double* lam_s = (double*)tsm;                              // TB x nC multipliers (stages are free now)
        double* red = lam_s + (size_t)TB * nC;                     // 8 warps x Np partial sums of D^T lambda
        for (int e = tid; e < TB * nC; e += TC_THREADS) {
            const int b = b0 + e / nC;
            lam_s[e] = b < B ? P.lamt[(size_t)b * nC + e % nC] : 0.0;
        }
        __syncthreads();
        const int row = 32 * (w & 3) + lane, half = w >> 2;
        const int nhalf = (Np / 2 + 7) & ~7;
        const int n_lo = half * nhalf, n_hi = min(Np, n_lo + nhalf);
        const BlkLayout BL = blk_layout(ni, nG, nC);
        for (int n0 = n_lo; n0 < n_hi; n0 += 8) {
            uint32_t r[8];
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7])
                         : "r"(tmem + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)n0));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int n = n0 + j;
                const int t = n / nG, k = n - t * nG;
                const bool live = n < cols && row < nC && s_run[t];
                const double v = (double)__uint_as_float(r[j]);
                if (live) P.blk[(size_t)(b0 + t) * P.blk_stride + S.blk + BL.D + row * nG + k] = v;
                double p = (n < cols && row < nC) ? v * lam_s[(size_t)t * nC + row] : 0.0;
                p = warp_sum_d(p);
                if (lane == 0) red[(size_t)w * Np + n] = p;
            }
        }
        __syncthreads();
        // rho_i^G += D_i^T lambda (E_i = [0, D_i]): the four row quarters added in order
        for (int n = tid; n < cols; n += TC_THREADS) {
            const int t = n / nG, k = n - t * nG;
            if (!s_run[t]) continue;
            const int wh = n >= nhalf ? 4 : 0;
            const double v = ((red[(size_t)(wh + 0) * Np + n] + red[(size_t)(wh + 1) * Np + n]) +
                              red[(size_t)(wh + 2) * Np + n]) + red[(size_t)(wh + 3) * Np + n];
            P.blk[(size_t)(b0 + t) * P.blk_stride + S.blk + BL.rho + nO + k] += v;
        }
        __syncthreads();
        for (int t = tid; t < TB; t += TC_THREADS) {
            if (!s_run[t]) continue;
            double* blk = P.blk + (size_t)(b0 + t) * P.blk_stride;
            double ph = 0.0;
            for (int jj = 0; jj < ni; ++jj) ph += blk[S.blk + BL.rho + jj] * blk[S.blk + BL.rho + jj];
            blk[S.phio] = ph;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_MAXN));
}

}  // namespace

// Dynamic shared memory of k_dgemm_tc for Np columns: two stages of the Q chunk (hi, lo) and the P_G chunk
// (hi, lo); the epilogue reuses them for TB x n_C multipliers and 8 x Np partial sums.
static size_t dgemm_tc_smem(int Np, int TB, int nC) {
    const size_t stages = 4 * (size_t)TC_ABYTES + 4 * (size_t)Np * TC_KC * 4;
    const size_t epi = ((size_t)TB * nC + 8 * (size_t)Np) * 8;
    return std::max(stages, epi);
}

bool ddnm_dgemm_tc_ok(const ddnm_ctx* ctx) {
    return ctx->precision == DDNM_MIXED && ctx->d_Qtc && ctx->n_C <= TC_M && ctx->max_nG <= 16;
}

cudaError_t ddnm_launch_dgemm_tc(ddnm_ctx* ctx, const ProbDev& P, int B, cudaStream_t st) {
    const int nG = std::max(1, ctx->max_nG);
    const int TB = std::max(1, std::min(std::min(B, 64), TC_MAXN / nG));
    const int Np = std::min(TC_MAXN, (TB * nG + 15) / 16 * 16);
    const size_t smem = dgemm_tc_smem(Np, TB, P.n_C);
    static thread_local int attr_dev = -1;
    if (attr_dev != ctx->device) {
        const cudaError_t e = cudaFuncSetAttribute(k_dgemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)dgemm_tc_smem(TC_MAXN, 64, MAX_NC));
        if (e != cudaSuccess) return e;
        attr_dev = ctx->device;
    }
    k_dgemm_tc<<<dim3(P.n_sub, (B + TB - 1) / TB), TC_THREADS, smem, st>>>(P, B, TB, Np);
    return cudaGetLastError();
}

// Q_i of every subdomain split into TF32 hi and lo parts in k_dgemm_tc's shared-memory order: per subdomain,
// h_G padded to a multiple of 32 (S.hGp), chunks of 32 hidden units, each [16 row groups][8 K blocks][8 rows]
// [4 hidden units] floats for hi, then the same for lo.  Qt: h_G x qld doubles (Q_i^T).
static float tf32_host(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u = (u + 0x1000u) & 0xFFFFE000u;               // round to nearest, ties away from zero, on the dropped bits
    float y;
    std::memcpy(&y, &u, 4);
    return y;
}

void ddnm_tile_q_tc(std::vector<float>& out, const double* Qt, int hG, int qld, int nC, long long& off, int& hGp) {
    hGp = (hG + TC_KC - 1) / TC_KC * TC_KC;
    off = (long long)out.size();
    out.resize(out.size() + (size_t)2 * hGp * TC_M, 0.f);
    float* hi = out.data() + off;
    float* lo = hi + (size_t)hGp * TC_M;
    for (int h = 0; h < hG; ++h)
        for (int c = 0; c < nC; ++c) {
            const double q = Qt[(size_t)h * qld + c];
            const float qh = tf32_host((float)q);
            const float ql = tf32_host((float)(q - (double)qh));
            const int ch = h / TC_KC, kk = h % TC_KC;
            const size_t idx = (size_t)ch * TC_M * TC_KC + (size_t)((c >> 3) * (TC_KC / 4) + (kk >> 2)) * 32 +
                               (c & 7) * 4 + (kk & 3);
            hi[idx] = qh;
            lo[idx] = ql;
        }
}
