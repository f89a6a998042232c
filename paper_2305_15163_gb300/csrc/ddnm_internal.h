// Internal layout shared by the host set-up (ddnm_host.cpp) and the kernels
// (ddnm_kernels.cu).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace ddnm {

constexpr int MAX_NI = 16;     // n_i^O + n_i^G per subdomain
constexpr int MAX_NG = 8;      // n_i^G
constexpr int MAX_K = 64;      // ELL slots of a decoder output row
constexpr int MAX_NC = 128;    // weak constraints
constexpr int EVAL_THREADS = 256;
constexpr int STEP_THREADS = 128;
constexpr int CON_THREADS = 256;

// HR stencil operand codes: (kind << 28) | index
constexpr int OP_SHIFT = 28;
constexpr int OP_MASK = (1 << OP_SHIFT) - 1;
enum { OP_INTERIOR = 0, OP_INTERFACE = 1, OP_BOUNDARY = 2 };
constexpr int HR_INTS = 7;     // comp, then operands: centre, E, W, N, S (same comp), other comp at centre

// per-instance solver state
enum { MODE_INIT0 = 0, MODE_INIT1 = 1, MODE_LS = 2 };
constexpr int ST_RUNNING = -1;
enum { I_STATUS = 0, I_MODE, I_ITERS, I_NBT, I_FLAGS, I_NEVALS, I_KKTFAIL, I_PAD, INST_INTS };
enum { D_PHI0 = 0, D_ALPHA, D_PHI, D_ALPHA_LAST, INST_DBLS };

// One subdomain: latent sizes, HR rows, subnet layout, offsets into the pools.
struct SubDev {
    int nO, nG, ni, xoff;          // latent dims and offset of xh_i in xh
    int NB, hr_off;                // collocation rows, offset into the HR table
    int hO, mO;                    // interior subnet: hidden units |I_h|, needed outputs |I_o|
    int hG, NG;                    // interface subnet: hidden units, outputs (all N^G)
    int K;                         // ELL slots per output row
    int actO, actG;
    int goff;                      // offset of this subdomain's interface outputs in the concatenation
    int smem_bytes;                // dynamic shared memory the evaluation of this subdomain needs
    long long w1O, b1O, w2O, outO; // interior subnet in the value pool (outO: scale[mO], offset[mO])
    long long colO;                // interior subnet ELL columns (compacted to I_h) in the int pool
    long long w1G, b1G, w2G, outG; // interface subnet
    long long colG;
    long long M;                   // M_i = C A_i stored N^G x n_C (row = interface output), value pool
    // per-instance block (doubles) of this subdomain
    int blk;                       // offset of the block
    // full (not subnet) decoders for reconstruction
    int NO_full, wO_full, wG_full;
    long long fw1O, fb1O, fw2O, foutO, fcolO;
    long long fw1G, fb1G, fw2G, foutG, fcolG;
    long long own;                 // offset into the owned-variable table (int pool): NO_full + NG entries, 1 = owned
    long long ids;                 // global variable ids of interior then interface outputs (int pool)
};

// per-subdomain block layout (doubles) inside an instance's block area
struct BlkLayout {
    int H, rho, D, L, t, W, S, u, phi, flag, size;
};

__host__ __device__ inline BlkLayout blk_layout(int ni, int nG, int nC) {
    BlkLayout b;
    int o = 0;
    b.H = o; o += ni * ni;
    b.rho = o; o += ni;
    b.D = o; o += nC * nG;
    b.L = o; o += ni * ni;
    b.t = o; o += ni;
    b.W = o; o += nG * nC;
    b.S = o; o += nC * nC;
    b.u = o; o += nC;
    b.phi = o; o += 1;
    b.flag = o; o += 1;
    b.size = o;
    return b;
}

struct ProbDev {
    int n_sub, n_D, n_C, N_A, sum_NG, sum_NB, n_bnd, N_x;
    int nx, ny;
    double hx, hy, nu, bx0, by0;
    double tol, c1, beta;
    int max_iter, max_bt;
    int blk_stride;                // doubles per instance of the block area
    const SubDev* sub;
    const void* vpool;             // decoder values and M_i, float (MIXED) or double (FP64)
    const int* ipool;
    const int* hr;                 // HR_INTS per collocation row, all subdomains
    const int* con_lo;             // flat interface index (goff + local) of the +1 side of each constraint row
    const int* con_hi;             // ... of the -1 side
    const double* C;               // n_C x N_A
    const int* bnd_ij;             // n_bnd x 2 grid indices of the Dirichlet points the stencils touch
    // workspace (B instances)
    double* mu;
    double* x;
    double* lam;
    double* xt;
    double* lamt;
    double* s;
    double* slam;
    double* Atil;
    double* dst;                   // INST_DBLS per instance
    int* ist;                      // INST_INTS per instance
    double* bnd;                   // B x n_bnd x 2 (u, v)
    void* gG;                      // B x sum_NG interface outputs (value type)
    double* blk;                   // B x blk_stride
    double* r_hr;                  // optional output B x sum_NB
    int* active;                   // count of running instances after a step pass
};

// Shared-memory carve-out (bytes) of one subdomain evaluation; tsize = sizeof(value type).
struct EvalSmem {
    int sx, sO, PO, sG, PG, yO, JO, yG, JG, Rr, red;      // value-type arrays
    int dH, drho, dD, dL, dt, dW, dlam;                    // double arrays
    int bytes;
};

__host__ __device__ inline int align16(int x) { return (x + 15) & ~15; }

__host__ __device__ inline EvalSmem eval_smem(const SubDev& s, int nC, int tsize) {
    EvalSmem e;
    int o = 0;
    e.sx = o; o = align16(o + MAX_NI * tsize);
    e.sO = o; o = align16(o + s.hO * tsize);
    e.PO = o; o = align16(o + s.hO * s.nO * tsize);
    e.sG = o; o = align16(o + s.hG * tsize);
    e.PG = o; o = align16(o + s.hG * s.nG * tsize);
    e.yO = o; o = align16(o + s.mO * tsize);
    e.JO = o; o = align16(o + s.mO * s.nO * tsize);
    e.yG = o; o = align16(o + s.NG * tsize);
    e.JG = o; o = align16(o + s.NG * s.nG * tsize);
    e.Rr = o; o = align16(o + s.NB * (s.ni + 1) * tsize);
    e.red = o; o = align16(o + EVAL_THREADS * tsize);
    e.dH = o; o = align16(o + s.ni * s.ni * 8);
    e.drho = o; o = align16(o + s.ni * 8);
    e.dD = o; o = align16(o + nC * s.nG * 8);
    e.dL = o; o = align16(o + s.ni * s.ni * 8);
    e.dt = o; o = align16(o + s.ni * 8);
    e.dW = o; o = align16(o + s.nG * nC * 8);
    e.dlam = o; o = align16(o + nC * 8);
    e.bytes = o;
    return e;
}

}  // namespace ddnm
