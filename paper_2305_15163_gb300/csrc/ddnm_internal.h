// Internal layout shared by the host set-up (ddnm_host.cpp) and the kernels
// (ddnm_kernels.cu).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace ddnm {

constexpr int MAX_NI = 16;     // n_i^O + n_i^G per subdomain
constexpr int MAX_TRI = MAX_NI * (MAX_NI - 1) / 2;   // entries of the largest trailing triangle of an H_i
constexpr int MAX_NG = 11;     // n_i^G (round4(n_i^G + 1) <= 12: the interface width classes of the evaluation)
constexpr int NG_SMALL = 8;    // the factorisation variant register-sized for n_i^G <= 8
constexpr int MAX_K = 64;      // ELL slots of a decoder output row
constexpr int MAX_NC = 128;    // weak constraints
constexpr int MAX_SUB = 256;   // subdomains
constexpr int MAX_NR = 64;     // rows of a gappy-POD projector (Z_i Phi_i^r)^+
// threads of one evaluation group: eval_threads(...) below
constexpr int STEP_THREADS = 256;
constexpr int CON_THREADS = 256;
constexpr int CON_SPLIT = 512; // default constraint rows per constraint CTA (the N_A axis is split)
constexpr int CON_BLOCK = 512;  // constraint rows of one canonical partial of Atil (fixes the summation order)
constexpr int MIN_CON_SPLIT = CON_BLOCK, MAX_CON_SPLIT = 4 * CON_BLOCK;
// double-float Atil of the mixed path (k_atil_df): constraint rows staged per chunk, rows between the FP64 folds
// of a double-float sum, constraint rows per slice (one Atil partial per slice and instance)
constexpr int ATIL_KC = 32, ATIL_FOLD = 64, ATIL_KS = MAX_CON_SPLIT;
constexpr int DDNM_TC_TIMEOUT = 1;   // value of ProbDev::err after a k_dgemm_tc wait ran out
constexpr int MAX_CHAINS = 64; // instance groups iterating concurrently inside the solve graph
constexpr int PASSES_PER_BODY = 2;   // SQP passes per turn of an instance group's device-side loop
constexpr int MAX_CLASSES = 12; // width classes (RO, RG) of the evaluation kernel
constexpr int HR_CHUNK = 128;  // largest collocation rows per evaluation chunk (the set-up may choose fewer)

// HR stencil operand codes: (kind << 28) | index
constexpr int OP_SHIFT = 28;
constexpr int OP_MASK = (1 << OP_SHIFT) - 1;
enum { OP_INTERIOR = 0, OP_INTERFACE = 1, OP_BOUNDARY = 2 };
constexpr int HR_INTS = 7;     // comp, then operands: centre, E, W, N, S (same comp), other comp at centre

// per-instance solver state
enum { MODE_INIT0 = 0, MODE_INIT1 = 1, MODE_LS = 2 };
constexpr int ST_RUNNING = -1;
enum { I_STATUS = 0, I_MODE, I_ITERS, I_NBT, I_FLAGS, I_NEVALS, I_XTMODE, I_PAD, INST_INTS };
constexpr int DG_THREADS = 256;    // k_dgemm
constexpr int DG_KT = 32;          // interface hidden units per staged chunk of k_dgemm
constexpr int KKT_THREADS = 512;   // k_kkt: one CTA per instance
constexpr int FAC_WARPS = 4;       // factorisation CTAs of k_constraint: warps with a pair of subdomains each
constexpr int SS_ROWS_DBL = 3072;  // staged W rows (doubles) per Schur-sum chunk, each for W, D_G^{-1} W and u
constexpr int FAC_SHARE_SMEM = 32768;   // largest staging (bytes) of a factorisation CTA's Schur-sum share
constexpr int KKT_DW = 4;          // k_kkt: warps that judge the trial point while the others form the Schur sums
// how the next evaluation forms its trial point xt (ist[I_XTMODE]): unchanged (xt = x), a new SQP step
// (each subdomain back-substitutes s_i from s_lambda, then xt = x + s), or a backtrack (xt = x + alpha s)
enum { XT_KEEP = 0, XT_NEWSTEP = 1, XT_BACKTRACK = 2 };
enum { D_PHI0 = 0, D_ALPHA, D_PHI, D_ALPHA_LAST, INST_DBLS };

__host__ __device__ inline int round4(int x) { return (x + 3) & ~3; }

// register budget of the evaluation kernel, as the threads per SM it is sized for: 1024 for the narrow FP32
// records, 768 or 512 for the wider ones; FP64 records take twice the registers
__host__ __device__ constexpr int eval_reg_threads(int tsize, int ro, int rg) {
    return tsize == 8 ? 512 : (ro + rg <= 12 ? 1024 : (ro + rg <= 20 ? 768 : 512));
}
// threads of one (instance, subdomain) evaluation.  256 for every class: 512-thread CTAs of the narrow FP32
// class (two per SM at the same budget) cut an evaluation's latency by a third on the 128 x 128 / 4 x 4
// workload but lowered the SM's throughput by a quarter (half as many evaluations resident), a loss at 64
// instances per batch.
__host__ __device__ constexpr int eval_threads(int, int, int) { return 256; }
// (instance, subdomain) evaluations per SM within the register budget
__host__ __device__ constexpr int eval_ctas_by_regs(int tsize, int ro, int rg) {
    return eval_reg_threads(tsize, ro, rg) / eval_threads(tsize, ro, rg);
}

// 32 consecutive output rows of a decoder subnet whose mask columns (in I_h numbering) all lie in the
// window [c0, c0 + tw) (tw a multiple of 4, c0 + tw <= round4(|I_h|)): values dense over the window, zero
// off the mask, stored [tw / 4][32 rows][4 columns] in the value pool at voff.
struct TileDev {
    int c0, tw;
    long long voff;
};

// One chunk of a subdomain's collocation rows with the interior decoder outputs it needs.
struct ChunkDev {
    int q0, nq;                    // first collocation row (subdomain-local) and row count
    int m;                         // interior outputs needed by these rows (chunk-local slots 0..m-1)
    int ntiles;                    // dense-window tiles of these outputs (0: the ELL table is used)
    long long col;                 // int pool: Kp x m ELL columns (slot-major), renumbered into I_h
    long long val;                 // value pool: Kp x m ELL values (slot-major)
    long long so;                  // value pool: scale[m], offset[m]
    int tile0, pad;                // first tile in the tile table
};

// One subdomain: latent sizes, HR rows, subnet layout, offsets into the pools.
struct SubDev {
    int nO, nG, ni, xoff;          // latent dims and offset of xh_i in xh
    int NB, hr_off;                // collocation rows, offset into the HR table (rows; the table is HR_INTS x N_B)
    int hO, hG, NG;                // hidden units of the interior / interface subnets, interface outputs
    int Kp;                        // ELL slots per row, padded to a multiple of 8 (padding: column 0, value 0)
    int actO, actG;
    int goff;                      // offset of this subdomain's interface outputs in the concatenation
    int n_chunks, chunk0, mmax;    // HR chunks: count, first index in the chunk table, max outputs per chunk
    int smem_bytes;                // dynamic shared memory the evaluation of this subdomain needs
    int blk;                       // offset of this subdomain's block in an instance's block area
    int phio;                      // offset of ||rho_i||^2 in an instance's block area (a header of n_sub doubles)
    long long w1O, b1O;            // interior subnet hidden layer: W1~ (hO x round4(nO)), b1~ (hO)
    long long w1G, b1G;            // interface subnet hidden layer: W1~ (hG x round4(nG)), b1~ (hG)
    long long colG, valG, soG;     // interface outputs, all rows: ELL slot-major (Kp x NG), scale/offset
    int tileG0, ntilesG;           // dense-window tiles of the interface outputs (0 tiles: ELL)
    int NGn, hr_chunk;             // interface outputs the stencils use; collocation rows per chunk
    long long colGn, valGn, soGn;  // those outputs: ELL slot-major (Kp x NGn), scale/offset
    long long Qt;                  // value pool: Q_i^T = (C A_i diag(scale) W2~)^T, h_G x n_C
    int nr, pad_nr;                // gappy-POD HR: rows of (Z_i Phi_i^r)^+ (0: collocation, B_i = Z_i)
    long long gp;                  // value pool: (Z_i Phi_i^r)^+, nr x N_B row-major
    long long ahat;                // SRPC: offset of A^_i (n_C x n_i^G, FP64) in P.Ahat
    long long qtc;                 // mixed path: Q_i split into TF32 hi / lo in k_dgemm_tc's order (floats into
    int hGp, pad_tc;               // P.Qtc); h_G rounded up to the tensor-core K chunk
    long long pgoff;               // offset of this subdomain's P_G (h_G x n^G) in an instance's P_G area
    // full (not subnet) decoders for reconstruction
    int NO_full, wO_full, wG_full, K;
    long long fw1O, fb1O, fw2O, foutO, fcolO;
    long long fw1G, fb1G, fw2G, foutG, fcolG;
    long long own;                 // int pool: NO_full + NG flags, 1 = variable owned by this subdomain
    long long ids;                 // int pool: global ids of interior then interface outputs
};

// per-subdomain block layout (doubles) inside an instance's block area
struct BlkLayout {
    int H, rho, D, L, rinv, t, W, u, G, flag, size;
};

// per-subdomain flag values written by the factorisation
constexpr double FLAG_PD = 0.0;          // H_i positive definite: L, rinv, t, W, u valid
constexpr double FLAG_OMEGA_FAIL = 1.0;  // H_i^{OO} not positive definite: not solvable by this route
constexpr double FLAG_GAMMA_SING = 2.0;  // H_i^{OO} PD but H_i not: L, rinv (first n^O columns), t (t_O,
                                         // then rho_G - L_GO t_O) and G = H_GG - L_GO D_O L_GO^T valid
constexpr int MAX_MF = 32;               // interface unknowns of such subdomains handled per instance

__host__ __device__ inline BlkLayout blk_layout(int ni, int nG, int nC) {
    BlkLayout b;
    int o = 0;
    b.H = o; o += ni * ni;
    b.rho = o; o += ni;
    b.D = o; o += nC * nG;
    b.L = o; o += ni * ni;
    b.rinv = o; o += ni;           // 1 / D_jj of H_i = L D L^T (L unit lower, stored below the diagonal)
    b.t = o; o += ni;
    b.W = o; o += nG * nC;
    b.u = o; o += nC;
    b.G = o; o += nG * nG;         // Schur complement of H^{OO} in H_i (used when H_i is singular)
    b.flag = o; o += 1;
    b.size = o;
    return b;
}

struct ProbDev {
    int n_sub, n_D, n_C, N_A, sum_NG, sum_NB, n_bnd, N_x;
    int nx, ny;
    int fac_stride;                // factorisation scratch doubles per warp: max_i n_i^2 + 4 n_i + (n_i^G)^2
    int d_gemm;                    // 1: D_i by the batched k_dgemm; 0: inside the evaluation
    int n_split;                   // constraint CTAs per instance (ceil(N_A / con_split))
    int con_split;                 // constraint rows per constraint CTA
    double hx, hy, nu, bx0, by0;
    double cst[4];                 // stencil constants 1/(2h_x), 1/(2h_y), nu/h_x^2, nu/h_y^2 (from the host)
    float cstf[4];                 // the same in FP32
    double tol, c1, beta;
    double piv_eps;                // block pivots d_j <= piv_eps max_k H_kk count as zero (rank test)
    int max_iter, max_bt;
    double step_tol;               // mixed path: stop on a first trial whose step is below step_tol of the iterate
    int blk_stride;                // doubles per instance of the block area
    const SubDev* sub;
    const ChunkDev* chunk;
    const TileDev* tiles;
    const void* vpool;             // decoder values and M_i, float (MIXED) or double (FP64)
    const int* ipool;
    const int* hr;                 // per subdomain HR_INTS x N_B (operand-major), all subdomains
    const int* con_lo;             // flat interface index (goff + local) of the +1 side of each constraint row
    const int* con_hi;             // ... of the -1 side
    const double* C;               // n_C x N_A
    const float* Cthi;             // N_A x ldct: C transposed and split, C[c][l] = Cthi[l][c] + Ctlo[l][c] (to
    const float* Ctlo;             // 2^-48), zero for c >= n_C; mixed path only
    int ldct;                      // row stride of Cthi / Ctlo: n_C rounded up to 32, 64 or a multiple of 128
    const float* Qtc;              // mixed path: every Q_i split and tiled for k_dgemm_tc (SubDev::qtc)
    int* err;                      // device error word (DDNM_TC_TIMEOUT: a bounded tensor-core wait ran out)
    int srpc;                      // SRPC formulation: D_i = A^_i constant, Atil = sum_i A^_i xh_i^G
    const double* Ahat;            // SRPC: the A^_i (SubDev::ahat)
    int atil_df;                   // 1: Atil by k_atil_df (instance tiles, double-float); 0: FP64 slices
    int qld;                       // row stride of every Q_i^T in the value pool: round4(n_C)
    const int* bnd_ij;             // n_bnd x 2 grid indices of the Dirichlet points the stencils touch
    // workspace (B instances)
    double* mu;
    double* x;
    double* lam;
    double* xt;
    double* lamt;
    double* s;
    double* slam;
    double* Atil;                  // B x n_split x n_C partial sums of C * jump
    double* Spart;                 // B x nfc x (n_C (n_C + 1) / 2 + n_C): per factorisation CTA, the sums over
                                   // its PD subdomains of W_i^T D_G,i^{-1} W_i (lower triangle, row by row), u_i;
                                   // null when the border is too wide for that (the KKT step sums the blocks)
    int ss_rows;                   // rows of W staged per Schur-sum chunk of the KKT step
    int n_ss_chunks;               // Schur-sum chunks: subdomains [ss_chunk[k], ss_chunk[k + 1])
    const int* ss_chunk;
    int nfc;                       // factorisation CTAs per instance: ceil(n_sub / (2 FAC_WARPS))
    int fac_rows;                  // largest sum of n_i^G over the subdomains of one factorisation CTA
    double* dst;                   // INST_DBLS per instance
    int* ist;                      // INST_INTS per instance
    void* bnd;                     // B x n_bnd x 2 (u, v) Dirichlet data, value type
    void* gG;                      // B x sum_NG interface outputs (value type)
    void* PG;                      // B x pg_stride: per subdomain sigma'(z_h) W1~[h, :], value type
    long long pg_stride;
    double* blk;                   // B x blk_stride
    double* r_hr;                  // optional output B x sum_NB
    int* active;                   // count of running instances after a step pass
    int* pass;                     // loop passes of the solve graph's instance group
    int* ctr;                      // MAX_CLASSES work counters of the persistent evaluation
    int* arrive;                   // step CTAs of the pass that have finished (the last one runs the loop control)
};

// Control area at the end of the workspace: per instance group, the running count, the loop passes, the
// persistent evaluation's work counters and the step kernel's arrival count.
constexpr int CTL_INTS = MAX_CHAINS * (3 + MAX_CLASSES);

// Shared-memory carve-out (bytes) of one subdomain evaluation; tsize = sizeof(value type).
struct EvalSmem {
    int Rt, hp, hpair;
    int sx, hidO, hidG, outGn, outO, Rr, red;  // value-type arrays
    int dH, drho, dt, dD;                      // double arrays
    int bytes;
};

__host__ __device__ inline int align16(int x) { return (x + 15) & ~15; }

__host__ __device__ inline EvalSmem eval_smem(const SubDev& s, int nC, int tsize) {
    EvalSmem e;
    const int rO = round4(s.nO + 1), rG = round4(s.nG + 1);
    int o = 0;
    e.sx = o; o = align16(o + MAX_NI * tsize);
    // [sigma, sigma' W1 row] per hidden unit (+ zero rows): the interface records during the interface phase,
    // then the interior records in the same place for the chunk loop
    e.hidO = e.hidG = o;
    const int recO = round4(s.hO) * rO, recG = round4(s.hG) * rG;
    o = align16(o + (recO > recG ? recO : recG) * tsize);
    e.outGn = o; o = align16(o + s.NGn * rG * tsize);        // [y, Jacobian row] per interface output the stencils use
    // the chunk loop's [y, Jacobian row] per needed interior output and [R row, r] per collocation row; the
    // D_i partials per thread group of the interface phase in the same place
    const int o_chunk = o;
    e.outO = o; o = align16(o + s.mmax * rO * tsize);
    e.Rr = o; o = align16(o + s.hr_chunk * (s.ni + 1) * tsize);
    e.red = o_chunk;
    const int o_red = align16(o_chunk + (eval_threads(tsize, rO, rG) / nC) * nC * s.nG * tsize);
    o = o > o_red ? o : o_red;
    e.Rt = o; o = align16(o + s.nr * (s.ni + 1) * tsize);  // gappy POD: (Z Phi)^+ [R, r] over the rows
    e.hp = o; o = align16(o + (eval_threads(tsize, rO, rG) / 32) * (s.ni * (s.ni + 3) / 2) * tsize);  // H_i, R_i^T r partials per warp
    e.hpair = o; o = align16(o + (s.ni * (s.ni + 3) / 2) * 4);    // (a, c) of each of those entries
    e.dH = o; o = align16(o + s.ni * s.ni * 8);
    e.drho = o; o = align16(o + s.ni * 8);
    e.dt = o; o = align16(o + s.ni * 8);
    e.dD = o; o = align16(o + nC * s.nG * 8);
    e.bytes = o;
    return e;
}

}  // namespace ddnm
