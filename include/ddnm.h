/*
 * ddnm.h -- C ABI of the GB300 (sm_103a) library for the online solve of the
 * domain-decomposition nonlinear-manifold ROM with hyper-reduction of
 * Diaz, Choi & Heinkenschloss, arXiv 2305.15163 ("the paper").
 *
 * The library solves, for a batch of parameters mu = (a, lambda), the WFPC
 * DD-LSPG-ROM of Sec. 3.1, Eq. (dd_lspg_NLP):
 *
 *     min  1/2 sum_i || Z_i r_i( g_i^O(xh_i^O), g_i^G(xh_i^G) ) ||^2
 *     s.t. sum_i C A_i g_i^G(xh_i^G) = 0
 *
 * on the steady 2D Burgers problem of Sec. 7.1 (centred finite differences,
 * Dirichlet data from the exact solution Eq. (burgers_pde_exact_solution)),
 * with the Lagrange-Gauss-Newton SQP of Sec. 4.1 (KKT system Eq. (sqp_system),
 * Gauss-Newton Hessian Eq. (gauss_newton_hessian), update Eq. (sqp_update)).
 *
 * Conventions shared by every call:
 *  - Grid: nx x ny interior nodes of the box [box0,box1] x [box2,box3],
 *    x_i = box0 + i h_x, h_x = (box1-box0)/(nx+1), i = 1..nx (same in y).
 *  - State ordering x = [u; v], each block x-fastest: u at node (i,j) has
 *    global id (j-1)*nx + (i-1), v at that node has id nx*ny + that.
 *  - Subdomains are boxes of nodes cut at breakpoints xb[0..kx], yb[0..ky]
 *    (0 = xb[0] < ... < xb[kx] = nx); subdomain s = sy*kx + sx.
 *  - Residual rows of subdomain s (Sec. 2, P_s^r): u rows of its owned nodes in
 *    ascending node order, then the v rows; HR rows are indices into that list.
 *  - Interior / interface states of s (Sec. 2, P_s^O, P_s^G): global variable
 *    ids in ascending order.  Interface = variables entering the residual rows
 *    of s and of at least one other subdomain; interior = the rest.
 *  - Compatibility rows (Eq. compatibility_conditions_mat): for every shared
 *    variable (ascending id), with S = sorted subdomains sharing it, the rows
 *    x_{S0} - x_{S1} = 0, x_{S1} - x_{S2} = 0, ...; N_A rows in total.
 *  - Latent vector xh = [xh_0^O; xh_0^G; xh_1^O; ...] (Eq. sqp_notation), n_D
 *    entries; multipliers lambda have n_C entries; the KKT right-hand side is
 *    F = [rho_0; ...; rho_{n-1}; Atil] (n_D + n_C), rho_i of
 *    Eq. (optimality_residuals_GN), Atil = sum_i C A_i g_i^G.
 *  - All arrays are dense, row-major, FP64 unless stated.
 *
 * Ownership: every call copies what it needs from the caller's arrays; the
 * caller keeps ownership and may free them on return (for mem_kind
 * DDNM_MEM_DEVICE, once the stream has passed the call).
 *
 * Errors: every int-returning call returns DDNM_OK (0) or a negative DDNM_E_*
 * code; ddnm_last_error(ctx) then holds a one-line message.  A solve that does
 * not converge is not an error: it is a per-instance status in ddnm_stats.
 * No call falls back to a CPU implementation.  ddnm_setup and the query calls
 * are host bookkeeping and work without a GPU; the first call that computes
 * (solve, residual, linearize) uploads the tables to the device and fails with
 * DDNM_E_CUDA when no usable CUDA device is present.
 *
 * Threading: one context per host thread at a time; calls on one context are
 * not thread-safe.  Work is queued on the caller's stream (NULL = legacy
 * default stream).  With DDNM_MEM_HOST the call returns after the results are
 * in the caller's host arrays; with DDNM_MEM_DEVICE it returns once the work is
 * queued and the output pointers are device pointers written by that stream.
 */
#ifndef DDNM_H
#define DDNM_H

#ifdef __cplusplus
extern "C" {
#endif

#define DDNM_OK 0
#define DDNM_E_INVALID (-1)      /* bad argument or size mismatch */
#define DDNM_E_STATE (-2)        /* call made in the wrong order (e.g. solve before all decoders are loaded) */
#define DDNM_E_CUDA (-3)         /* CUDA runtime error, or no usable device */
#define DDNM_E_NOMEM (-4)        /* device or host allocation failed */
#define DDNM_E_UNSUPPORTED (-5)  /* sizes beyond what the kernels are built for */

enum { DDNM_FP64 = 0, DDNM_MIXED = 1 };                       /* evaluation precision */
enum { DDNM_ACT_SWISH = 0, DDNM_ACT_SIGMOID = 1, DDNM_ACT_IDENTITY = 2 };
enum { DDNM_MEM_HOST = 0, DDNM_MEM_DEVICE = 1 };
enum { DDNM_DECODER_INTERIOR = 0, DDNM_DECODER_INTERFACE = 1 };

/* per-instance termination status (ddnm_stats.status) */
enum {
    DDNM_CONVERGED = 0,  /* ||F||_2 < tol at an accepted iterate */
    DDNM_MAX_ITER = 1,   /* max_iter accepted steps taken without convergence */
    DDNM_NONFINITE = 2,  /* the merit became NaN or Inf at an accepted iterate */
    DDNM_KKT_FAIL = 3    /* KKT system not solvable by the Schur route (Lemma 1 fails) */
};
/* per-instance flags (ddnm_stats.flags, bit mask) */
#define DDNM_FLAG_LS_FAIL 1   /* some line search took its last trial without passing Armijo */
#define DDNM_FLAG_WS_FALLBACK 2 /* learned warm start enabled, but the default start had the smaller merit */
#define DDNM_FLAG_STEP 4      /* stopped on a step below options.step_tol (mixed path) */

/* Problem statement (Sec. 2, 3.1, 7.1). */
typedef struct ddnm_problem {
    int nx, ny;             /* interior grid nodes */
    double nu;              /* viscosity */
    double box[4];          /* x0, x1, y0, y1 of the domain */
    int kx, ky;             /* subdomains in x and y */
    const int* xb;          /* kx+1 node breakpoints, 0 .. nx */
    const int* yb;          /* ky+1 node breakpoints, 0 .. ny */
    const int* n_omega;     /* kx*ky interior latent dims n_i^O (1..16) */
    const int* n_gamma;     /* kx*ky interface latent dims n_i^G (1..11, n_i^O + n_i^G <= 16) */
    const int* hr_count;    /* kx*ky collocation row counts N_i^B (>= n_i^O + n_i^G) */
    const int* hr_rows;     /* sum(hr_count) local residual-row ids, sorted ascending per subdomain */
    int n_c;                /* rows of the test matrix C (weak constraints), 1..128 */
    int precision;          /* DDNM_FP64 or DDNM_MIXED (FP32 evaluation, FP64 KKT/merit) */
    int device;             /* CUDA device ordinal */
} ddnm_problem;

/* SQP options (Sec. 4.1, 7.1).  Defaults: tol 1e-4, max_iter 15, c1 1e-4, beta 0.5, 20 backtracks. */
typedef struct ddnm_options {
    double tol;             /* stop when ||F||_2 < tol */
    int max_iter;           /* accepted SQP steps */
    double armijo_c1;       /* accept alpha when phi(alpha)^2 <= (1 - 2 c1 alpha) phi(0)^2 */
    double beta;            /* backtracking factor */
    int max_backtracks;     /* after this many halvings the last trial is taken (flag LS_FAIL) */
    double step_tol;        /* mixed path only (0 = off, the default: the paper's rule alone).  With the FP32
                               evaluation ||F||_2 stalls near the solution at the rounding level of rho_i, where
                               the Armijo test compares rounding noise and backtracks.  With step_tol > 0, the
                               first trial of a step with ||s||_2 <= step_tol ||xh||_2 (the Gauss-Newton step of
                               the latent coordinates) is accepted and the instance stops there (status
                               CONVERGED, flag DDNM_FLAG_STEP).  Ignored by the FP64 path; 0 <= step_tol < 1. */
} ddnm_options;

/* One sparse-masked shallow decoder g(x) = offset + scale o (W2 sigma(W1 x + b1))
 * (Sec. 5.1 Eq. autoencoder_architecture b/d, de-normalisation layer Sec. 7.3).
 * W2 in ELL form: row r has its nonzero columns cols[r*K .. r*K+K-1] (ascending,
 * -1 padding at the end) with values vals[...].  Host FP64 arrays, copied. */
typedef struct ddnm_decoder {
    int N;                  /* outputs (must equal N_i^O or N_i^G) */
    int w;                  /* width (hidden units) */
    int n;                  /* latent dim (must equal n_i^O or n_i^G) */
    int act;                /* DDNM_ACT_* */
    int K;                  /* ELL slots per row (<= 64) */
    const double* W1;       /* w x n */
    const double* b1;       /* w */
    const int* cols;        /* N x K */
    const double* vals;     /* N x K */
    const double* scale;    /* N (NULL = ones) */
    const double* offset;   /* N (NULL = zeros) */
} ddnm_decoder;

typedef struct ddnm_sizes {
    int n_sub;              /* kx*ky */
    int N_x;                /* 2 nx ny */
    int n_D;                /* sum_i n_i^O + n_i^G */
    int n_C;                /* weak constraints */
    int N_A;                /* compatibility rows */
    int sum_hr;             /* sum_i N_i^B */
    int sum_gamma;          /* sum_i N_i^G */
} ddnm_sizes;

typedef struct ddnm_stats {
    int iters;              /* accepted SQP steps */
    int status;             /* DDNM_CONVERGED .. DDNM_KKT_FAIL */
    int flags;              /* DDNM_FLAG_* */
    int n_evals;            /* residual/Jacobian evaluations, line-search trials included */
    double merit;           /* ||F||_2 at the returned iterate */
    double alpha_last;      /* step length of the last accepted step (0 if none) */
} ddnm_stats;

/* Per-kernel device time and launch counts, accumulated while timing is on
 * (ddnm_timing_enable).  Times come from CUDA events recorded on the caller's
 * stream around every launch of that kernel. */
typedef struct ddnm_timing {
    double eval_ms;             /* k_eval: fused decoder / residual / Gauss-Newton blocks */
    double constraint_ms;       /* k_constraint: FP64 weak-constraint residual (and, in a solve, the FP64
                                   per-subdomain L D L^T of the Gauss-Newton blocks in CTAs of its own) */
    double step_ms;             /* k_kkt: merit, Armijo, update; FP64 Schur sums and border solve of the
                                   KKT system */
    long long eval_launches;
    long long constraint_launches;
    long long step_launches;
    long long other_launches;   /* set-up, statistics and reconstruction kernels */
} ddnm_timing;

/* Algorithmic work of ONE evaluation of ONE instance (all subdomains), counted
 * from the sizes of the set-up (subnets, HR rows, constraint rows): what the
 * method must compute, independent of how the kernels do it. */
typedef struct ddnm_work {
    double eval_flops;          /* value-type flops of k_eval: hidden layers, decoder outputs and
                                   Jacobian rows, residual rows and chain rule, H_i and R_i^T r_i, D_i */
    double eval_fp64_flops;     /* FP64 flops of k_eval: rho_i += D_i^T lambda, ||rho_i||^2 */
    double eval_bytes;          /* global bytes of one instance-evaluation on its own: table_bytes +
                                   instance_bytes */
    double constraint_fp64_flops;  /* 2 n_C N_A */
    double step_fp64_flops;     /* per accepted point: per-subdomain L D L^T, t, W, u; the Schur sums
                                   S = sum_i W_i^T D_G^{-1} W_i and sum_i u_i; the n_C L D L^T and solves;
                                   the back-substitution */
    double table_bytes;         /* bytes an evaluation reads that every instance shares: subnet weights, mask
                                   values and columns, scale/offset, Q_i, collocation-row table */
    double instance_bytes;      /* bytes an evaluation reads or writes for one instance: latents, mu,
                                   multipliers, Dirichlet values, interface values, H_i, rho_i, D_i.  The
                                   algorithmic bytes of a launch of B instances: table_bytes + B instance_bytes */
} ddnm_work;

typedef struct ddnm_ctx ddnm_ctx;

/* Build the algebraic DD (Sec. 2: residual/interior/interface sampling, ports,
 * compatibility rows) and the HR stencil tables (Sec. 5.3) on the host.
 * Copies every array of p.  Returns DDNM_E_INVALID for inconsistent sizes,
 * DDNM_E_UNSUPPORTED beyond the limits stated above (or with a single
 * subdomain).  *out is NULL on failure.  Device memory is allocated by the
 * first solve / residual / linearize call on p->device. */
int ddnm_setup(const ddnm_problem* p, ddnm_ctx** out);

/* Free all host and device memory of ctx (NULL is a no-op). */
void ddnm_destroy(ddnm_ctx* ctx);

/* Message of the last failed call on ctx ("" if none); valid until the next call.
 * ddnm_last_error(NULL) gives the message of the last failed ddnm_setup on this thread. */
const char* ddnm_last_error(const ddnm_ctx* ctx);

/* Sizes of the decomposition. */
int ddnm_get_sizes(const ddnm_ctx* ctx, ddnm_sizes* out);

/* Subdomain sub: info[6] = {N_r, N^O, N^G, n^O, n^G, N^B}; interior_ids (N^O) and
 * interface_ids (N^G) receive global variable ids if non-NULL. */
int ddnm_get_subdomain(const ddnm_ctx* ctx, int sub, int* info, int* interior_ids, int* interface_ids);

/* Compatibility rows (Eq. compatibility_conditions_mat): for row k, the shared
 * variable row_var[k] and the two subdomains it equates, row_lo[k] (+1) and
 * row_hi[k] (-1).  Arrays of N_A entries; any may be NULL. */
int ddnm_get_constraints(const ddnm_ctx* ctx, int* row_var, int* row_lo, int* row_hi);

/* Gaussian test matrix C of the weak constraint (Sec. 3.1), n_C x N_A, FP64. */
int ddnm_set_test_matrix(ddnm_ctx* ctx, const double* C);

/* Load decoder `kind` (DDNM_DECODER_INTERIOR / _INTERFACE) of subdomain `sub`
 * and build its HR subnet (Sec. 5.4, Eq. subnet) for the outputs the HR
 * stencils (interior) or the constraint (interface, all rows; Sec. 5.3 remark)
 * need.  DDNM_E_INVALID on size mismatch or a column outside [-1, w). */
int ddnm_load_decoders(ddnm_ctx* ctx, int sub, int kind, const ddnm_decoder* d);

/* Gappy-POD hyper-reduction for subdomain `sub` (Sec. 3.1, Eq. dd_lspg_NLP with B_i = (Z_i Phi_i^r)^+ Z_i):
 * proj = (Z_i Phi_i^r)^+, nr x N_i^B row-major, its columns in the order of the subdomain's HR rows given to
 * ddnm_setup (Z_i), Phi_i^r the subdomain's residual basis (nr columns).  The evaluation then forms
 * R_i = proj Z_i dr_i/dxh and r~_i = proj Z_i r_i, H_i = R_i^T R_i and R_i^T r~_i from them.  nr = 0 returns
 * to collocation (B_i = Z_i).  1 <= nr <= min(64, N_i^B); host memory, copied; takes effect at the next
 * compute call.  DDNM_E_INVALID for sizes out of range or non-finite entries. */
int ddnm_set_hr_projection(ddnm_ctx* ctx, int sub, int nr, const double* proj);

/* Offline choice of the gappy-POD sample rows and projectors (Sec. 5.3, greedy-sampling remark) from residual
 * snapshots snaps (n_snap x N_x host array: FOM residuals at Newton iterates, e.g. from ddnm_fom_residual).
 * Per subdomain i: the residual basis Phi_i^r = the leading nr[i] left singular vectors of its rows of the
 * snapshots; n_samples[i] rows chosen greedily (interpolation error of basis vector k for the first nr[i]
 * rows, then the row of largest leverage against the rows taken); the projector (Z_i Phi_i^r)^+.
 *   rows_out  sum_i n_samples[i] ascending local residual-row ids per subdomain, in subdomain order (the
 *             hr_rows of a new ddnm_setup)
 *   proj_out  sum_i nr[i] n_samples[i]: per subdomain the nr[i] x n_samples[i] projector, row-major (for
 *             ddnm_set_hr_projection on that new context)
 * Host computation (no device); 1 <= nr[i] <= min(64, n_snap), nr[i] <= n_samples[i] <= N_i^r. */
int ddnm_hr_select(ddnm_ctx* ctx, int n_snap, const double* snaps, const int* nr, const int* n_samples, int* rows_out,
                   double* proj_out);

/* ---- SRPC formulation (Sec. 3.2, Eq. dd_lspg_NLP_rom_port; Sec. 5.2, Eq. interface_decoder_rom_port_blocks) ----
 * Ports: the interface variables grouped by the set P(j) of subdomains sharing them, in ascending
 * lexicographic order of P(j), each port's variables in ascending global order.  Port j has a decoder g_j^p
 * with n_j^p = max(min(N_j^p - 1, n~), 1) latents (Sec. 7.5); subdomain i's interface latents are its ports'
 * latents stacked in port order, so n_i^G = sum over its ports of n_j^p, and its interface decoder is the
 * block-diagonal assembly of its ports' decoders.  The constraints become linear, sum_i A^_i x^_i^G = 0: for
 * every port, latent component c and consecutive pair s_k < s_{k+1} of P(j), the row x^_{s_k}[c] -
 * x^_{s_{k+1}}[c] (rows by port, then component, then pair); n_A rows in all.  The SQP then has D_i = A^_i and
 * Atil = sum_i A^_i x^_i^G (no test matrix).
 *
 * ddnm_get_ports: the ports of ctx's decomposition under n~ (host bookkeeping, on any context of the same
 * grid and partition): n_ports; when cap >= n_ports, per port its subdomains (port_subs, 4 per port, -1
 * padded), N_j^p and n_j^p; n_gamma[n_sub] the interface latent sizes to pass to ddnm_setup, whose n_c must
 * be n_A = sum_j (|P(j)| - 1) n_j^p. */
int ddnm_get_ports(const ddnm_ctx* ctx, int n_tilde, int cap, int* n_ports, int* port_subs, int* port_N, int* port_n,
                   int* n_gamma);
/* Switch ctx to SRPC under n~: checks n_gamma and n_c against the ports, builds A^_i; every interface decoder is
 * then assembled from port decoders (ddnm_load_port_decoder) and ddnm_set_test_matrix is not needed.
 * DDNM_E_INVALID on a size mismatch (the message gives the expected sizes). */
int ddnm_set_srpc(ddnm_ctx* ctx, int n_tilde);
/* Port decoder g_j^p (N = N_j^p outputs in the port's variable order, n = n_j^p), copied; once all ports of a
 * subdomain are loaded its interface decoder is assembled and loaded. */
int ddnm_load_port_decoder(ddnm_ctx* ctx, int port, const ddnm_decoder* d);
/* A^_i of subdomain `sub` (n_C x n_i^G row-major) of an SRPC context. */
int ddnm_get_port_matrix(const ddnm_ctx* ctx, int sub, double* out);

/* Replace the SQP options. */
int ddnm_set_options(ddnm_ctx* ctx, const ddnm_options* opt);

/* Batched SQP solve (Sec. 4.1) of B instances.
 *   mu      B x 2 (a, lambda)
 *   x0      B x n_D start, or NULL for xh0 = 0
 *   lam0    B x n_C start, or NULL for the least-squares multiplier of
 *           Eq. (optimality_residuals b) at x0 (Sec. 7.2)
 *   x_out   B x n_D, lam_out B x n_C  (either may be NULL)
 *   state_out B x N_x reconstructed state g(xh) taking every variable from its
 *           owning subdomain, or NULL
 *   stats   B entries, or NULL
 * Pointers are host (DDNM_MEM_HOST) or device (DDNM_MEM_DEVICE) memory;
 * stream is a cudaStream_t (NULL = default stream). */
int ddnm_solve_batch(ddnm_ctx* ctx, int B, const double* mu, const double* x0, const double* lam0,
                     double* x_out, double* lam_out, double* state_out, ddnm_stats* stats,
                     int mem_kind, void* stream);

/* Reconstructed states g(xh) of B latent vectors (the state the relative error of Eq. relative_error
 * measures, Sec. 7.1): every variable from its owning subdomain's interior or interface decoder.
 *   x          B x n_D latent coordinates
 *   state_out  B x N_x
 * Host or device memory (mem_kind), queued on stream; with host memory the call returns once the state is
 * copied back. */
int ddnm_reconstruct(ddnm_ctx* ctx, int B, const double* x, double* state_out, int mem_kind, void* stream);

/* One evaluation at (x, lam) without iterating.
 *   F_out      B x (n_D + n_C) KKT right-hand side F (NULL to skip)
 *   r_hr_out   B x sum(N_i^B) collocation residuals Z_i r_i (NULL to skip)
 *   r_full_out B x N_x FOM residual r(g(xh); mu) of the reconstructed state (NULL to skip) */
int ddnm_residual(ddnm_ctx* ctx, int B, const double* mu, const double* x, const double* lam,
                  double* F_out, double* r_hr_out, double* r_full_out, int mem_kind, void* stream);

/* The blocks one evaluation builds (for checking them): per instance and
 * subdomain H_i = R_i^T R_i (n_i x n_i, Eq. gauss_newton_hessian) and
 * D_i = C A_i dg_i^G/dxh (n_C x n_i^G), concatenated over subdomains;
 * Atil (n_C).  Any output may be NULL. */
int ddnm_linearize(ddnm_ctx* ctx, int B, const double* mu, const double* x, const double* lam,
                   double* H_out, double* D_out, double* Atil_out, int mem_kind, void* stream);

/* ddnm_residual without any device allocation.  The paper has no counterpart of
 * this call: it exists for callers that cannot call cudaMalloc -- code running
 * under a device-memory cap or a pool that forbids growth, latency-critical
 * loops where an allocation's implicit device synchronisation is not
 * acceptable, or code that must not allocate after start-up.
 *
 * Computes F = [rho_0; ...; rho_{n-1}; Atil] (B x (n_D + n_C)) at (x, lam) like
 * ddnm_residual's F_out.  mu (B x 2), x (B x n_D), lam (B x n_C, or NULL for
 * lambda = 0) and F_out are DEVICE pointers; the work is queued on `stream`
 * and the call returns without waiting.  Nothing is allocated: the scratch
 * the evaluation needs lives in one static device array of 16 MiB that every
 * GPU loading the library holds until the process exits.
 *  - The decoder and constraint tables must already be on the device: make one
 *    allocating call (ddnm_residual, ddnm_linearize or ddnm_solve_batch) on ctx
 *    first, else DDNM_E_STATE.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.  The address is kept per device and CUDA
 *    context: after the application resets the device (cudaDeviceReset), the
 *    next call is again a first call and looks it up anew.
 *  - mu, x, lam and F_out must be device (or managed) memory of ctx's device;
 *    any other pointer returns DDNM_E_INVALID before anything is queued
 *    (checked with cudaPointerGetAttributes, which allocates nothing).  The
 *    sizes of the arrays cannot be checked here: they must hold the counts
 *    stated above.
 *  - B beyond what fits in 16 MiB (about 210 instances of the 128x128 4x4
 *    workload) returns DDNM_E_UNSUPPORTED with the limit in the message.
 *  - All calls share the array and it keeps the last call's contents; calls
 *    that overlap on the GPU (two streams, or two threads) race on it and give
 *    wrong results.  Serialise them. */
int ddnm_residual_noalloc(ddnm_ctx* ctx, int B, const double* mu, const double* x, const double* lam,
                          double* F_out, void* stream);

/* ---- Learned warm start (replaces the paper's RBF starting point, Sec. 7.2) ----
 * An MLP z = (mu - mu_c)/mu_s -> a1 = tanh(W1 z + b1) -> a2 = tanh(W2 a1 + b2) -> y = W3 a2 + b3,
 * xh0 = out_mean + out_std * y, trained on the device with hand-written forward, backward and Adam
 * kernels (bfloat16 weights in the products, FP32 accumulation and FP32 master weights).
 * Flat FP32 parameter layout: W1 (H x 2), b1 (H), W2 (H x H), b2 (H), W3 (n_D x H), b3 (n_D). */

/* Set the architecture (hidden width H, 1..4096) and the initial parameters (host, copied);
 * resets the Adam state and the normalisation (identity). */
int ddnm_ws_init(ddnm_ctx* ctx, int hidden, const float* params);

/* Input/output standardisation: mu_c[2], mu_s[2], out_mean[n_D], out_std[n_D] (host). */
int ddnm_ws_set_norm(ddnm_ctx* ctx, const double* mu_c, const double* mu_s, const double* out_mean,
                     const double* out_std);

/* Mean squared error and its gradient (P floats, host) on one batch of standardised inputs z
 * (nb x 2) and targets t (nb x n_D), at the current parameters (no update). */
int ddnm_ws_loss_grad(ddnm_ctx* ctx, int nb, const float* z, const float* t, float* grad, double* loss);

/* Mini-batch Adam (lr; beta1 0.9, beta2 0.999, eps 1e-8) on n samples mu (n x 2) -> x_star (n x n_D),
 * host FP64 arrays; order (epochs x n) gives each epoch's sample order (NULL: 0..n-1).  The
 * standardisation is taken from the training set.  losses (epochs, may be NULL) receives each
 * epoch's mean batch loss. */
int ddnm_ws_train(ddnm_ctx* ctx, int n, const double* mu, const double* x_star, int epochs, int batch, double lr,
                  const int* order, double* losses);

/* xh0 = MLP(mu) for B instances (mem_kind as in ddnm_solve_batch); a row with a non-finite
 * prediction is replaced by the default start 0. */
int ddnm_ws_predict(ddnm_ctx* ctx, int B, const double* mu, double* x0, int mem_kind, void* stream);

/* Current parameters (P floats) and normalisation (4 + 2 n_D doubles); either may be NULL. */
int ddnm_ws_get_params(const ddnm_ctx* ctx, float* params, double* norm);

/* With on != 0, ddnm_solve_batch calls with x0 == lam0 == NULL start each instance from the MLP
 * prediction; the default start xh0 = 0 is linearised alongside and kept when its merit is not larger
 * (flag DDNM_FLAG_WS_FALLBACK).  The screening evaluations are counted in n_evals. */
int ddnm_ws_enable(ddnm_ctx* ctx, int on);

/* Checkpoint of the warm start ("DDNMWS01", H, n_D, Adam step count, parameters, normalisation). */
int ddnm_ws_save(const ddnm_ctx* ctx, const char* path);
int ddnm_ws_load(ddnm_ctx* ctx, const char* path);

/* ---- Launch plan (batching of many mu and uneven subdomains) ----
 * By default ddnm_solve_batch queues the whole SQP loop of a batch as ONE CUDA
 * graph launch.  The graph runs the start-up passes of Sec. 4.1 / 7.2 (and the
 * warm-start screening), then splits the batch into `chains` groups of
 * consecutive instances.  Each group iterates in its own device-side while
 * loop, a conditional graph node whose body is two passes; the KKT kernel's
 * last CTA counts each pass and ends the loop when every instance of the
 * group has finished, or at the latest after 3 + max_iter * (max_backtracks
 * + 1) passes (a guard the per-instance limits reach first; a body's second
 * pass after the end finds no running instance).  One group's small FP64
 * kernels then overlap another group's evaluation.
 * Inside a pass, each width class of subdomains (equal padded latent widths) is
 * one evaluation launch.  With eval_persist > 0 that launch is persistent:
 * eval_persist CTAs per SM claim (instance, subdomain) items from a device
 * counter, largest subdomains first.
 * Results do not depend on the plan, bit for bit, apart from d_gemm (a different summation order of D_i):
 * instances are independent, and every kernel sums in a fixed order.  Atil in particular is one pairwise
 * tree over 512-row blocks of the constraint rows, whatever con_split is.  The graph is captured on first use and
 * re-captured when B, the options, the plan or the device tables change.
 * Per-kernel timing (ddnm_timing_enable) runs the host-driven loop instead. */
typedef struct ddnm_tune {
    int graph;          /* 1: graph-resident loop (default); 0: host-driven passes */
    int chains;         /* instance groups iterating concurrently, 1..64 (capped at B) */
    int con_split;      /* constraint rows per constraint CTA: 512, 1024 or 2048 */
    int eval_persist;   /* persistent evaluation: CTAs per SM per width class (1..8), or 0 for one CTA per item */
    int d_gemm;         /* D_i = C A_i dg_i^G: 1 in one GEMM launch per pass over all instances of a subdomain
                           (they share the decoder); 2 the same GEMM on the tensor cores (tcgen05, TF32 operands
                           split hi + lo for FP32 accuracy; mixed path with n_C <= 128, else taken as 1); 0
                           inside each evaluation CTA; -1 (default) picks the GEMM (2 in the mixed path, 1
                           in the FP64 path) when some subdomain has h^G n_C >= 65536 (hidden units of its
                           interface decoder times n_C), else 0 */
    int eval_groups;    /* 1 (default): one instance per evaluation CTA; 0: an evaluation CTA holds as many
                           independent 256-thread groups as one-instance CTAs would fit an SM, on neighbouring
                           instances of one subdomain (they share its tables through L1) */
    int atil;           /* the constraint residual Atil = C jump of the mixed path: 1 over tiles of instances
                           (C read once per tile) on the FP32 pipe in double-float arithmetic (C split into two
                           floats; each jump, a difference of two FP32 outputs, held exactly as two floats;
                           FP64 folds every 64 rows), accurate to about 2^-48 of sum_l |C_kl jump_l|;
                           0 per instance in FP64; -1 (default) picks 1 when n_C N_A >= 2^20.  The FP64 path
                           always takes 0. */
} ddnm_tune;

/* Set / read the plan (ddnm_get_tune reports d_gemm as given, -1 included).  DDNM_E_INVALID outside the
 * ranges above. */
int ddnm_set_tune(ddnm_ctx* ctx, const ddnm_tune* t);
int ddnm_get_tune(const ddnm_ctx* ctx, ddnm_tune* t);

/* Autotuner: times ddnm_solve_batch on this batch (B, mu; mem_kind as in
 * ddnm_solve_batch) under candidate plans and keeps the fastest in ctx.
 *  - Each candidate gets one untimed solve, then `reps` solves timed with CUDA
 *    events on `stream`; the median decides.
 *  - The search is coordinate-wise:
 *      chains       in {1, 2, 4, 8, 16, 32, 64}, capped at B;
 *      eval_persist in {0, 1, 2, 4};
 *      con_split    in {512, 1024, 2048};
 *      d_gemm       in {0, 1};
 *      eval_groups  in {0, 1}.
 *    Each knob is swept with the best values found so far for the others.
 *  - max_iter > 0 caps the SQP iterations of the timed solves, to keep tuning
 *    short (the options are restored on return).
 *  - best (may be NULL) receives the chosen plan, best_ms (may be NULL) its
 *    median time per solve call.
 * No result of a tuning solve is returned. */
int ddnm_autotune(ddnm_ctx* ctx, int B, const double* mu, int mem_kind, void* stream, int max_iter, int reps,
                  ddnm_tune* best, float* best_ms);

/* ---- Offline: training the autoencoders (Sec. 3.4, 5.1, 7.2-7.3) ----
 * Every subdomain has two sparse-masked shallow autoencoders, one for its interior states and one for its
 * interface states.  The decoder g (ddnm_decoder, loaded with ddnm_load_decoders) carries the three-band
 * mask on W2; the encoder h(x) = W2 sigma(W1 x + b1) carries the transposed mask on W1 (the encoder is
 * symmetric to the decoder across the latent layer, Sec. 5.1).  Training minimises the mean squared error
 * of Eq. (autoencoder_AbsMSE_loss) on snapshots normalised onto [-1, 1] (Sec. 7.3) by mini-batch Adam
 * (beta 0.9 / 0.999, eps 1e-8, constant learning rate), in FP32 with FP32 master weights.  On return the
 * trained decoders, with the normalisation as their de-normalisation layer (offset, scale), replace the
 * context's decoders: the next solve uses them. */
typedef struct ddnm_encoder {
    int N;                  /* inputs (must equal N_i^O or N_i^G) */
    int w;                  /* width (hidden units; must equal the decoder's) */
    int n;                  /* latent dim (must equal n_i^O or n_i^G; <= 16) */
    int Kt;                 /* ELL slots per hidden unit of W1 */
    const int* cols;        /* w x Kt: the inputs of each hidden unit, ascending, -1 padding at the end;
                               must be the transpose of the decoder's mask */
    const double* vals;     /* w x Kt */
    const double* b1;       /* w */
    const double* W2;       /* n x w */
} ddnm_encoder;

/* Initial encoder of subdomain `sub`, kind DDNM_DECODER_INTERIOR / _INTERFACE (host arrays, copied). */
int ddnm_load_encoder(ddnm_ctx* ctx, int sub, int kind, const ddnm_encoder* e);

/* Train all 2 n_sub autoencoders together on n_snap snapshots X (n_snap x N_x full FOM states, restricted
 * here to each subdomain's interior / interface states), starting from the loaded decoders and encoders.
 * The normalisation (offset = (max+min)/2, scale = (max-min)/2 per state, 1 for a constant state) is taken
 * over X.  Each epoch visits the snapshots in the order order[epoch * n_snap ..] (NULL: 0..n_snap-1) in
 * mini-batches of `batch` (1..32; the last batch of an epoch may be smaller).  losses (epochs x 2 n_sub,
 * may be NULL; autoencoder 2 s + kind) receives each epoch's mean batch loss.  X in host or device memory
 * (mem_kind); the snapshots are copied to the device for the call. */
int ddnm_ae_train(ddnm_ctx* ctx, int n_snap, const double* X, int epochs, int batch, double lr, const int* order,
                  double* losses, int mem_kind, void* stream);

/* Loss and gradient of one batch of normalised inputs Xt (nb x N, host FP32, nb <= 32) for the autoencoder
 * (sub, kind) at the loaded weights, without an update (for checking the gradient).  grad receives the
 * flat FP32 parameter block of that autoencoder; ddnm_ae_layout gives its layout: offsets[0..5] of W1 of
 * the encoder (w x Kt, ELL), b1 of the encoder, W2 of the encoder (n x w), W1 of the decoder (w x n), b1 of
 * the decoder, the decoder's W2 (N x K, ELL), and offsets[6] = the block's length. */
int ddnm_ae_loss_grad(ddnm_ctx* ctx, int sub, int kind, int nb, const float* Xt, float* grad, double* loss);
int ddnm_ae_layout(const ddnm_ctx* ctx, int sub, int kind, long long* offsets);

/* Current decoder (sub, kind): W1 (w x n), b1 (w), vals (N x K, in the loaded decoder's mask), scale and
 * offset (N); any may be NULL. */
int ddnm_get_decoder(const ddnm_ctx* ctx, int sub, int kind, double* W1, double* b1, double* vals, double* scale,
                     double* offset);

/* ---- Full-order model (Sec. 7.1) ----
 * Batched solve of the steady 2D Burgers finite-difference system r(x; mu) = 0 of
 * Eq. (burgers_discretized) on ctx's grid (the monolithic FOM; the paper's ROM errors,
 * Eq. relative_error, and speed-ups are measured against it, and its solutions are the
 * snapshots the decoders are trained on, Sec. 7.2).  Needs only ddnm_setup: no decoders.
 *
 * Newton's method; each step J dx = -r solved by BiCGSTAB in FP64, right-preconditioned by
 * the exact inverse of the diffusion part nu (D_xx + D_yy) per component (a sine transform in x
 * and tridiagonal solves in y, in FP32).  Newton stops when ||r||_2 <= 1e-12 max(1, ||r(x0)||_2),
 * or after a step that fails to halve ||r||_2 (the rounding floor; that step is kept), or after
 * max_newton steps; each linear solve stops at ||J dx + r||_2 <= 1e-10 ||r||_2 or after
 * max_krylov iterations.
 *   mu     B x 2
 *   x0     B x N_x start, or NULL for the exact solution Eq. (burgers_pde_exact_solution)
 *          sampled at the grid nodes
 *   x_out  B x N_x solution (ordering as everywhere: [u; v], x-fastest)
 *   stats  B entries (host memory), or NULL
 * mem_kind as in ddnm_solve_batch for mu, x0 and x_out.  Device memory: about 92 N_x bytes per
 * instance, allocated on first use and kept with ctx.  Returns DDNM_E_NOMEM if it does not fit. */
typedef struct ddnm_fom_stats {
    int newton_iters;       /* Newton steps taken */
    int krylov_iters;       /* BiCGSTAB iterations, summed over the Newton steps */
    int status;             /* 0 converged, 1 no convergence (stall above the rounding floor, or
                               max_newton reached), 2 non-finite residual */
    int pad;
    double res0;            /* ||r(x0)||_2 */
    double res;             /* ||r(x)||_2 at the returned state */
} ddnm_fom_stats;

int ddnm_fom_solve(ddnm_ctx* ctx, int B, const double* mu, const double* x0, double* x_out, ddnm_fom_stats* stats,
                   int max_newton, int max_krylov, int mem_kind, void* stream);

/* FOM residual r(x; mu) of Eq. (burgers_discretized) at B given full states x (B x N_x, ordering [u; v],
 * x-fastest), into r_out (B x N_x).  Used to collect residual snapshots along Newton's iterations for the
 * gappy-POD basis (Sec. 5.3, greedy-sampling remark).  mem_kind as in ddnm_solve_batch; with host memory the
 * call returns once r_out is written. */
int ddnm_fom_residual(ddnm_ctx* ctx, int B, const double* mu, const double* x, double* r_out, int mem_kind,
                      void* stream);

/* Measured FP32 and FP64 fused multiply-add throughput of ctx's device (TFLOP/s, 2 flops per FMA): a
 * grid of 8 CTAs x 256 threads per SM, every thread running 8 independent FMA chains, timed with CUDA
 * events (best of 3 after a warm-up launch).  The paper has no counterpart: it is the denominator of the
 * FP32 / FP64 roofline fractions that the benchmark reports.  Takes about a quarter of a second. */
int ddnm_measure_peaks(ddnm_ctx* ctx, double* fp32_tflops, double* fp64_tflops);

/* Turn per-kernel timing on (resets the counters) or off.  While on, every
 * compute call synchronises its stream before returning. */
int ddnm_timing_enable(ddnm_ctx* ctx, int on);

/* Read the accumulated per-kernel timing (launch counts are kept even when timing is off). */
int ddnm_get_timing(const ddnm_ctx* ctx, ddnm_timing* out);

/* Algorithmic work per instance-evaluation (valid once decoders and C are loaded;
 * DDNM_E_STATE before). */
int ddnm_get_work(ddnm_ctx* ctx, ddnm_work* out);

#ifdef __cplusplus
}
#endif
#endif /* DDNM_H */
