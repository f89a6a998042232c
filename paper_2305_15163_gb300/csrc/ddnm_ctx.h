// Library context: host copy of the problem and device handles.  Internal.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "ddnm.h"
#include "ddnm_internal.h"

struct DecoderHost {
    bool loaded = false;
    int N = 0, w = 0, n = 0, act = 0, K = 0;
    std::vector<double> W1, b1, vals, scale, offset;
    std::vector<int> cols;
};

// one port of the SRPC formulation: the sorted subdomains P(j) sharing it, its variables (ascending global ids)
struct PortHost {
    std::vector<int> subs, vars;
    int N = 0, n = 0;            // variables, latents n_j^p
};

struct SubHost {
    std::vector<int> owned;      // owned node ids, ascending
    std::vector<int> interior;   // global variable ids, ascending
    std::vector<int> interface;  // global variable ids, ascending
    std::vector<int> hr_rows;    // local residual-row ids
    std::vector<int> hr_raw;     // HR_INTS per row: component, then 6 operands (global variable id, or
                                 // -(2 * Dirichlet point + component) - 1)
    std::vector<int> need;       // interior outputs the stencils use (I_o), ascending local indices
    std::vector<int> needG;      // interface outputs the stencils use, ascending local indices
    int nO = 0, nG = 0;
    int nr = 0;                  // gappy-POD HR: rows of the projector (Z_i Phi_i^r)^+ (0: collocation)
    std::vector<double> proj;    // nr x N_B, columns in the order of hr_rows
};

// learned warm start (ddnm_mlp.cu): MLP mu -> xh0 with FP32 master weights and a bfloat16 copy
struct WarmStart {
    bool ready = false, enabled = false;
    int H = 0, n = 0;                  // hidden width, outputs (= n_D)
    long long steps = 0;               // Adam steps taken
    float* p = nullptr;                // parameters (FP32 master)
    __nv_bfloat16* pb = nullptr;       // bfloat16 copy read by the GEMMs
    float* m = nullptr;                // Adam moments
    float* v = nullptr;
    float* norm = nullptr;             // mu_c[2], mu_s[2], out_mean[n], out_std[n]
    void* act = nullptr;               // batch buffers
    int cap = 0;
    float *z = nullptr, *a1 = nullptr, *a2 = nullptr, *y = nullptr, *t = nullptr;
    float *dy = nullptr, *d2 = nullptr, *d1 = nullptr, *g = nullptr;
    double* lpart = nullptr;
    void* data = nullptr;              // training set on the device
};

// subdomains sharing the padded record widths of the evaluation kernel
struct EvalClass {
    int ro, rg;      // round4(n^O + 1), round4(n^G + 1)
    int off, n;      // range in the class index table
    int smem;        // largest dynamic shared memory of its subdomains (one instance)
    int stride;      // smem rounded up to 128 bytes: one group's area in a grouped CTA
    int groups;      // instances per CTA when grouped: the one-instance CTAs of this class that fit an SM
    int nt;          // threads of one instance's evaluation (eval_threads)
};

struct ddnm_ctx {
    // problem
    int nx = 0, ny = 0, kx = 0, ky = 0, n_sub = 0, N = 0, n_C = 0, N_A = 0;
    int precision = DDNM_MIXED, device = 0;
    double nu = 0.1, box[4] = {-1, 1, -1, 1}, hx = 0, hy = 0;
    ddnm_options opt{1e-4, 15, 1e-4, 0.5, 20, 0.0};
    std::vector<int> xb, yb;
    std::vector<SubHost> subs;
    std::vector<int> con_var, con_lo, con_hi, con_lo_flat, con_hi_flat;
    std::vector<int> bnd_ij;     // 2 per Dirichlet point (I, J), 0 <= I <= nx+1
    std::vector<int> goff;       // offset of each subdomain's interface outputs
    std::vector<double> C;
    bool have_C = false;
    std::vector<DecoderHost> decO, decG;
    // SRPC formulation (ddnm_srpc.cpp): ports, their decoders, A^_i (n_C x n_i^G each)
    bool srpc = false;
    std::vector<PortHost> ports;
    std::vector<DecoderHost> port_dec;
    std::vector<std::vector<double>> Ahat;
    int n_D = 0, sum_NG = 0, sum_NB = 0;

    // device side (valid once finalized)
    bool finalized = false;
    std::vector<ddnm::SubDev> hsub;
    ddnm::ProbDev pd{};
    int eval_smem = 0, kkt_smem = 0, rec_smem = 0, ss_rows = 0, max_nG = 1;
    int fac_smem = 0;                  // dynamic shared memory of a factorisation CTA of k_constraint
    bool fac_share = false;            // the factorisation CTAs form the Schur-sum shares (Spart)
    void* d_vpool = nullptr;
    int* d_ipool = nullptr;
    int* d_hr = nullptr;
    int* d_con = nullptr;
    double* d_C = nullptr;
    float* d_Ct = nullptr;             // mixed path: C transposed, split into FP32 hi and lo parts (2 N_A ldct)
    float* d_Qtc = nullptr;            // mixed path: Q_i split into TF32 hi / lo, tiled for k_dgemm_tc
    int* d_err = nullptr;              // device error word (ddnm::DDNM_TC_TIMEOUT)
    double* d_Ahat = nullptr;          // SRPC: every A^_i, n_C x n_i^G, at SubDev::ahat
    int* d_bnd_ij = nullptr;
    ddnm::SubDev* d_sub = nullptr;
    ddnm::ChunkDev* d_chunk = nullptr;
    ddnm::TileDev* d_tiles = nullptr;
    std::vector<ddnm::TileDev> htiles;
    std::vector<EvalClass> eval_classes;
    int* d_classes = nullptr;          // subdomain indices, grouped by class
    std::vector<ddnm::ChunkDev> hchunk;

    // workspace for up to cap_B instances
    int cap_B = 0;
    void* d_ws = nullptr;
    int* h_active = nullptr;     // pinned

    std::vector<long long> nnzO, nnzG, nnzGn;   // mask nonzeros: interior subnet rows, all interface rows,
                                                // interface rows the stencils use

    WarmStart ws;

    void* fom = nullptr;               // batched FOM solver workspace (ddnm_fom.cu)
    void* ae = nullptr;                // autoencoder training state (ddnm_ae.cu)

    // per-kernel timing (ddnm_timing_enable)
    bool timing = false;
    ddnm_timing tm{};
    std::vector<cudaEvent_t> events;   // pool, pairs (start, stop)
    std::vector<int> event_kind;       // 0 eval, 1 constraint, 2 step for each recorded pair
    size_t n_events = 0;               // pairs in use for the current call

    // launch plan and the captured solve graph (ddnm_kernels.cu)
    ddnm_tune tune{1, 1, ddnm::CON_SPLIT, 0, -1, 1, -1};
    int dgemm_auto = 0;                // the d_gemm = -1 choice for these sizes (set with the tables)
    int atil_auto = 0;                 // the atil = -1 choice
    long long gen = 0;                 // bumped whenever device tables or workspace pointers change
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::vector<long long> gkey;       // what the captured graph was built for
    cudaStream_t cap_main = nullptr, cap_body = nullptr;   // capture streams
    int n_sm = 0;
    int* h_pass = nullptr;             // pinned: loop passes per instance group of the last graph solve
    cudaEvent_t pass_ev = nullptr;
    bool pass_pending = false;
    int pending_chains = 0, pending_classes = 0;

    std::string err;
};

// set-up helpers implemented in ddnm_host.cpp
int ddnm_fail(ddnm_ctx* ctx, int code, const std::string& msg);
int ddnm_finalize(ddnm_ctx* ctx);
int ddnm_reserve(ddnm_ctx* ctx, int B);
void ddnm_release_events(ddnm_ctx* ctx);
void ddnm_release_graph(ddnm_ctx* ctx);
void ddnm_ws_release(ddnm_ctx* ctx);
void ddnm_fom_release(ddnm_ctx* ctx);
void ddnm_ae_release(ddnm_ctx* ctx);
int ddnm_ws_predict_dev(ddnm_ctx* ctx, int B, const double* mu_dev, double* x0_dev, int* fell_back, cudaStream_t st);
// tensor-core D_i GEMM of the mixed path (ddnm_tc.cu)
bool ddnm_dgemm_tc_ok(const ddnm_ctx* ctx);
cudaError_t ddnm_launch_dgemm_tc(ddnm_ctx* ctx, const ddnm::ProbDev& P, int B, cudaStream_t st);
void ddnm_tile_q_tc(std::vector<float>& out, const double* Qt, int hG, int qld, int nC, long long& off, int& hGp);
