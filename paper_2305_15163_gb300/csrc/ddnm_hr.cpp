// Offline set-up of gappy-POD hyper-reduction (Sec. 3.1 Eq. dd_lspg_NLP with B_i = (Z_i Phi_i^r)^+ Z_i;
// Sec. 5.3, greedy-sampling remark), host code in FP64.
//
// Per subdomain, from residual snapshots (FOM residuals along Newton's iterations, ddnm_fom_residual):
//   1. the residual basis Phi_i^r: the leading nr left singular vectors of the snapshots restricted to the
//      subdomain's residual rows, by the method of snapshots (eigenvectors of the small Gram matrix Y^T Y by
//      cyclic Jacobi rotations, Phi = Y V Lambda^{-1/2}), re-orthonormalised by two Gram-Schmidt passes;
//   2. the sampled rows Z_i, one per greedy step: a step k < nr takes the row where basis vector k is worst
//      reproduced by the interpolation of basis vectors 0..k-1 on the rows taken so far (the first step: the
//      largest entry of vector 0); a step k >= nr takes the row of largest leverage phi_l^T G^{-1} phi_l with
//      G = Phi_S^T Phi_S over the rows taken (the row that most increases det G), the leverages kept current by
//      the Sherman-Morrison update of G^{-1} after each added row;
//   3. the projector (Z_i Phi_i^r)^+ = G^{-1} Phi_S^T (G by Cholesky), columns in ascending row order.
// Ties go to the smaller row.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "ddnm_ctx.h"

namespace {

// eigen-decomposition of the symmetric n x n matrix A (row-major, destroyed): eigenvalues w, eigenvectors in
// the columns of V, by cyclic Jacobi rotations
void jacobi_eigen(std::vector<double>& A, int n, std::vector<double>& w, std::vector<double>& V) {
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = 0; q < n; ++q) (p == q ? diag : off) += A[(size_t)p * n + q] * A[(size_t)p * n + q];
        if (off <= 1e-30 * diag || off == 0.0) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[(size_t)p * n + q];
                if (apq == 0.0) continue;
                const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {          // A <- A J (columns p, q)
                    const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * akq;
                    A[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {          // A <- J^T A (rows p, q)
                    const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * aqk;
                    A[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {          // V <- V J
                    const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * vkp - s * vkq;
                    V[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    w.resize(n);
    for (int i = 0; i < n; ++i) w[i] = A[(size_t)i * n + i];
}

// Cholesky of the SPD m x m matrix G (row-major) into its lower factor; false if not positive definite
bool cholesky(std::vector<double>& G, int m) {
    for (int j = 0; j < m; ++j) {
        double d = G[(size_t)j * m + j];
        for (int k = 0; k < j; ++k) d -= G[(size_t)j * m + k] * G[(size_t)j * m + k];
        if (!(d > 0.0)) return false;
        d = std::sqrt(d);
        G[(size_t)j * m + j] = d;
        for (int i = j + 1; i < m; ++i) {
            double v = G[(size_t)i * m + j];
            for (int k = 0; k < j; ++k) v -= G[(size_t)i * m + k] * G[(size_t)j * m + k];
            G[(size_t)i * m + j] = v / d;
        }
    }
    return true;
}

// x <- G^{-1} x with the Cholesky factor L of G
void chol_solve(const std::vector<double>& L, int m, double* x) {
    for (int i = 0; i < m; ++i) {
        double v = x[i];
        for (int k = 0; k < i; ++k) v -= L[(size_t)i * m + k] * x[k];
        x[i] = v / L[(size_t)i * m + i];
    }
    for (int i = m - 1; i >= 0; --i) {
        double v = x[i];
        for (int k = i + 1; k < m; ++k) v -= L[(size_t)k * m + i] * x[k];
        x[i] = v / L[(size_t)i * m + i];
    }
}

// Solve the k x k system A c = b (row-major A, destroyed) by Gaussian elimination with partial pivoting
bool dense_solve(std::vector<double>& A, int k, std::vector<double>& b) {
    for (int j = 0; j < k; ++j) {
        int p = j;
        for (int i = j + 1; i < k; ++i)
            if (std::fabs(A[(size_t)i * k + j]) > std::fabs(A[(size_t)p * k + j])) p = i;
        if (A[(size_t)p * k + j] == 0.0) return false;
        if (p != j) {
            for (int c = 0; c < k; ++c) std::swap(A[(size_t)p * k + c], A[(size_t)j * k + c]);
            std::swap(b[p], b[j]);
        }
        for (int i = j + 1; i < k; ++i) {
            const double f = A[(size_t)i * k + j] / A[(size_t)j * k + j];
            for (int c = j; c < k; ++c) A[(size_t)i * k + c] -= f * A[(size_t)j * k + c];
            b[i] -= f * b[j];
        }
    }
    for (int i = k - 1; i >= 0; --i) {
        double v = b[i];
        for (int c = i + 1; c < k; ++c) v -= A[(size_t)i * k + c] * b[c];
        b[i] = v / A[(size_t)i * k + i];
    }
    return true;
}

}  // namespace

extern "C" int ddnm_hr_select(ddnm_ctx* ctx, int n_snap, const double* snaps, const int* nr, const int* n_samples,
                              int* rows_out, double* proj_out) {
    if (!ctx) return DDNM_E_INVALID;
    if (n_snap < 1 || !snaps || !nr || !n_samples || !rows_out || !proj_out)
        return ddnm_fail(ctx, DDNM_E_INVALID, "ddnm_hr_select: n_snap >= 1 and every array are required");
    const int Nx = 2 * ctx->nx * ctx->ny;
    size_t rpos = 0, ppos = 0;
    for (int i = 0; i < ctx->n_sub; ++i) {
        const SubHost& sd = ctx->subs[i];
        // the subdomain's residual rows: both components of its owned nodes (local order: u rows, then v rows)
        std::vector<int> grows;
        for (int p : sd.owned) grows.push_back(p);
        for (int p : sd.owned) grows.push_back(ctx->nx * ctx->ny + p);
        const int Nr = (int)grows.size(), m = nr[i], ns = n_samples[i];
        if (m < 1 || m > ddnm::MAX_NR || m > n_snap || ns < m || ns > Nr)
            return ddnm_fail(ctx, DDNM_E_INVALID, "ddnm_hr_select: subdomain " + std::to_string(i) +
                                                      ": need 1 <= nr <= min(64, n_snap) and nr <= n_samples <= N_r");
        // 1. POD by the method of snapshots
        std::vector<double> Y((size_t)Nr * n_snap);
        for (int r = 0; r < Nr; ++r)
            for (int s = 0; s < n_snap; ++s) Y[(size_t)r * n_snap + s] = snaps[(size_t)s * Nx + grows[r]];
        std::vector<double> G((size_t)n_snap * n_snap, 0.0), w, V;
        for (int a = 0; a < n_snap; ++a)
            for (int b = a; b < n_snap; ++b) {
                double v = 0.0;
                for (int r = 0; r < Nr; ++r) v += Y[(size_t)r * n_snap + a] * Y[(size_t)r * n_snap + b];
                G[(size_t)a * n_snap + b] = G[(size_t)b * n_snap + a] = v;
            }
        jacobi_eigen(G, n_snap, w, V);
        std::vector<int> ord(n_snap);
        for (int k = 0; k < n_snap; ++k) ord[k] = k;
        std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return w[a] > w[b]; });
        if (!(w[ord[m - 1]] > 0.0))
            return ddnm_fail(ctx, DDNM_E_INVALID, "ddnm_hr_select: subdomain " + std::to_string(i) +
                                                      ": the snapshots span fewer than nr directions");
        std::vector<double> Phi((size_t)Nr * m);          // row-major N_r x m
        for (int j = 0; j < m; ++j) {
            const int e = ord[j];
            const double sc = 1.0 / std::sqrt(w[e]);
            for (int r = 0; r < Nr; ++r) {
                double v = 0.0;
                for (int s = 0; s < n_snap; ++s) v += Y[(size_t)r * n_snap + s] * V[(size_t)s * n_snap + e];
                Phi[(size_t)r * m + j] = v * sc;
            }
        }
        for (int pass = 0; pass < 2; ++pass)              // modified Gram-Schmidt, twice
            for (int j = 0; j < m; ++j) {
                for (int k = 0; k < j; ++k) {
                    double d = 0.0;
                    for (int r = 0; r < Nr; ++r) d += Phi[(size_t)r * m + k] * Phi[(size_t)r * m + j];
                    for (int r = 0; r < Nr; ++r) Phi[(size_t)r * m + j] -= d * Phi[(size_t)r * m + k];
                }
                double nn = 0.0;
                for (int r = 0; r < Nr; ++r) nn += Phi[(size_t)r * m + j] * Phi[(size_t)r * m + j];
                nn = 1.0 / std::sqrt(nn);
                for (int r = 0; r < Nr; ++r) Phi[(size_t)r * m + j] *= nn;
            }
        // 2. greedy rows
        std::vector<int> S;
        std::vector<char> taken(Nr, 0);
        auto pick = [&](const std::vector<double>& score) {
            int best = -1;
            for (int r = 0; r < Nr; ++r)
                if (!taken[r] && (best < 0 || score[r] > score[best])) best = r;
            taken[best] = 1;
            S.push_back(best);
        };
        std::vector<double> score(Nr);
        for (int k = 0; k < m; ++k) {                    // interpolation error of basis vector k
            std::vector<double> c(k, 0.0);
            if (k > 0) {
                std::vector<double> A((size_t)k * k);
                for (int a = 0; a < k; ++a)
                    for (int b = 0; b < k; ++b) A[(size_t)a * k + b] = Phi[(size_t)S[a] * m + b];
                for (int a = 0; a < k; ++a) c[a] = Phi[(size_t)S[a] * m + k];
                if (!dense_solve(A, k, c))
                    return ddnm_fail(ctx, DDNM_E_INVALID, "ddnm_hr_select: singular interpolation matrix");
            }
            for (int r = 0; r < Nr; ++r) {
                double e = Phi[(size_t)r * m + k];
                for (int b = 0; b < k; ++b) e -= Phi[(size_t)r * m + b] * c[b];
                score[r] = std::fabs(e);
            }
            pick(score);
        }
        // leverages against G = Phi_S^T Phi_S, kept current after each added row (Sherman-Morrison)
        std::vector<double> Gm((size_t)m * m, 0.0);
        for (int s : S)
            for (int a = 0; a < m; ++a)
                for (int b = 0; b < m; ++b) Gm[(size_t)a * m + b] += Phi[(size_t)s * m + a] * Phi[(size_t)s * m + b];
        std::vector<double> L = Gm;
        if (!cholesky(L, m)) return ddnm_fail(ctx, DDNM_E_INVALID, "ddnm_hr_select: rank-deficient sample");
        std::vector<double> Ginv((size_t)m * m, 0.0);
        for (int j = 0; j < m; ++j) {
            std::vector<double> e(m, 0.0);
            e[j] = 1.0;
            chol_solve(L, m, e.data());
            for (int a = 0; a < m; ++a) Ginv[(size_t)a * m + j] = e[a];
        }
        std::vector<double> lev(Nr), gphi(m);
        for (int r = 0; r < Nr; ++r) {
            double v = 0.0;
            for (int a = 0; a < m; ++a) {
                double t = 0.0;
                for (int b = 0; b < m; ++b) t += Ginv[(size_t)a * m + b] * Phi[(size_t)r * m + b];
                v += Phi[(size_t)r * m + a] * t;
            }
            lev[r] = v;
        }
        for (int k = m; k < ns; ++k) {
            pick(lev);
            const int s = S.back();
            for (int a = 0; a < m; ++a) {                // g = G^{-1} phi_s
                double t = 0.0;
                for (int b = 0; b < m; ++b) t += Ginv[(size_t)a * m + b] * Phi[(size_t)s * m + b];
                gphi[a] = t;
            }
            const double den = 1.0 + lev[s];
            for (int r = 0; r < Nr; ++r) {               // phi_r^T G'^{-1} phi_r = lev_r - (phi_r^T g)^2 / (1 + lev_s)
                double u = 0.0;
                for (int a = 0; a < m; ++a) u += Phi[(size_t)r * m + a] * gphi[a];
                lev[r] -= u * u / den;
            }
            for (int a = 0; a < m; ++a)
                for (int b = 0; b < m; ++b) Ginv[(size_t)a * m + b] -= gphi[a] * gphi[b] / den;
        }
        std::sort(S.begin(), S.end());
        // 3. (Z Phi)^+ = (Phi_S^T Phi_S)^{-1} Phi_S^T, columns in ascending row order
        std::fill(Gm.begin(), Gm.end(), 0.0);
        for (int s : S)
            for (int a = 0; a < m; ++a)
                for (int b = 0; b < m; ++b) Gm[(size_t)a * m + b] += Phi[(size_t)s * m + a] * Phi[(size_t)s * m + b];
        L = Gm;
        if (!cholesky(L, m)) return ddnm_fail(ctx, DDNM_E_INVALID, "ddnm_hr_select: rank-deficient sample");
        for (int q = 0; q < ns; ++q) {
            std::vector<double> col(m);
            for (int a = 0; a < m; ++a) col[a] = Phi[(size_t)S[q] * m + a];
            chol_solve(L, m, col.data());
            for (int a = 0; a < m; ++a) proj_out[ppos + (size_t)a * ns + q] = col[a];
        }
        for (int q = 0; q < ns; ++q) rows_out[rpos + q] = S[q];
        rpos += ns;
        ppos += (size_t)m * ns;
    }
    return DDNM_OK;
}
