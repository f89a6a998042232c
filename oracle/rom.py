"""WFPC DD-LSPG-ROM with collocation HR and its Lagrange-Gauss-Newton SQP solver, FP64.

Test infrastructure only (see ``oracle/__init__``).

Problem, Eq. (dd_lspg_NLP) / (dd_lspg_NLP_general) with the WFPC constraint (Sec. 3.1):

    min  1/2 sum_i || B_i r_i(g_i^O(xh_i^O), g_i^G(xh_i^G)) ||^2
    s.t. sum_i C A_i g_i^G(xh_i^G) = 0

with r_i(xO, xG) = P_i^r r(P_i^O^T xO + P_i^G^T xG)  (Eq. subdomain_residual_def) and
collocation HR B_i = Z_i (Sec. 3.1 / 5.3), B_i = I when no HR rows are given, or gappy-POD HR
B_i = (Z_i Phi_i^r)^+ Z_i when the projector (Z_i Phi_i^r)^+ is given (``hr_proj``, see ``oracle.hr``).

One evaluation builds, per subdomain (Sec. 4.1):
    R_i   = B_i [dr_i/dxO dg^O/dxh^O , dr_i/dxG dg^G/dxh^G]   (Eq. gauss_newton_hessian b)
    H_i   = R_i^T R_i                                          (Eq. gauss_newton_hessian a)
    E_i   = [0, D_i],  D_i = C A_i dg^G/dxh^G                  (Eq. sqp_block_matrices)
    rho_i = R_i^T r_i + E_i^T lambda                           (Eq. optimality_residuals_GN)
and Atil = sum_i C A_i g_i^G.  The KKT matrix of Eq. (sqp_system) is assembled densely and
solved by LU with partial pivoting (numpy.linalg.solve); RHS = -F, F = [rho_1..rho_n; Atil].

Readings (the paper leaves these open):
* merit phi = ||F||_2 ("the norm of the gradients", Sec. 4.1); Armijo backtracking accepts
  alpha when phi(alpha)^2 <= (1 - 2 c1 alpha) phi(0)^2, c1 = 1e-4, alpha <- beta alpha,
  beta = 1/2, at most ``max_bt`` halvings; if none is accepted the last trial is taken and
  the instance is flagged (FLAG_LS_FAIL);
* the multiplier estimate is kept and updated with the same alpha (Eq. sqp_update);
* stop when phi < tol (paper: 1e-4) or after max_iter accepted steps (paper: 15);
* default start xh0 = 0; lambda0 from the least-squares solve of Eq. (optimality_residuals b)
  at xh0 (Sec. 7.2), i.e. min_lambda sum_i ||(R_i^T r_i)_G + D_i^T lambda||^2.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .burgers import Burgers
from .dd import Decomposition

CONVERGED, MAX_ITER, NONFINITE = 0, 1, 2
FLAG_LS_FAIL = 1


@dataclass
class Evaluation:
    r: list            # Z_i r_i (the sampled rows, before a gappy projection)
    R: list            # Z_i [dr_i/dx dg_i/dxh] (the same rows)
    H: list            # H_i
    grad: list         # R_i^T r_i
    D: list            # D_i = C A_i dg_i^G
    Atil: np.ndarray   # sum_i C A_i g_i^G
    rho: list          # rho_i
    F: np.ndarray
    phi: float
    gO: list = field(default_factory=list)
    gG: list = field(default_factory=list)


@dataclass
class SolveResult:
    x: np.ndarray
    lam: np.ndarray
    iters: int
    status: int
    flags: int
    phi: float
    phi_hist: list
    alpha_hist: list
    n_evals: int


def _value_jacobian_rows(dec, x, rows):
    if hasattr(dec, "value_jacobian_rows"):
        return dec.value_jacobian_rows(x, rows)
    g, J = dec.value_jacobian(x)
    return g[rows], J[rows]


class DDROM:
    """decoders_O/decoders_G: objects with value_jacobian(x) -> (g, dg/dx);
    hr: per subdomain local residual-row ids (None = all rows, i.e. B_i = I);
    C: n_C x N_A test matrix;
    hr_proj: per subdomain (Z_i Phi_i^r)^+ (n_r x N_B, columns in the order of hr[i]) for gappy-POD HR,
    or None (collocation);
    Ahat: per subdomain A^_i (n_A x n_i^G) for the SRPC formulation (Sec. 3.2, Eq. dd_lspg_NLP_rom_port:
    linear constraints sum_i A^_i xh_i^G = 0, D_i = A^_i; see ``oracle.srpc``), or None (WFPC with C)."""

    def __init__(self, fom: Burgers, dd: Decomposition, decoders_O, decoders_G, hr, C, hr_proj=None, Ahat=None):
        self.fom, self.dd = fom, dd
        self.dO, self.dG = list(decoders_O), list(decoders_G)
        self.C = np.asarray(C, dtype=np.float64).reshape(-1, dd.N_A) if dd.N_A else np.zeros((0, 0))
        self.n_C = self.C.shape[0]
        # C A_i (n_C x N_i^G) through the sparse A_i
        self.CA = [np.asarray((A.T @ self.C.T).T) for A in dd.A] if dd.N_A else \
            [np.zeros((0, sd.interface.size)) for sd in dd.subs]
        self.Ahat = None if Ahat is None else [np.asarray(a, dtype=np.float64) for a in Ahat]
        if self.Ahat is not None:
            self.n_C = self.Ahat[0].shape[0]
        self.proj = [None] * len(dd.subs) if hr_proj is None else \
            [None if p is None else np.asarray(p, dtype=np.float64) for p in hr_proj]
        self.rows = []
        self.need = []
        N = fom.N
        for i, sd in enumerate(dd.subs):
            loc = np.arange(sd.res_rows.size) if (hr is None or hr[i] is None) else np.asarray(hr[i])
            rows = sd.res_rows[loc]
            self.rows.append(rows)                      # global rows of Z_i P_i^r
            # the interior outputs these rows' 5-point stencils touch (both components), as indices into
            # x_i^Omega: no other interior output enters Z_i r_i (the set I_o of Sec. 5.4)
            p = rows % N
            ii, jj = p % fom.nx, p // fom.nx
            q = np.concatenate([p, p[ii > 0] - 1, p[ii < fom.nx - 1] + 1, p[jj > 0] - fom.nx,
                                p[jj < fom.ny - 1] + fom.nx])
            self.need.append(np.flatnonzero(np.isin(sd.interior, np.concatenate([q, N + q]))))
        self._x = np.zeros(2 * N)
        self.nO = [d.n for d in self.dO]
        self.nG = [d.n for d in self.dG]
        self.n_i = [a + b for a, b in zip(self.nO, self.nG)]
        self.off = np.concatenate([[0], np.cumsum(self.n_i)]).astype(int)
        self.n_D = int(self.off[-1])

    # -- pieces of the latent vector xh = [xh_1^O; xh_1^G; ...] (Eq. sqp_notation a) -------
    def split(self, xh):
        out = []
        for i in range(len(self.n_i)):
            xi = xh[self.off[i]:self.off[i + 1]]
            out.append((xi[:self.nO[i]], xi[self.nO[i]:]))
        return out

    def evaluate(self, xh, lam, mu) -> Evaluation:
        """Blocks of Eq. (sqp_system) at (xh, lam): for every subdomain the collocated residual Z_i r_i and
        R_i = Z_i dr_i/dx_i dg_i/dxh_i (Eq. gauss_newton_hessian), from the decoder outputs the rows touch,
        H_i = R_i^T R_i, rho_i = R_i^T r_i + E_i^T lam, D_i = C A_i dg_i^G; Atil = sum_i C A_i g_i^G."""
        fom, dd = self.fom, self.dd
        bvec = fom.boundary_vectors(mu)
        ev = Evaluation([], [], [], [], [], np.zeros(self.n_C), [], None, 0.0)
        x = self._x
        for i, (xo, xg) in enumerate(self.split(xh)):
            sd = dd.subs[i]
            need = self.need[i]
            gO, JO = _value_jacobian_rows(self.dO[i], xo, need)
            gG, JG = self.dG[i].value_jacobian(xg)
            x[sd.interior[need]] = gO                    # the touched part of P_i^O^T gO + P_i^G^T gG
            x[sd.interface] = gG
            rows = self.rows[i]
            r = fom.residual_rows(x, mu, rows, bvec)
            J = fom.jacobian_rows(x, mu, rows, bvec)
            x[sd.interior[need]] = 0.0
            x[sd.interface] = 0.0
            R = np.hstack([J[:, sd.interior[need]] @ JO, J[:, sd.interface] @ JG])
            D = self.CA[i] @ JG if self.Ahat is None else self.Ahat[i]
            Pg = self.proj[i]
            Rb, rb = (R, r) if Pg is None else (Pg @ R, Pg @ r)      # B_i applied (gappy POD) or Z_i alone
            grad = Rb.T @ rb
            rho = grad.copy()
            rho[self.nO[i]:] += D.T @ lam
            ev.r.append(r); ev.R.append(R); ev.H.append(Rb.T @ Rb); ev.grad.append(grad)
            ev.D.append(D); ev.rho.append(rho); ev.gO.append(gO); ev.gG.append(gG)
            ev.Atil = ev.Atil + (self.CA[i] @ gG if self.Ahat is None else self.Ahat[i] @ xg)
        ev.F = np.concatenate(ev.rho + [ev.Atil])
        ev.phi = float(np.linalg.norm(ev.F))
        return ev

    def evaluate_dense(self, xh, lam, mu) -> Evaluation:
        """evaluate() written on the whole state and the whole FOM residual and Jacobian (rows picked
        afterwards): the plain form that pins the row-restricted one on small problems."""
        fom, dd = self.fom, self.dd
        bvec = fom.boundary_vectors(mu)
        ev = Evaluation([], [], [], [], [], np.zeros(self.n_C), [], None, 0.0)
        for i, (xo, xg) in enumerate(self.split(xh)):
            sd = dd.subs[i]
            gO, JO = self.dO[i].value_jacobian(xo)
            gG, JG = self.dG[i].value_jacobian(xg)
            x = np.zeros(2 * fom.N)                      # P_i^O^T gO + P_i^G^T gG
            x[sd.interior] = gO
            x[sd.interface] = gG
            rows = self.rows[i]
            r = fom.residual(x, mu, bvec)[rows]
            J = fom.jacobian(x, mu, bvec)[rows]
            R = np.hstack([J[:, sd.interior] @ JO, J[:, sd.interface] @ JG])
            D = self.CA[i] @ JG if self.Ahat is None else self.Ahat[i]
            Pg = self.proj[i]
            Rb, rb = (R, r) if Pg is None else (Pg @ R, Pg @ r)      # B_i applied (gappy POD) or Z_i alone
            grad = Rb.T @ rb
            rho = grad.copy()
            rho[self.nO[i]:] += D.T @ lam
            ev.r.append(r); ev.R.append(R); ev.H.append(Rb.T @ Rb); ev.grad.append(grad)
            ev.D.append(D); ev.rho.append(rho); ev.gO.append(gO); ev.gG.append(gG)
            ev.Atil = ev.Atil + (self.CA[i] @ gG if self.Ahat is None else self.Ahat[i] @ xg)
        ev.F = np.concatenate(ev.rho + [ev.Atil])
        ev.phi = float(np.linalg.norm(ev.F))
        return ev

    def kkt_matrix(self, ev: Evaluation):
        """Dense block-arrowhead matrix of Eq. (sqp_system), size n_D + n_C."""
        n = self.n_D + self.n_C
        K = np.zeros((n, n))
        for i in range(len(self.n_i)):
            a, b = self.off[i], self.off[i + 1]
            K[a:b, a:b] = ev.H[i]
            E = np.hstack([np.zeros((self.n_C, self.nO[i])), ev.D[i]])
            K[self.n_D:, a:b] = E
            K[a:b, self.n_D:] = E.T
        return K

    def kkt_step(self, ev: Evaluation):
        sol = np.linalg.solve(self.kkt_matrix(ev), -ev.F)
        return sol[:self.n_D], sol[self.n_D:]

    def lambda_ls(self, ev: Evaluation):
        """Least-squares multiplier from Eq. (optimality_residuals b) at the current point."""
        if self.n_C == 0:
            return np.zeros(0)
        M = np.vstack([D.T for D in ev.D])
        b = -np.concatenate([g[self.nO[i]:] for i, g in enumerate(ev.grad)])
        return np.linalg.lstsq(M, b, rcond=None)[0]

    def solve(self, mu, x0=None, lam0=None, tol=1e-4, max_iter=15, c1=1e-4, beta=0.5,
              max_bt=20) -> SolveResult:
        x = np.zeros(self.n_D) if x0 is None else np.array(x0, dtype=np.float64)
        if lam0 is None:
            lam = self.lambda_ls(self.evaluate(x, np.zeros(self.n_C), mu))
            n_evals = 1
        else:
            lam = np.array(lam0, dtype=np.float64)
            n_evals = 0
        ev = self.evaluate(x, lam, mu)
        n_evals += 1
        phi = ev.phi
        hist, ahist = [phi], []
        iters, flags = 0, 0
        while True:
            if not np.isfinite(phi):
                status = NONFINITE
                break
            if phi < tol:
                status = CONVERGED
                break
            if iters == max_iter:
                status = MAX_ITER
                break
            s, sl = self.kkt_step(ev)
            alpha, nbt = 1.0, 0
            while True:
                xt, lt = x + alpha * s, lam + alpha * sl
                evt = self.evaluate(xt, lt, mu)
                n_evals += 1
                if evt.phi ** 2 <= (1.0 - 2.0 * c1 * alpha) * phi ** 2:
                    break
                if nbt == max_bt:
                    flags |= FLAG_LS_FAIL
                    break
                alpha *= beta
                nbt += 1
            x, lam, ev, phi = xt, lt, evt, evt.phi
            iters += 1
            hist.append(phi)
            ahist.append(alpha)
        return SolveResult(x, lam, iters, status, flags, phi, hist, ahist, n_evals)

    # -- reconstruction and error ------------------------------------------------------------
    def states(self, xh):
        """[(g_i^O(xh_i^O), g_i^G(xh_i^G))] for every subdomain."""
        return [(self.dO[i].value(xo), self.dG[i].value(xg)) for i, (xo, xg) in enumerate(self.split(xh))]

    def full_state(self, xh):
        """Monolithic state assembled from each node's owning subdomain."""
        x = np.zeros(2 * self.fom.N)
        for i, (gO, gG) in enumerate(self.states(xh)):
            sd = self.dd.subs[i]
            own = np.zeros(2 * self.fom.N, dtype=bool)
            own[sd.res_rows] = True                     # owned variables = owned residual rows
            m = own[sd.interior]
            x[sd.interior[m]] = gO[m]
            m = own[sd.interface]
            x[sd.interface[m]] = gG[m]
        return x


def relative_error(ref_states, rom_states) -> float:
    """Eq. (relative_error): per-subdomain relative errors of interior+interface states,
    averaged over subdomains, square root taken last.  ``*_states``: [(xO, xG)] lists."""
    acc = 0.0
    for (xo, xg), (go, gg) in zip(ref_states, rom_states):
        num = np.sum((xo - go) ** 2) + np.sum((xg - gg) ** 2)
        den = np.sum(xo ** 2) + np.sum(xg ** 2)
        acc += num / den
    return float(np.sqrt(acc / len(ref_states)))
