"""Steady 2D viscous Burgers FOM (Sec. 7.1), FP64.

Test infrastructure only (see ``oracle/__init__``).

The residual is written exactly in the paper's matrix form, Eq. (burgers_discretized):

    r_u = u o (B_x u - b_{u,x}) + v o (B_y u - b_{u,y}) + L u + c_u
    r_v = u o (B_x v - b_{v,x}) + v o (B_y v - b_{v,y}) + L v + c_v

with B_x = -(1/2h_x) (I_{ny} (x) Bt_x), B_y = -(1/2h_y) (Bt_y (x) I_{nx}),
L = nu/h_x^2 (I (x) Ct_x) + nu/h_y^2 (Ct_y (x) I)  (the paper calls L "C"; renamed here
to keep it apart from the Gaussian test matrix of Sec. 3.1), and boundary vectors from the
exact solution Eq. (burgers_pde_exact_solution).

Readings:
* domain: a box, default [-1,1]^2 (the paper's is [-1,1]x[0,0.05]); x_i = x0 + i h_x,
  h_x = (x1-x0)/(nx+1), likewise in y;
* the paper names the y boundary vectors b_{uy l}/b_{uy r} in b_{u,y} and c_u but defines
  b_{uyb}/b_{uyt}: l = bottom (y_0), r = top (y_{ny+1}), which makes B_y u - b_{u,y} the
  centred -du/dy at the first and last rows;
* state ordering x = [u; v], each block x-fastest (u^{[j]} rows).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

BOX = (-1.0, 1.0, -1.0, 1.0)


def exact_solution(x, y, a, lam, nu):
    """(u_ex, v_ex) of Eq. (burgers_pde_exact_solution) with psi = a(1+x) + 2cosh(lam(x-1))cos(lam y)."""
    ep = np.exp(lam * (x - 1.0))
    em = np.exp(-lam * (x - 1.0))
    psi = a * (1.0 + x) + (ep + em) * np.cos(lam * y)
    u = -2.0 * nu * (a + lam * (ep - em) * np.cos(lam * y)) / psi
    v = 2.0 * nu * (lam * (ep + em) * np.sin(lam * y)) / psi
    return u, v


class Burgers:
    """FOM r(x; mu) = 0 on an nx x ny interior grid, mu = (a, lambda)."""

    def __init__(self, nx: int, ny: int, nu: float = 0.1, box=BOX):
        self.nx, self.ny, self.nu, self.box = nx, ny, nu, box
        self.N = nx * ny
        self.hx = (box[1] - box[0]) / (nx + 1)
        self.hy = (box[3] - box[2]) / (ny + 1)
        self.xs = box[0] + self.hx * np.arange(nx + 2)          # x_0 .. x_{nx+1}
        self.ys = box[2] + self.hy * np.arange(ny + 2)          # y_0 .. y_{ny+1}

        def skew(n):  # tridiag(-1, 0, 1)
            return sp.diags([-np.ones(n - 1), np.ones(n - 1)], [-1, 1], format="csr")

        def second(n):  # tridiag(1, -2, 1)
            return sp.diags([np.ones(n - 1), -2.0 * np.ones(n), np.ones(n - 1)], [-1, 0, 1], format="csr")

        Ix, Iy = sp.identity(nx, format="csr"), sp.identity(ny, format="csr")
        self.Bx = (-1.0 / (2.0 * self.hx)) * sp.kron(Iy, skew(nx), format="csr")
        self.By = (-1.0 / (2.0 * self.hy)) * sp.kron(skew(ny), Ix, format="csr")
        self.L = (nu / self.hx ** 2) * sp.kron(Iy, second(nx), format="csr") \
            + (nu / self.hy ** 2) * sp.kron(second(ny), Ix, format="csr")

    # -- boundary data ------------------------------------------------------------------
    def boundary_vectors(self, mu):
        """(b_{u,x}, b_{u,y}, c_u, b_{v,x}, b_{v,y}, c_v) for mu = (a, lambda)."""
        a, lam = float(mu[0]), float(mu[1])
        nx, ny, nu = self.nx, self.ny, self.nu
        xs, ys = self.xs, self.ys
        e1x = np.zeros(nx); e1x[0] = 1.0
        enx = np.zeros(nx); enx[-1] = 1.0
        e1y = np.zeros(ny); e1y[0] = 1.0
        eny = np.zeros(ny); eny[-1] = 1.0
        uL, vL = exact_solution(xs[0], ys[1:ny + 1], a, lam, nu)        # x_0, y_1..y_ny
        uR, vR = exact_solution(xs[nx + 1], ys[1:ny + 1], a, lam, nu)   # x_{nx+1}
        uB, vB = exact_solution(xs[1:nx + 1], ys[0], a, lam, nu)        # y_0
        uT, vT = exact_solution(xs[1:nx + 1], ys[ny + 1], a, lam, nu)   # y_{ny+1}
        out = []
        for (bl, br, bb, bt) in ((uL, uR, uB, uT), (vL, vR, vB, vT)):
            bxl = np.kron(bl, e1x)
            bxr = np.kron(br, enx)
            byb = np.kron(e1y, bb)
            byt = np.kron(eny, bt)
            b_x = -(1.0 / (2.0 * self.hx)) * (bxl - bxr)
            b_y = -(1.0 / (2.0 * self.hy)) * (byb - byt)
            c = (nu / self.hx ** 2) * (bxl + bxr) + (nu / self.hy ** 2) * (byb + byt)
            out += [b_x, b_y, c]
        return tuple(out)

    # -- residual and Jacobian -----------------------------------------------------------
    def residual(self, x, mu, bvec=None):
        N = self.N
        u, v = x[:N], x[N:]
        bux, buy, cu, bvx, bvy, cv = self.boundary_vectors(mu) if bvec is None else bvec
        ru = u * (self.Bx @ u - bux) + v * (self.By @ u - buy) + self.L @ u + cu
        rv = u * (self.Bx @ v - bvx) + v * (self.By @ v - bvy) + self.L @ v + cv
        return np.concatenate([ru, rv])

    def jacobian(self, x, mu, bvec=None):
        """dr/dx (sparse 2N x 2N), differentiating Eq. (burgers_discretized) term by term."""
        N = self.N
        u, v = x[:N], x[N:]
        bux, buy, cu, bvx, bvy, cv = self.boundary_vectors(mu) if bvec is None else bvec
        D = sp.diags
        Juu = D(self.Bx @ u - bux) + D(u) @ self.Bx + D(v) @ self.By + self.L
        Juv = D(self.By @ u - buy)
        Jvu = D(self.Bx @ v - bvx)
        Jvv = D(u) @ self.Bx + D(self.By @ v - bvy) + D(v) @ self.By + self.L
        return sp.bmat([[Juu, Juv], [Jvu, Jvv]], format="csr")

    # -- the same, restricted to some residual rows ----------------------------------------
    # Eq. (burgers_discretized) row by row: the rows `rows` (ascending global ids; u rows are < N) of r and
    # of dr/dx, built from those rows of B_x, B_y and L only, so that the cost follows the rows (the
    # collocation rows of Sec. 5.3) rather than the grid.
    def _split_rows(self, rows):
        rows = np.asarray(rows, dtype=np.int64)
        if rows.size > 1 and np.any(np.diff(rows) <= 0):
            raise ValueError("rows must be ascending")
        N = self.N
        return rows[rows < N], rows[rows >= N] - N

    def residual_rows(self, x, mu, rows, bvec=None):
        N = self.N
        u, v = x[:N], x[N:]
        bux, buy, cu, bvx, bvy, cv = self.boundary_vectors(mu) if bvec is None else bvec
        pu, pv = self._split_rows(rows)
        ru = u[pu] * (self.Bx[pu] @ u - bux[pu]) + v[pu] * (self.By[pu] @ u - buy[pu]) + self.L[pu] @ u + cu[pu]
        rv = u[pv] * (self.Bx[pv] @ v - bvx[pv]) + v[pv] * (self.By[pv] @ v - bvy[pv]) + self.L[pv] @ v + cv[pv]
        return np.concatenate([ru, rv])

    def jacobian_rows(self, x, mu, rows, bvec=None):
        """Rows `rows` of dr/dx (sparse |rows| x 2N)."""
        N = self.N
        u, v = x[:N], x[N:]
        bux, buy, cu, bvx, bvy, cv = self.boundary_vectors(mu) if bvec is None else bvec
        pu, pv = self._split_rows(rows)
        D = sp.diags

        def sel(p):          # rows e_p^T of the identity
            return sp.csr_matrix((np.ones(p.size), (np.arange(p.size), p)), shape=(p.size, N))

        Juu = D(self.Bx[pu] @ u - bux[pu]) @ sel(pu) + D(u[pu]) @ self.Bx[pu] + D(v[pu]) @ self.By[pu] + self.L[pu]
        Juv = D(self.By[pu] @ u - buy[pu]) @ sel(pu)
        Jvu = D(self.Bx[pv] @ v - bvx[pv]) @ sel(pv)
        Jvv = D(u[pv]) @ self.Bx[pv] + D(self.By[pv] @ v - bvy[pv]) @ sel(pv) + D(v[pv]) @ self.By[pv] + self.L[pv]
        return sp.bmat([[Juu, Juv], [Jvu, Jvv]], format="csr")

    # -- monolithic FOM solve ------------------------------------------------------------
    def newton(self, mu, x0=None, rtol=1e-12, max_iter=50, residuals=None):
        """Newton on r(x; mu) = 0 from x0 (default 0), sparse LU; stops at
        ||r|| <= rtol * max(1, ||r(x0)||), or once a step fails to halve ||r||: in Newton's quadratic regime
        that happens only at the rounding floor of the residual (a start close to the solution, e.g. the
        exact solution at the nodes, can begin below rtol * max(1, ||r(x0)||) of nothing but that floor).
        Returns (x, residual history).  residuals: a list that receives the residual vector r(x_k) of every
        iterate (the residual snapshots of Sec. 5.3's greedy HR remark)."""
        bvec = self.boundary_vectors(mu)
        x = np.zeros(2 * self.N) if x0 is None else np.array(x0, dtype=np.float64)
        r = self.residual(x, mu, bvec)
        if residuals is not None:
            residuals.append(r.copy())
        stop = rtol * max(1.0, np.linalg.norm(r))
        hist = [np.linalg.norm(r)]
        for _ in range(max_iter):
            if hist[-1] <= stop:
                break
            dx = spla.spsolve(self.jacobian(x, mu, bvec).tocsc(), -r)
            x = x + dx
            r = self.residual(x, mu, bvec)
            if residuals is not None:
                residuals.append(r.copy())
            hist.append(np.linalg.norm(r))
            if hist[-1] > 0.5 * hist[-2]:
                break
        return x, hist

    def exact_state(self, mu):
        """Exact solution sampled at the interior nodes, ordered like x."""
        X, Y = np.meshgrid(self.xs[1:self.nx + 1], self.ys[1:self.ny + 1])   # row j, col i
        u, v = exact_solution(X.ravel(), Y.ravel(), float(mu[0]), float(mu[1]), self.nu)
        return np.concatenate([u, v])
