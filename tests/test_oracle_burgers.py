"""Pins of the oracle's Burgers FOM (Sec. 7.1) against the mathematics."""
import numpy as np
import pytest

from oracle.burgers import Burgers, exact_solution

NU = 0.1


def _pde_residual(x, y, a, lam, nu, h=1e-3):
    """Continuous Burgers residual of the closed form, by 4th-order central differences."""
    def d1(f, x, y, ax):
        if ax == 0:
            return (-f(x + 2 * h, y) + 8 * f(x + h, y) - 8 * f(x - h, y) + f(x - 2 * h, y)) / (12 * h)
        return (-f(x, y + 2 * h) + 8 * f(x, y + h) - 8 * f(x, y - h) + f(x, y - 2 * h)) / (12 * h)

    def d2(f, x, y, ax):
        if ax == 0:
            return (-f(x + 2 * h, y) + 16 * f(x + h, y) - 30 * f(x, y) + 16 * f(x - h, y) - f(x - 2 * h, y)) / (12 * h * h)
        return (-f(x, y + 2 * h) + 16 * f(x, y + h) - 30 * f(x, y) + 16 * f(x, y - h) - f(x, y - 2 * h)) / (12 * h * h)

    U = lambda x, y: exact_solution(x, y, a, lam, nu)[0]
    V = lambda x, y: exact_solution(x, y, a, lam, nu)[1]
    u, v = U(x, y), V(x, y)
    terms_u = [u * d1(U, x, y, 0), v * d1(U, x, y, 1), -nu * d2(U, x, y, 0), -nu * d2(U, x, y, 1)]
    terms_v = [u * d1(V, x, y, 0), v * d1(V, x, y, 1), -nu * d2(V, x, y, 0), -nu * d2(V, x, y, 1)]
    # residual relative to the largest term magnitude seen over the sample
    scale_u = np.max(sum(np.abs(t) for t in terms_u))
    scale_v = np.max(sum(np.abs(t) for t in terms_v))
    return sum(terms_u) / scale_u, sum(terms_v) / scale_v


@pytest.mark.parametrize("a,lam", [(1.0, 1.0), (0.9, 1.1), (1.1, 0.9), (7692.5384, 21.9230)])
def test_exact_solution_solves_pde(a, lam):
    """Eq. (burgers_pde_exact_solution) solves Eq. (burgers_pde_2d) (Cole-Hopf, harmonic psi)."""
    r = np.random.default_rng(0)
    if lam > 5:   # the paper's own domain and parameters: [-1,1] x [0,0.05]
        x, y = r.uniform(-0.9, 0.9, 50), r.uniform(0.005, 0.045, 50)
    else:
        x, y = r.uniform(-0.9, 0.9, 50), r.uniform(-0.9, 0.9, 50)
    h = 1e-3 if lam < 5 else 1e-4
    ru, rv = _pde_residual(x, y, a, lam, NU, h)
    assert np.max(np.abs(ru)) < 1e-6
    assert np.max(np.abs(rv)) < 1e-6


def test_exact_solution_sign_and_symmetry():
    # v vanishes on y = 0 (sin term) and u is negative where psi_x > 0 (u = -2 nu psi_x / psi)
    u, v = exact_solution(np.array([-0.5, 0.3]), np.array([0.0, 0.0]), 1.0, 1.0, NU)
    assert np.allclose(v, 0.0)
    ep, em = np.exp(-1.5), np.exp(1.5)
    psi = 0.5 + ep + em
    assert np.isclose(u[0], -2 * NU * (1.0 + (ep - em)) / psi)


def test_fom_matches_pointwise_stencil():
    """The Kronecker matrix form equals a node-by-node centred-difference loop (tiny grid)."""
    nx, ny, mu = 4, 3, (1.05, 0.95)
    fom = Burgers(nx, ny, NU)
    r = np.random.default_rng(1)
    x = r.standard_normal(2 * nx * ny) * 0.3
    res = fom.residual(x, mu)
    U = np.zeros((ny + 2, nx + 2)); V = np.zeros((ny + 2, nx + 2))
    for j in range(ny + 2):
        for i in range(nx + 2):
            if 1 <= i <= nx and 1 <= j <= ny:
                p = (j - 1) * nx + (i - 1)
                U[j, i], V[j, i] = x[p], x[nx * ny + p]
            else:
                U[j, i], V[j, i] = exact_solution(fom.xs[i], fom.ys[j], mu[0], mu[1], NU)
    hx, hy = fom.hx, fom.hy
    for j in range(1, ny + 1):
        for i in range(1, nx + 1):
            p = (j - 1) * nx + (i - 1)
            for F, k in ((U, p), (V, nx * ny + p)):
                fx = (F[j, i + 1] - F[j, i - 1]) / (2 * hx)
                fy = (F[j + 1, i] - F[j - 1, i]) / (2 * hy)
                lap = (F[j, i + 1] - 2 * F[j, i] + F[j, i - 1]) / hx ** 2 + (F[j + 1, i] - 2 * F[j, i] + F[j - 1, i]) / hy ** 2
                expect = -U[j, i] * fx - V[j, i] * fy + NU * lap
                assert np.isclose(res[k], expect, rtol=1e-12, atol=1e-12)


def test_jacobian_exact_central_difference():
    """r is quadratic in x, so a central difference of any step equals J v up to rounding."""
    fom = Burgers(7, 5, NU)
    mu = (0.97, 1.04)
    r = np.random.default_rng(2)
    x = r.standard_normal(70) * 0.2
    J = fom.jacobian(x, mu)
    for _ in range(3):
        d = r.standard_normal(70)
        eps = 0.5
        fd = (fom.residual(x + eps * d, mu) - fom.residual(x - eps * d, mu)) / (2 * eps)
        assert np.allclose(J @ d, fd, rtol=1e-11, atol=1e-9)


def test_fom_second_order_convergence():
    """FD solution error vs the exact solution decays like h^2 (ratio ~4 per refinement)."""
    mu = (1.0, 1.0)
    errs = []
    for n in (8, 16, 32):
        fom = Burgers(n, n, NU)
        x, hist = fom.newton(mu)
        assert hist[-1] < 1e-10
        errs.append(np.max(np.abs(x - fom.exact_state(mu))))
    rates = [errs[k] / errs[k + 1] for k in range(2)]
    assert all(3.3 < q < 4.7 for q in rates), rates


def test_truncation_error_second_order():
    """Residual of the sampled exact solution is the O(h^2) truncation error."""
    mu = (1.1, 0.9)
    t = []
    for n in (16, 32, 64, 128):
        fom = Burgers(n, n, NU)
        t.append(np.max(np.abs(fom.residual(fom.exact_state(mu), mu))))
    rates = [t[k] / t[k + 1] for k in range(3)]
    # pre-asymptotic at coarse h, approaching 4 from below
    assert rates[0] < rates[1] < rates[2] and 3.4 < rates[-1] < 4.3, rates


def test_newton_quadratic():
    fom = Burgers(16, 16, NU)
    _, hist = fom.newton((0.9, 1.1))
    h = [v for v in hist if v > 1e-11]
    # quadratic: log-ratio of successive reductions approaches 2
    assert len(hist) <= 8
    assert h[-1] < h[-2] ** 1.5 * 10
