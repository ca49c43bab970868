"""Pins of the manufactured solution of the convergence study (Sec. 6) and of its forcing.

* u* and its derivatives against central finite differences of u* itself;
* zero normal derivative on the boundary (the condition the paper states);
* the forcing against the model's residual at u* built from finite differences,
  with the nonlinear diffusion taken as the divergence of the flux u^3 grad u
  (not the expanded form the oracle uses);
* the forcing load vector against a brute-force integration with scipy's B-splines;
* first-order convergence in time of the PR, Strang and explicit schemes with the
  forcing switched on (the paper's conclusion), on a coarse grid;
* the study's tools: the L2 projection against an independent projection (scipy's B-splines,
  numpy's Gauss rule), exact for constants, converging at O(h^(p+1)); the reference norm against
  the closed form of the modes' integrals; the error norm against a ten-point brute force.
"""
import numpy as np
import pytest
from scipy.interpolate import BSpline

from oracle.bspline import ElementTables, gauss01, knots
from oracle.mms import Manufactured
from oracle.physics import Params, derived_constants
from oracle.step import Problem


def _consts(linear):
    prm = Params(heat_scale=0.0, sigma=0.0) if linear else Params(heat_scale=0.0)
    return prm, derived_constants(prm)


def test_derivatives_match_finite_differences():
    m = Manufactured()
    rng = np.random.default_rng(1)
    x, y, t = rng.uniform(5, 95, 20), rng.uniform(5, 95, 20), rng.uniform(0, 1, 20)
    u, ut, ux, uy, uxx, uyy = m.fields(x, y, t)
    d = 1e-4
    U = lambda a, b, c: m.fields(a, b, c)[0]  # noqa: E731
    assert np.allclose(ut, (U(x, y, t + d) - U(x, y, t - d)) / (2 * d), rtol=1e-6, atol=1e-6)
    assert np.allclose(ux, (U(x + d, y, t) - U(x - d, y, t)) / (2 * d), rtol=1e-6, atol=1e-6)
    assert np.allclose(uy, (U(x, y + d, t) - U(x, y - d, t)) / (2 * d), rtol=1e-6, atol=1e-6)
    d = 1e-3
    assert np.allclose(uxx, (U(x + d, y, t) - 2 * u + U(x - d, y, t)) / d ** 2, rtol=1e-4, atol=1e-4)
    assert np.allclose(uyy, (U(x, y + d, t) - 2 * u + U(x, y - d, t)) / d ** 2, rtol=1e-4, atol=1e-4)
    # the paper's amplitudes: u*(50, 50, 0) = 300 + 4 (80 + 30 + 110) for n = m = 1 ... the
    # wave-number-2 modes vanish at the centre: 1 - cos(2 pi) = 0
    assert abs(m.fields(50.0, 50.0, 0.0)[0] - (300.0 + 4 * 80.0)) < 1e-9


def test_zero_normal_derivative_on_the_boundary():
    m = Manufactured()
    s = np.linspace(0, 100, 11)
    for t in (0.0, 0.7):
        assert np.abs(m.fields(0.0, s, t)[2]).max() < 1e-9 and np.abs(m.fields(100.0, s, t)[2]).max() < 1e-9
        assert np.abs(m.fields(s, 0.0, t)[3]).max() < 1e-9 and np.abs(m.fields(s, 100.0, t)[3]).max() < 1e-9


@pytest.mark.parametrize("linear", [True, False])
def test_forcing_is_the_model_residual(linear):
    m = Manufactured()
    prm, c = _consts(linear)
    wind = (1.0, 0.5)
    rng = np.random.default_rng(2)
    x, y, t = rng.uniform(5, 95, 15), rng.uniform(5, 95, 15), rng.uniform(0, 1, 15)
    U = lambda a, b, s: m.fields(a, b, s)[0]  # noqa: E731
    d = 1e-3
    u = U(x, y, t)
    ut = (U(x, y, t + d) - U(x, y, t - d)) / (2 * d)
    ux = (U(x + d, y, t) - U(x - d, y, t)) / (2 * d)
    uy = (U(x, y + d, t) - U(x, y - d, t)) / (2 * d)
    lap = (U(x + d, y, t) + U(x - d, y, t) + U(x, y + d, t) + U(x, y - d, t) - 4 * u) / d ** 2

    def flux_div(a, b, s):  # div(u^3 grad u) as differences of the flux
        h = d
        fxp = U(a + h / 2, b, s) ** 3 * (U(a + h, b, s) - U(a, b, s)) / h
        fxm = U(a - h / 2, b, s) ** 3 * (U(a, b, s) - U(a - h, b, s)) / h
        fyp = U(a, b + h / 2, s) ** 3 * (U(a, b + h, s) - U(a, b, s)) / h
        fym = U(a, b - h / 2, s) ** 3 * (U(a, b, s) - U(a, b - h, s)) / h
        return (fxp - fxm + fyp - fym) / h

    resid = (ut - c["C_d"] * lap + c["c_W"] * (wind[0] * ux + wind[1] * uy) + c["c_chi"] * u
             - c["c_chi"] * c["T_amb"] - c["c_rad"] * (c["T_amb"] ** 4 - u ** 4) - c["C_nld"] * flux_div(x, y, t))
    f = m.forcing(x, y, t, c, wind)
    assert np.allclose(f, resid, rtol=1e-4, atol=1e-3 * np.abs(f).max())


def test_load_vector_matches_brute_force():
    m = Manufactured(Lx=30.0, Ly=20.0)
    nx, ny, p = 5, 4, 2
    tx, ty = ElementTables(nx, p, 30.0), ElementTables(ny, p, 20.0)
    _, c = _consts(False)
    wind = (0.3, -0.8)
    t = 0.4
    F = m.load(tx, ty, t, c, wind)
    kx, ky = knots(nx, p, 30.0), knots(ny, p, 20.0)
    xi, w = gauss01(p + 1)
    ref = np.zeros((ny + p, nx + p))
    for ey in range(ny):
        for ex in range(nx):
            xs = kx[ex + p] + xi * (30.0 / nx)
            ys = ky[ey + p] + xi * (20.0 / ny)
            W = np.outer(w * (20.0 / ny), w * (30.0 / nx))
            fv = m.forcing(xs[None, :], ys[:, None], t, c, wind) * W
            for j in range(ny + p):
                bj = BSpline.basis_element(ky[j:j + p + 2], extrapolate=False)(ys)
                bj = np.nan_to_num(bj)
                if not bj.any():
                    continue
                for i in range(nx + p):
                    bi = np.nan_to_num(BSpline.basis_element(kx[i:i + p + 2], extrapolate=False)(xs))
                    if bi.any():
                        ref[j, i] += (fv * np.outer(bj, bi)).sum()
    assert np.abs(F - ref).max() <= 1e-10 * np.abs(ref).max()


def _study_error(scheme, n, tau, linear=True):
    """Relative error over [0, 1]: sqrt(sum_n ||u_h - u*||^2) / sqrt(sum_n ||u*||^2)."""
    m = Manufactured()
    prm, _ = _consts(linear)
    P = Problem(n, n, 2, 100.0, 100.0, tau, wind=(1.0, 0.5), prm=prm, scheme=scheme, mode="ads", forcing=m)
    T = m.project(P.tx, P.ty, 0.0)
    phi = np.zeros_like(T)
    se = sr = 0.0
    steps = int(round(1.0 / tau))
    for k in range(steps):
        T, phi = P.step(T, phi)
        e, r = m.l2_norms(P.tx, P.ty, T, (k + 1) * tau)
        se += e * e
        sr += r * r
    return np.sqrt(se / sr)


@pytest.mark.parametrize("scheme", ["pr", "strang", "explicit"])
def test_first_order_in_time(scheme):
    taus = [1 / 16, 1 / 32, 1 / 64]
    errs = [_study_error(scheme, 20, tau) for tau in taus]
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert all(0.8 < r < 1.3 for r in rates), (errs, rates)


# ---- the study's projection and norms, pinned by independent code (scipy's B-splines, numpy's
# Gauss-Legendre rule, the closed form of the modes' integrals) ----------------------------------

def _open_knots(n, p, L):
    return np.r_[np.zeros(p), np.linspace(0.0, L, n + 1), np.full(p, L)]


def _gauss_points(n, L, q):
    """Points and weights of the q-point Gauss-Legendre rule on each of n equal elements of [0, L]."""
    xi, w = np.polynomial.legendre.leggauss(q)
    h = L / n
    xs = ((np.arange(n)[:, None] + 0.5 * (xi[None, :] + 1.0)) * h).ravel()
    return xs, np.tile(0.5 * h * w, n)


def _design(xs, n, p, L):
    return BSpline.design_matrix(xs, _open_knots(n, p, L), p).toarray()  # (points, n + p)


def test_projection_equals_an_independent_l2_projection():
    # rectangular domain and grid, so a transposed operand fails
    m = Manufactured(Lx=100.0, Ly=60.0)
    nx, ny, p, t = 7, 5, 2, 0.3
    tx, ty = ElementTables(nx, p, 100.0), ElementTables(ny, p, 60.0)
    C = m.project(tx, ty, t)
    xs, wx = _gauss_points(nx, 100.0, p + 1)
    ys, wy = _gauss_points(ny, 60.0, p + 1)
    Bx, By = _design(xs, nx, p, 100.0), _design(ys, ny, p, 60.0)
    Mx, My = Bx.T @ (wx[:, None] * Bx), By.T @ (wy[:, None] * By)
    U = m.fields(xs[None, :], ys[:, None], t)[0]  # (y, x)
    b = By.T @ (wy[:, None] * U * wx[None, :]) @ Bx  # int u* B_i(x) B_j(y), (Ny, Nx)
    ref = np.linalg.solve(My, np.linalg.solve(Mx, b.T).T)
    assert C.shape == (ny + p, nx + p)
    assert np.abs(C - ref).max() <= 1e-11 * np.abs(ref).max()


def test_projection_of_a_constant_is_exact():
    # B-splines sum to one: the constant's coefficients are the constant
    m = Manufactured(modes=(), base=300.0)
    tx, ty = ElementTables(6, 3, 100.0), ElementTables(4, 3, 100.0)
    C = m.project(tx, ty, 0.0)
    assert np.abs(C - 300.0).max() <= 1e-10


def test_reference_norm_matches_the_closed_form():
    # over whole periods: int (1 - cos kx) = L, int (1 - cos k x)(1 - cos k' x) = L + L/2 [k = k']
    m = Manufactured(Lx=100.0, Ly=80.0)
    t = 0.25
    tx, ty = ElementTables(20, 2, 100.0), ElementTables(16, 2, 80.0)
    _, ref = m.l2_norms(tx, ty, np.zeros((16 + 2, 20 + 2)), t)
    Lx, Ly, base = 100.0, 80.0, 300.0
    amp = [(a * np.exp(-lam * t), n, mm) for a, n, mm, lam in m.modes]
    sq = base * base * Lx * Ly + 2.0 * base * Lx * Ly * sum(e for e, _, _ in amp)
    for ea, na, ma in amp:
        for eb, nb, mb in amp:
            sq += ea * eb * (Lx + 0.5 * Lx * (na == nb)) * (Ly + 0.5 * Ly * (ma == mb))
    assert ref == pytest.approx(np.sqrt(sq), rel=1e-12)


def test_error_norm_matches_brute_force():
    m = Manufactured(Lx=100.0, Ly=60.0)
    nx, ny, p, t = 9, 6, 2, 0.1
    tx, ty = ElementTables(nx, p, 100.0), ElementTables(ny, p, 60.0)
    rng = np.random.default_rng(7)
    C = 300.0 + 50.0 * rng.standard_normal((ny + p, nx + p))
    err, _ = m.l2_norms(tx, ty, C, t)
    # ten points per element: far more accurate than the oracle's p + 4
    xs, wx = _gauss_points(nx, 100.0, 10)
    ys, wy = _gauss_points(ny, 60.0, 10)
    uh = _design(ys, ny, p, 60.0) @ C @ _design(xs, nx, p, 100.0).T
    d = uh - m.fields(xs[None, :], ys[:, None], t)[0]
    ref = np.sqrt((wy[:, None] * d * d * wx[None, :]).sum())
    assert err == pytest.approx(ref, rel=1e-9)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_projection_error_converges_at_order_p_plus_one(p):
    # the L2 projection onto splines of degree p approximates a smooth function to O(h^(p+1))
    # (grids fine enough for the asymptotic rate: at least eight elements per shortest wavelength)
    m = Manufactured()
    errs = []
    for n in (32, 64, 128):
        tx = ElementTables(n, p, 100.0)
        e, _ = m.l2_norms(tx, tx, m.project(tx, tx, 0.0), 0.0)
        errs.append(e)
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(r - (p + 1)) < 0.15 for r in rates), (errs, rates)
