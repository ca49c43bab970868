"""Pins of the oracle's B-spline basis and 1-D matrices against mathematics that does not use it.

* partition of unity, zero derivative sum and nonnegativity at random points;
* exact rational integration (sympy's own B-spline construction) of M, K, G;
* the closed-form interior rows of M (values of the cardinal B-spline of
  degree 2p+1 at the integers, times h);
* integral identities: M 1 = int B_i = (t_{i+p+1} - t_i)/(p+1), K 1 = 0,
  G 1 = 0 and G + G^T = e_last e_last^T - e_0 e_0^T (integration by parts);
* the Gauss rule: closed-form nodes and weights of the 1- to 3-point rules, exactness up to degree
  2q - 1 and the closed-form remainder at degree 2q.
"""
import numpy as np
import pytest

from oracle.bspline import ElementTables, element_of, eval_local, knots
from oracle.matrices import matrices_1d


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("n", [1, 2, 5, 17])
def test_partition_of_unity(p, n):
    L = 3.7
    rng = np.random.default_rng(10 * p + n)
    x = np.concatenate([rng.uniform(0, L, 200), [0.0, L]])
    e = element_of(x, n, L)
    v, d = eval_local(knots(n, p, L), p, e, x)
    assert np.allclose(v.sum(-1), 1.0, atol=1e-14, rtol=0)
    assert np.allclose(d.sum(-1), 0.0, atol=1e-12 * n / L, rtol=0)
    assert (v >= -1e-15).all()


def test_derivative_matches_finite_difference():
    n, p, L = 7, 3, 2.0
    t = knots(n, p, L)
    x = np.linspace(0.05, L - 0.05, 41)
    e = element_of(x, n, L)
    hstep = 1e-6
    v1, _ = eval_local(t, p, e, x + hstep)
    v0, _ = eval_local(t, p, e, x - hstep)
    _, d = eval_local(t, p, e, x)
    # points stay inside their element (none is within 1e-6 of a knot)
    assert np.allclose((v1 - v0) / (2 * hstep), d, atol=1e-6)


def _sympy_matrices(n, p):
    sy = pytest.importorskip("sympy")
    x = sy.Symbol("x")
    kn = [0] * p + list(range(n + 1)) + [n] * p
    B = sy.bspline_basis_set(p, kn, x)
    iv = [(kn[i], kn[i + 1]) for i in range(len(kn) - 1) if kn[i] < kn[i + 1]]

    def pieces(f):
        out = []
        for a, b in iv:
            mid = sy.Rational(a + b, 2)
            for expr, cond in f.args:
                if cond.subs(x, mid) == True:  # noqa: E712
                    out.append(sy.Poly(expr, x))
                    break
        return out

    P = [pieces(b) for b in B]
    N = len(B)

    def integ(i, k, di, dk):
        s = sy.Integer(0)
        for m, (a, b) in enumerate(iv):
            pi = P[i][m].diff(x) if di else P[i][m]
            pk = P[k][m].diff(x) if dk else P[k][m]
            F = (pi * pk).integrate()
            s += F.eval(b) - F.eval(a)
        return float(s)

    M = np.array([[integ(i, k, 0, 0) for k in range(N)] for i in range(N)])
    K = np.array([[integ(i, k, 1, 1) for k in range(N)] for i in range(N)])
    G = np.array([[integ(i, k, 0, 1) for k in range(N)] for i in range(N)])
    return M, K, G


@pytest.mark.parametrize("n,p", [(4, 1), (6, 2), (7, 3)])
def test_matrices_equal_exact_rational_integration(n, p):
    Ms, Ks, Gs = _sympy_matrices(n, p)
    M, K, G = matrices_1d(ElementTables(n, p, float(n)))  # h = 1 on [0, n]
    assert np.allclose(M.toarray(), Ms, atol=1e-14, rtol=0)
    assert np.allclose(K.toarray(), Ks, atol=1e-13, rtol=0)
    assert np.allclose(G.toarray(), Gs, atol=1e-14, rtol=0)


@pytest.mark.parametrize("p,row", [(2, [1, 26, 66, 26, 1]), (3, [1, 120, 1191, 2416, 1191, 120, 1])])
def test_mass_interior_row_closed_form(p, row):
    # h * (cardinal B-spline of degree 2p+1 at the integers); 120 = 5!, 5040 = 7!
    n, L = 20, 31.25
    tab = ElementTables(n, p, L)
    M, _, _ = matrices_1d(tab)
    denom = {2: 120.0, 3: 5040.0}[p]
    expect = tab.h * np.array(row) / denom
    Md = M.toarray()
    for i in range(2 * p, tab.N - 2 * p):
        assert np.allclose(Md[i, i - p:i + p + 1], expect, rtol=1e-13, atol=0)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_integral_identities(p):
    n, L = 9, 14.0625
    tab = ElementTables(n, p, L)
    M, K, G = matrices_1d(tab)
    one = np.ones(tab.N)
    t = tab.t
    integ = np.array([(t[i + p + 1] - t[i]) / (p + 1) for i in range(tab.N)])
    assert np.allclose(M @ one, integ, rtol=1e-13)
    assert abs(M.sum() - L) < 1e-12 * L
    assert np.abs(K @ one).max() < 1e-13
    assert np.abs(G @ one).max() < 1e-14
    S = (G + G.T).toarray()
    E = np.zeros_like(S)
    E[0, 0] = -1.0
    E[-1, -1] = 1.0
    assert np.allclose(S, E, atol=1e-13)
    # G's column sums are the boundary jumps of each B_k, which fixes its orientation
    colsum = one @ G.toarray()
    jump = np.zeros(tab.N)
    jump[0], jump[-1] = -1.0, 1.0
    assert np.allclose(colsum, jump, atol=1e-13)


def test_neumann_eigenvalues_converge():
    # generalised eigenvalues of (K, M) approach the Neumann Laplacian's (k pi / L)^2 with refinement
    sla = pytest.importorskip("scipy.linalg")
    L = 100.0
    errs = []
    for n in (8, 16, 32):
        tab = ElementTables(n, 2, L)
        M, K, _ = matrices_1d(tab)
        lam = sla.eigh(K.toarray(), M.toarray(), eigvals_only=True)
        assert abs(lam[0]) < 1e-10
        errs.append(abs(lam[3] - (3 * np.pi / L) ** 2) / (3 * np.pi / L) ** 2)
    # quadratic splines: eigenvalue error O(h^4)
    assert errs[1] < errs[0] / 10 and errs[2] < errs[1] / 10


def test_gauss_rule_closed_forms_and_exactness():
    # nodes and weights of the 1-, 2- and 3-point rules on [0, 1] in closed form (roots of the
    # shifted Legendre polynomials), and exactness of the q-point rule for x^k, k <= 2q - 1
    from oracle.bspline import gauss01

    x, w = gauss01(1)
    assert np.allclose(x, [0.5], rtol=0, atol=1e-15) and np.allclose(w, [1.0], rtol=0, atol=1e-15)
    x, w = gauss01(2)
    d = 0.5 / np.sqrt(3.0)
    assert np.allclose(np.sort(x), [0.5 - d, 0.5 + d], rtol=0, atol=1e-15)
    assert np.allclose(w, [0.5, 0.5], rtol=0, atol=1e-15)
    x, w = gauss01(3)
    d = 0.5 * np.sqrt(0.6)
    order = np.argsort(x)
    assert np.allclose(x[order], [0.5 - d, 0.5, 0.5 + d], rtol=0, atol=1e-15)
    assert np.allclose(w[order], [5 / 18, 4 / 9, 5 / 18], rtol=0, atol=1e-15)
    for q in range(1, 8):
        x, w = gauss01(q)
        for k in range(2 * q):
            assert abs((w * x ** k).sum() - 1.0 / (k + 1)) <= 1e-14, (q, k)
        # x^(2q) leaves the rule's remainder (q!)^4 / ((2q+1) ((2q)!)^2) (its (2q)-th derivative
        # is (2q)!): the rule has degree exactly 2q - 1
        from math import factorial
        rem = factorial(q) ** 4 / ((2 * q + 1) * factorial(2 * q) ** 2)
        assert (1.0 / (2 * q + 1) - (w * x ** (2 * q)).sum()) == pytest.approx(rem, rel=1e-8, abs=1e-16)
