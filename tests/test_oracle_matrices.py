"""Pins of the oracle's assembled 2-D operators.

* Every operator assembled by 2-D quadrature equals the Kronecker product of
  the 1-D matrices (Sec. 3.1 "Matrix formulation"), entry by entry.
* A rule with more Gauss points gives the same matrices (the integrands are
  polynomials of degree <= 2p, integrated exactly by p+1 points).
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle.bspline import ElementTables, eval_local, gauss01
from oracle.matrices import assemble_2d, matrices_1d
from oracle.physics import Params
from oracle.step import Problem


class _Tables(ElementTables):
    """The same tables with a q-point rule of the caller's choice."""

    def __init__(self, n, p, L, q):
        super().__init__(n, p, L)
        self.q = q
        xi, w = gauss01(q)
        e = np.arange(n)[:, None]
        self.x = self.t[e + p] + xi[None, :] * self.h
        self.w = w * self.h
        self.B, self.D = eval_local(self.t, p, np.broadcast_to(e, self.x.shape), self.x)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_assembled_equals_kronecker(p):
    nx, ny = 5, 4
    P = Problem(nx, ny, p, 7.8125, 6.25, 1e-3, wind=(1.3, -0.7), prm=Params(), mode="direct")
    for key in [("x", 5e-4, 1.0), ("x", 2.5e-4, -1.0), ("y", 5e-4, 1.0), ("y", 5e-4, -1.0), ("m",)]:
        A, B = P.factors(key)
        K = sp.kron(B, A).toarray()
        D = P.op2d(key).toarray()
        assert np.allclose(D, K, rtol=0, atol=1e-14 * np.abs(K).max())


@pytest.mark.parametrize("p", [2, 3])
def test_more_gauss_points_same_matrices(p):
    n, L = 6, 9.375
    a = matrices_1d(ElementTables(n, p, L))
    b = matrices_1d(_Tables(n, p, L, p + 3))
    for A, B in zip(a, b):
        assert np.allclose(A.toarray(), B.toarray(), atol=1e-14, rtol=0)
    tx, ty = ElementTables(n, p, L), ElementTables(n - 1, p, L)
    tx2, ty2 = _Tables(n, p, L, p + 2), _Tables(n - 1, p, L, p + 2)
    kw = dict(m=1.1, kx=0.3, ky=0.2, gx=0.05, gy=-0.07)
    A1 = assemble_2d(tx, ty, **kw).toarray()
    A2 = assemble_2d(tx2, ty2, **kw).toarray()
    assert np.allclose(A1, A2, atol=1e-14, rtol=0)
