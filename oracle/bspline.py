"""Open uniform B-spline spaces and Gauss-Legendre tables (oracle, FP64).

Test infrastructure only (see the package header).

The discrete space of Sec. 3.1 ("Matrix formulation") is the tensor product
V_h = V_h^x (x) V_h^y of 1-D B-spline spaces of degree p.  The paper's code
uses open (clamped) uniform knots with C^{p-1} continuity (Sec. 1, Sec. 5:
"fire <N> <p>"): n elements of size h = L/n, N = n + p basis functions.

Basis values follow the Cox-de Boor recursion written on global knot
indices:
    N_{i,0}(x) = 1 on [t_i, t_{i+1}), else 0
    N_{i,k}(x) = (x - t_i)/(t_{i+k} - t_i) N_{i,k-1}(x)
               + (t_{i+k+1} - x)/(t_{i+k+1} - t_{i+1}) N_{i+1,k-1}(x)      (0/0 := 0)
    N'_{i,p}(x) = p N_{i,p-1}(x)/(t_{i+p} - t_i) - p N_{i+1,p-1}(x)/(t_{i+p+1} - t_{i+1})
evaluated only for the p+1 indices that can be nonzero on the element that
holds x (all other terms of the recursion are identically zero there).

Quadrature: q = p + 1 Gauss-Legendre points per element and direction
(reading; the paper's listing loops over `quad_points()` without stating
the rule).  This integrates the mass, stiffness and advection matrices
exactly.

Parity: pinned by partition of unity, derivative sums, nonnegativity and
by exact rational integration of the same knot vectors with sympy
(tests/test_oracle_basis.py).
"""
from __future__ import annotations

import numpy as np


def knots(n: int, p: int, L: float) -> np.ndarray:
    """Open uniform knot vector with n elements of degree p on [0, L] (length n + 2p + 1)."""
    h = L / n
    inner = np.arange(n + 1, dtype=np.float64) * h
    inner[-1] = L
    return np.concatenate([np.zeros(p), inner, np.full(p, float(L))])


def gauss01(q: int):
    """Gauss-Legendre nodes and weights on [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(q)
    return 0.5 * (x + 1.0), 0.5 * w


def _ratio(num, den):
    den = np.asarray(den, dtype=np.float64)
    safe = np.where(den != 0.0, den, 1.0)
    return np.where(den != 0.0, num / safe, 0.0)


def eval_local(t: np.ndarray, p: int, e, x):
    """Values and first derivatives of B_{e}, ..., B_{e+p} at x, where x lies in element e.

    `e` and `x` broadcast together; the result has shape x.shape + (p+1,).
    Local index l corresponds to the global basis index e + l.
    """
    e = np.asarray(e)
    x = np.asarray(x, dtype=np.float64)
    e, x = np.broadcast_arrays(e, x)
    span = e + p  # t[span] <= x < t[span+1]
    # N[l] holds N_{span-k+l, k}
    N = [np.ones_like(x)]
    prev = None
    for k in range(1, p + 1):
        new = []
        for l in range(k + 1):
            i = span - k + l
            v = np.zeros_like(x)
            if l - 1 >= 0:  # N_{i,k-1} is entry l-1 of degree k-1
                v = v + _ratio(x - t[i], t[i + k] - t[i]) * N[l - 1]
            if l <= k - 1:  # N_{i+1,k-1} is entry l of degree k-1
                v = v + _ratio(t[i + k + 1] - x, t[i + k + 1] - t[i + 1]) * N[l]
            new.append(v)
        prev = N
        N = new
    vals = np.stack(N, axis=-1)
    if p == 0:
        return vals, np.zeros_like(vals)
    ders = []
    for l in range(p + 1):
        i = span - p + l
        d = np.zeros_like(x)
        if l - 1 >= 0:
            d = d + p * _ratio(prev[l - 1], t[i + p] - t[i])
        if l <= p - 1:
            d = d - p * _ratio(prev[l], t[i + p + 1] - t[i + 1])
        ders.append(d)
    return vals, np.stack(ders, axis=-1)


def element_of(x, n: int, L: float):
    """Element index holding x (the right end belongs to the last element)."""
    e = np.floor(np.asarray(x, dtype=np.float64) / (L / n)).astype(np.int64)
    return np.clip(e, 0, n - 1)


class ElementTables:
    """Gauss points, weights (times element length) and basis tables of one direction."""

    def __init__(self, n: int, p: int, L: float):
        self.n, self.p, self.L = n, p, float(L)
        self.N = n + p
        self.h = self.L / n
        self.q = p + 1
        self.t = knots(n, p, L)
        xi, w = gauss01(self.q)
        e = np.arange(n)[:, None]
        self.x = self.t[e + p] + xi[None, :] * self.h  # (n, q) physical points
        self.w = w * self.h  # (q,) weights including the Jacobian
        self.B, self.D = eval_local(self.t, p, np.broadcast_to(e, self.x.shape), self.x)  # (n, q, p+1)


def element_tables(n: int, p: int, L: float) -> ElementTables:
    return ElementTables(n, p, L)
