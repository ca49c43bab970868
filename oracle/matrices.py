"""1-D and assembled 2-D matrices of the discrete operators (oracle, FP64).

Test infrastructure only (see the package header).

Sec. 3.1, "Matrix formulation": the 1-D mass, stiffness and advection
matrices are
    M_{ik} = int B_i B_k,   K_{ik} = int B_i' B_k',   G_{ik} = int B_i B_k'
with the row index i belonging to the test function (reading: the paper
prints G with the derivative on the first index; with the advection term
(b dT/dx, v) of the variational form the derivative falls on the trial
function, so G 1 = 0 row by row).

The 2-D operators of the schemes are assembled here by 2-D Gauss quadrature
of the bilinear form
    a(u, v) = m (u, v) + k_x (u_x, v_x) + k_y (u_y, v_y) + g_x (u_x, v) + g_y (u_y, v)
over every element, with the tensor-product basis B_k(x) B_l(y) evaluated
point by point.  No Kronecker product is used to build them; the tests
check that they equal the Kronecker products of the 1-D matrices.

Unknowns are ordered row-major: index j*Nx + i for coefficient (i, j),
i along x.

Parity: pinned by exact rational integration (sympy) of M, K, G, by the
closed-form interior rows (cardinal B-spline values) and by K 1 = G 1 = 0
(tests/test_oracle_basis.py, tests/test_oracle_matrices.py).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .bspline import ElementTables


def matrices_1d(tab: ElementTables):
    """Return (M, K, G) as CSR matrices of size N x N, assembled element by element."""
    n, p, N = tab.n, tab.p, tab.N
    rows, cols, vm, vk, vg = [], [], [], [], []
    e = np.arange(n)
    for a in range(p + 1):  # test
        for b in range(p + 1):  # trial
            rows.append(e + a)
            cols.append(e + b)
            vm.append(np.einsum("q,eq,eq->e", tab.w, tab.B[:, :, a], tab.B[:, :, b]))
            vk.append(np.einsum("q,eq,eq->e", tab.w, tab.D[:, :, a], tab.D[:, :, b]))
            vg.append(np.einsum("q,eq,eq->e", tab.w, tab.B[:, :, a], tab.D[:, :, b]))
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    M = sp.coo_matrix((np.concatenate(vm), (r, c)), shape=(N, N)).tocsr()
    K = sp.coo_matrix((np.concatenate(vk), (r, c)), shape=(N, N)).tocsr()
    G = sp.coo_matrix((np.concatenate(vg), (r, c)), shape=(N, N)).tocsr()
    return M, K, G


def assemble_2d(tx: ElementTables, ty: ElementTables, m=0.0, kx=0.0, ky=0.0, gx=0.0, gy=0.0):
    """Assemble a(u, v) on the tensor-product space by 2-D Gauss quadrature (CSR, row-major dofs)."""
    p = tx.p
    nx, ny = tx.n, ty.n
    Nx, Ny = tx.N, ty.N
    W = ty.w[:, None] * tx.w[None, :]  # (qb, qa)
    ex = np.arange(nx)[None, :]
    ey = np.arange(ny)[:, None]
    rows, cols, vals = [], [], []
    for lj in range(p + 1):
        for li in range(p + 1):
            # test function B_{ex+li}(x) B_{ey+lj}(y) at every element point: (ny, nx, qb, qa)
            v = ty.B[:, None, :, None, lj] * tx.B[None, :, None, :, li]
            vx = ty.B[:, None, :, None, lj] * tx.D[None, :, None, :, li]
            vy = ty.D[:, None, :, None, lj] * tx.B[None, :, None, :, li]
            for ll in range(p + 1):
                for lk in range(p + 1):
                    u = ty.B[:, None, :, None, ll] * tx.B[None, :, None, :, lk]
                    ux = ty.B[:, None, :, None, ll] * tx.D[None, :, None, :, lk]
                    uy = ty.D[:, None, :, None, ll] * tx.B[None, :, None, :, lk]
                    integrand = m * u * v + kx * ux * vx + ky * uy * vy + gx * ux * v + gy * uy * v
                    val = np.einsum("ab,yxab->yx", W, integrand)
                    r = (ey + lj) * Nx + (ex + li)
                    c = (ey + ll) * Nx + (ex + lk)
                    rows.append(np.broadcast_to(r, val.shape).ravel())
                    cols.append(np.broadcast_to(c, val.shape).ravel())
                    vals.append(val.ravel())
    n = Nx * Ny
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, n)).tocsr()


def to_banded(A: sp.spmatrix, p: int) -> np.ndarray:
    """Dense (2p+1, N) band storage for scipy.linalg.solve_banded: ab[p + i - j, j] = A[i, j]."""
    A = A.tocoo()
    N = A.shape[0]
    ab = np.zeros((2 * p + 1, N))
    ab[p + A.row - A.col, A.col] = A.data
    return ab
