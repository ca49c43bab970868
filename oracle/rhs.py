"""Right-hand-side load vectors by a plain element loop (oracle, FP64).

Test infrastructure only (see the package header).

What it computes (Sec. 3, normalised form and Eq. termsPR; Sec. 3.1
variational form; Sec. 7 listing "compute_rhs"):

  F_ij   = sum_e sum_pts W [ s B_i B_j  -  c_W (b'.grad T) B_i B_j
                            + q (T_x B_i'(x) B_j(y) + T_y B_i(x) B_j'(y)) ]
  Phi_ij = sum_e sum_pts W (phi - tau k_f E phi) B_i B_j

with T, grad T and phi interpolated at each Gauss point from the
coefficients of the element, (s, E, q) the pointwise terms of
`physics.source_terms` (heat release, Newton forcing, vertical radiation;
q = -C_nld T^3 from the weak form of div(C_nld T^3 grad T) with the natural
boundary condition of Sec. 2.1 "Boundary conditions"), W the product of the
Gauss weights and element lengths, and b' the explicit, spatially varying
part of the wind (reading: the constant mean wind is implicit in the 1-D
operators; the variation, which has no Kronecker structure, is treated like
the other nonlinear terms).  Phi is the load vector of the explicit Euler
fuel update of the listing, with tau the full time step.

The wind variation is b'_c(x, y) = sum_r f_{c,r}(x) g_{c,r}(y), each factor a
1-D spline of the same degree and knots.

The loop visits element rows one block at a time and, inside a block, every
element, every local basis pair and every Gauss point; nothing is
sum-factorised.

Parity: pinned through the step tests (uniform states, ambient steady
state, closed-form decay with F switched off, mirror symmetry) and
tests/test_oracle_rhs.py (brute-force point-by-point integration on a tiny
grid).
"""
from __future__ import annotations

import numpy as np

from .bspline import ElementTables
from .physics import Params, derived_constants, source_terms


def _factor_at_points(tab: ElementTables, coef: np.ndarray) -> np.ndarray:
    """1-D spline with coefficients `coef` (R, N) at the Gauss points: (R, n, q)."""
    p = tab.p
    out = np.zeros((coef.shape[0], tab.n, tab.q))
    for k in range(p + 1):
        out += coef[:, k:k + tab.n, None] * tab.B[None, :, :, k]
    return out


def load_vectors(tx: ElementTables, ty: ElementTables, T: np.ndarray, phi: np.ndarray, prm: Params,
                 tau: float, wind_factors=None, block_rows: int = 64):
    """Return (F, Phi), both (Ny, Nx), for coefficient arrays T and phi of shape (Ny, Nx)."""
    c = derived_constants(prm)
    p, q = tx.p, tx.q
    nx, ny = tx.n, ty.n
    T = np.asarray(T, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    F = np.zeros_like(T)
    Phi = np.zeros_like(T)
    W = ty.w[None, None, :, None] * tx.w[None, None, None, :]
    if wind_factors is not None:
        fx, gx, fy, gy = wind_factors
        fxq = _factor_at_points(tx, np.atleast_2d(fx))
        gxq = _factor_at_points(ty, np.atleast_2d(gx))
        fyq = _factor_at_points(tx, np.atleast_2d(fy))
        gyq = _factor_at_points(ty, np.atleast_2d(gy))
    for y0 in range(0, ny, block_rows):
        y1 = min(ny, y0 + block_rows)
        shape = (y1 - y0, nx, q, q)  # (ey, ex, b, a)
        Tv = np.zeros(shape)
        Tx = np.zeros(shape)
        Ty = np.zeros(shape)
        Pv = np.zeros(shape)
        for l in range(p + 1):
            by = ty.B[y0:y1, None, :, None, l]
            dy = ty.D[y0:y1, None, :, None, l]
            for k in range(p + 1):
                bx = tx.B[None, :, None, :, k]
                dx = tx.D[None, :, None, :, k]
                cT = T[y0 + l:y1 + l, k:k + nx][:, :, None, None]
                cP = phi[y0 + l:y1 + l, k:k + nx][:, :, None, None]
                Tv += cT * by * bx
                Tx += cT * by * dx
                Ty += cT * dy * bx
                Pv += cP * by * bx
        s, E, qd = source_terms(Tv, Pv, prm)
        if wind_factors is not None:
            bpx = np.einsum("ryb,rxa->yxba", gxq[:, y0:y1, :], fxq)
            bpy = np.einsum("ryb,rxa->yxba", gyq[:, y0:y1, :], fyq)
            s = s - c["c_W"] * (bpx * Tx + bpy * Ty)
        fuel_val = Pv - tau * c["k_f"] * E * Pv
        for l in range(p + 1):
            by = ty.B[y0:y1, None, :, None, l]
            dy = ty.D[y0:y1, None, :, None, l]
            for k in range(p + 1):
                bx = tx.B[None, :, None, :, k]
                dx = tx.D[None, :, None, :, k]
                f = W * (s * by * bx + qd * Tx * by * dx + qd * Ty * dy * bx)
                g = W * fuel_val * by * bx
                F[y0 + l:y1 + l, k:k + nx] += f.sum(axis=(2, 3))
                Phi[y0 + l:y1 + l, k:k + nx] += g.sum(axis=(2, 3))
    return F, Phi
