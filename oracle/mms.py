"""Manufactured solution of the convergence study (oracle, FP64).

Test infrastructure only (see the package header).

Sec. 6, "Stability and order of the time integration scheme": on [0, 100]^2 the
exact solution is

  u*(x, y, t) = 300 + 80 u_{1,1,3} + 30 u_{2,1,5} + 110 u_{2,2,1.5},
  u_{n,m,lambda} = (1 - cos(2 pi n x / L_x)) (1 - cos(2 pi m y / L_y)) exp(-lambda t)

(reading: n and m are the wave numbers of the two cosines, which the printed
formula leaves out; every mode has zero normal derivative on the boundary, the
zero-Neumann condition the paper states), and a forcing f makes it solve the
model.  With the operators of the schemes (Sec. 3, normalised form) the model is

  u_t = C_d lap u - c_W b.grad u - c_chi u + N(u) + f,
  N(u) = c_chi T_amb + c_rad (T_amb^4 - u^4) + div(C_nld u^3 grad u),

so f = u_t - C_d lap u + c_W b.grad u + c_chi u - N(u) evaluated at u*, with
div(u^3 grad u) = u^3 lap u + 3 u^2 |grad u|^2.  The study runs without
combustion (K_ign = 0: u* exceeds T_ig while the fuel would evolve) and without
wind variation; the "linear" problem also switches off C_nld and c_rad
(sigma = 0).  f enters the explicit load vector F of every scheme, evaluated at
the time of the step's start (reading, as for the other explicit terms).

Functions:
  fields(x, y, t)            u, u_t, u_x, u_y, u_xx, u_yy
  forcing(x, y, t, c, wind)  f at points (c: derived constants)
  load(tx, ty, t, c, wind)   int f B_i(x) B_j(y), element loop with the q-point Gauss rule of F
  project(tx, ty, t)         coefficients of the L2 projection of u*(., t) (initial state)
  l2_norms(tx, ty, T, t)     (||u_h - u*||, ||u*||) in L2, by a (p+4)-point Gauss rule
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .bspline import eval_local, gauss01
from .matrices import matrices_1d

PAPER_MODES = ((80.0, 1, 1, 3.0), (30.0, 2, 1, 5.0), (110.0, 2, 2, 1.5))


class Manufactured:
    def __init__(self, modes=PAPER_MODES, base=300.0, Lx=100.0, Ly=100.0):
        self.modes = tuple((float(a), int(n), int(m), float(lam)) for a, n, m, lam in modes)
        self.base = float(base)
        self.Lx, self.Ly = float(Lx), float(Ly)

    def fields(self, x, y, t):
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        shape = np.broadcast(x, y).shape
        u = np.full(shape, self.base)
        ut, ux, uy, uxx, uyy = (np.zeros(shape) for _ in range(5))
        for a, n, m, lam in self.modes:
            kx = 2.0 * np.pi * n / self.Lx
            ky = 2.0 * np.pi * m / self.Ly
            e = a * np.exp(-lam * t)
            gx, gy = 1.0 - np.cos(kx * x), 1.0 - np.cos(ky * y)
            dgx, dgy = kx * np.sin(kx * x), ky * np.sin(ky * y)
            ddgx, ddgy = kx * kx * np.cos(kx * x), ky * ky * np.cos(ky * y)
            u = u + e * gx * gy
            ut = ut - lam * e * gx * gy
            ux = ux + e * dgx * gy
            uy = uy + e * gx * dgy
            uxx = uxx + e * ddgx * gy
            uyy = uyy + e * gx * ddgy
        return u, ut, ux, uy, uxx, uyy

    def forcing(self, x, y, t, c, wind):
        u, ut, ux, uy, uxx, uyy = self.fields(x, y, t)
        lap = uxx + uyy
        N = (c["c_chi"] * c["T_amb"] + c["c_rad"] * (c["T_amb"] ** 4 - u ** 4)
             + c["C_nld"] * (u ** 3 * lap + 3.0 * u ** 2 * (ux * ux + uy * uy)))
        return ut - c["C_d"] * lap + c["c_W"] * (wind[0] * ux + wind[1] * uy) + c["c_chi"] * u - N

    def load(self, tx, ty, t, c, wind):
        """int f(x, y, t) B_i(x) B_j(y) dx dy, (Ny, Nx), by the Gauss rule of the load vectors."""
        p = tx.p
        out = np.zeros((ty.N, tx.N))
        X = tx.x[None, :, None, :]  # (1, nx, 1, q)
        Y = ty.x[:, None, :, None]  # (ny, 1, q, 1)
        fv = self.forcing(X, Y, t, c, wind) * (ty.w[None, None, :, None] * tx.w[None, None, None, :])
        for l in range(p + 1):
            for k in range(p + 1):
                # element (ey, ex) adds to DOF (ey + l, ex + k)
                contrib = np.einsum("yxba,yb,xa->yx", fv, ty.B[:, :, l], tx.B[:, :, k])
                out[l:l + ty.n, k:k + tx.n] += contrib
        return out

    def project(self, tx, ty, t):
        """L2 projection of u*(., t): (M^x (x) M^y)^{-1} int u* B_i B_j (exact up to the q-point rule)."""
        p = tx.p
        rhs = np.zeros((ty.N, tx.N))
        X = tx.x[None, :, None, :]
        Y = ty.x[:, None, :, None]
        uv = self.fields(X, Y, t)[0] * (ty.w[None, None, :, None] * tx.w[None, None, None, :])
        for l in range(p + 1):
            for k in range(p + 1):
                rhs[l:l + ty.n, k:k + tx.n] += np.einsum("yxba,yb,xa->yx", uv, ty.B[:, :, l], tx.B[:, :, k])
        Mx = matrices_1d(tx)[0].toarray()
        My = matrices_1d(ty)[0].toarray()
        Z = sla.solve(My, rhs, assume_a="pos")
        return sla.solve(Mx, Z.T, assume_a="pos").T

    def l2_norms(self, tx, ty, T, t):
        """(||u_h - u*(t)||_L2, ||u*(t)||_L2) for the coefficients T, with a (p + 4)-point rule."""
        p = tx.p
        qq = p + 4
        xi, w = gauss01(qq)
        sq_err = 0.0
        sq_ref = 0.0
        ex = np.arange(tx.n)
        ey = np.arange(ty.n)
        xs = (tx.t[ex + p][:, None] + xi[None, :] * tx.h)  # (nx, qq)
        ys = (ty.t[ey + p][:, None] + xi[None, :] * ty.h)
        Bx, _ = eval_local(tx.t, p, np.broadcast_to(ex[:, None], xs.shape), xs)  # (nx, qq, p+1)
        By, _ = eval_local(ty.t, p, np.broadcast_to(ey[:, None], ys.shape), ys)
        uh = np.zeros((ty.n, tx.n, qq, qq))  # (ey, ex, b, a)
        for l in range(p + 1):
            for k in range(p + 1):
                c = T[l:l + ty.n, k:k + tx.n]
                uh += c[:, :, None, None] * By[:, None, :, None, l] * Bx[None, :, None, :, k]
        us = self.fields(xs[None, :, None, :], ys[:, None, :, None], t)[0]
        W = (w * ty.h)[None, None, :, None] * (w * tx.h)[None, None, None, :]
        sq_err = float(((uh - us) ** 2 * W).sum())
        sq_ref = float((us ** 2 * W).sum())
        return np.sqrt(sq_err), np.sqrt(sq_ref)
