"""One time step of the Peaceman-Rachford and Strang/Crank-Nicolson schemes (oracle, FP64).

Test infrastructure only (see the package header).

Notation: theta-scaled directional operators built from the 1-D matrices
of Sec. 3.1 and the normalised coefficients of Sec. 3,
    X(theta, +-) = M^x +- theta (C_d K^x + c_W b_x G^x + c_chi M^x)
    Y(theta, +-) = M^y +- theta (C_d K^y + c_W b_y G^y)
(the reaction term only in the x operator, as Eq. termsPR writes L_1 and
L_2; b = (b_x, b_y) the constant mean wind).  "X (x) M^y" is the 2-D
operator with X acting along x and M^y along y.

Peaceman-Rachford (Eq. matrixPR; reading: F^{n+1/2} is the explicit
F(T^n, phi^n), one evaluation shared by both substeps, `F_timing='once'`;
'per_substep' uses F(T*) in the second):
    (X(tau/2,+) (x) M^y) T*      = (M^x (x) Y(tau/2,-)) T^n + tau/2 F
    (M^x (x) Y(tau/2,+)) T^{n+1} = (X(tau/2,-) (x) M^y) T*  + tau/2 F

Strang + Crank-Nicolson (Eq. matrixCN; explicit reading of the F terms:
tau/4 (F^{n+1/2} + F^n) -> tau/2 F(T^n), tau/4 (F^{n+1} + F^{n+1/2}) -> tau/2 F(T**)):
    (X(tau/4,+) (x) M^y) T*      = (X(tau/4,-) (x) M^y) T^n + tau/2 F(T^n)
    (M^x (x) Y(tau/2,+)) T**     = (M^x (x) Y(tau/2,-)) T*
    (X(tau/4,+) (x) M^y) T^{n+1} = (X(tau/4,-) (x) M^y) T** + tau/2 F(T**)

Explicit L2 projection (the explicit dynamics of Sec. 6, the scheme the Sec. 7
listing runs; the comparator of the convergence study): every term at T^n,
    (M^x (x) M^y) T^{n+1} = (M^x (x) M^y) T^n - tau (A_x (x) M^y + M^x (x) A_y) T^n + tau F(T^n)
with A_x = C_d K^x + c_W b_x G^x + c_chi M^x and A_y = C_d K^y + c_W b_y G^y, written
with the operators above as (X(tau,-) (x) M^y) T + (M^x (x) Y(tau,-)) T - (M^x (x) M^y) T.

With a manufactured solution (oracle.mms), its forcing load vector, evaluated at the start
time of the step, is added to every F of the step.

Fuel (listing "compute_rhs"): (M^x (x) M^y) phi^{n+1} = Phi(T^n, phi^n), once
per step with the full tau; phi^n is the fuel seen by every F of the step.

Modes:
  'direct': every 2-D operator is assembled by 2-D quadrature
            (matrices.assemble_2d), applied as a sparse matrix and solved by
            sparse LU with partial pivoting (scipy.sparse.linalg.splu).
  'ads':    the same operators applied and solved through their 1-D factors:
            (A (x) B) T = B T A^T, and (A (x) B)^{-1} R by banded solves with
            partial pivoting (scipy.linalg.solve_banded) along y then x
            (Sec. 4: N_y solves of size N_x and N_x solves of size N_y).

Parity: 'ads' is pinned to 'direct' (<= 1e-12) and 'direct' to dense
brute force; both to the closed-form decay of discrete eigenmodes, to the
uniform-state recurrences, the ambient steady state, heat-content
conservation and mirror symmetry (tests/test_oracle_step.py).  The full
nonlinear front beyond these checks is "parity unpinned".
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from .bspline import ElementTables
from .matrices import assemble_2d, matrices_1d, to_banded
from .physics import Params, derived_constants
from .rhs import load_vectors


class Problem:
    """A grid, its operators and the scheme settings; `step` advances (T, phi) by one time step."""

    def __init__(self, nx, ny, p, Lx, Ly, dt, wind=(0.0, 0.0), wind_factors=None, prm: Params = None,
                 scheme: str = "pr", mode: str = "direct", forcing=None, t0: float = 0.0):
        assert scheme in ("pr", "strang", "explicit")
        assert mode in ("direct", "ads")
        self.prm = prm if prm is not None else Params()
        self.c = derived_constants(self.prm)
        self.tx = ElementTables(nx, p, Lx)
        self.ty = ElementTables(ny, p, Ly)
        self.p = p
        self.dt = float(dt)
        self.wind = (float(wind[0]), float(wind[1]))
        self.wind_factors = wind_factors
        self.scheme = scheme
        self.mode = mode
        # manufactured-solution forcing (oracle.mms.Manufactured) added to every F of a step,
        # evaluated at the step's start time self.t
        self.forcing = forcing
        self.t = float(t0)
        self.Mx, self.Kx, self.Gx = matrices_1d(self.tx)
        self.My, self.Ky, self.Gy = matrices_1d(self.ty)
        self._ops = {}
        self._lu = {}

    @classmethod
    def from_scenario(cls, sc, prm: Params = None, scheme="pr", mode="direct"):
        wf = None
        if sc.wind_rank:
            wf = (sc.fx, sc.gx, sc.fy, sc.gy)
        return cls(sc.nx, sc.ny, sc.p, sc.Lx, sc.Ly, sc.dt, sc.wind, wf, prm, scheme, mode)

    # ---- directional operators -------------------------------------------------
    def x_op(self, theta, sign):
        c = self.c
        return self.Mx + sign * theta * (c["C_d"] * self.Kx + c["c_W"] * self.wind[0] * self.Gx
                                         + c["c_chi"] * self.Mx)

    def y_op(self, theta, sign):
        c = self.c
        return self.My + sign * theta * (c["C_d"] * self.Ky + c["c_W"] * self.wind[1] * self.Gy)

    def factors(self, key):
        """1-D factors (A along x, B along y) of the 2-D operator named by key."""
        kind = key[0]
        if kind == "x":
            return self.x_op(key[1], key[2]), self.My
        if kind == "y":
            return self.Mx, self.y_op(key[1], key[2])
        return self.Mx, self.My

    def op2d(self, key):
        """2-D operator assembled by quadrature of its bilinear form."""
        if key not in self._ops:
            c = self.c
            kind = key[0]
            if kind == "x":
                th, sg = key[1], key[2]
                A = assemble_2d(self.tx, self.ty, m=1.0 + sg * th * c["c_chi"], kx=sg * th * c["C_d"],
                                gx=sg * th * c["c_W"] * self.wind[0])
            elif kind == "y":
                th, sg = key[1], key[2]
                A = assemble_2d(self.tx, self.ty, m=1.0, ky=sg * th * c["C_d"],
                                gy=sg * th * c["c_W"] * self.wind[1])
            else:
                A = assemble_2d(self.tx, self.ty, m=1.0)
            self._ops[key] = A
        return self._ops[key]

    def apply(self, key, T):
        if self.mode == "direct":
            return (self.op2d(key) @ T.ravel()).reshape(T.shape)
        A, B = self.factors(key)
        return np.asarray(B @ (A @ T.T).T)

    def solve(self, key, R):
        if self.mode == "direct":
            if key not in self._lu:
                self._lu[key] = spla.splu(self.op2d(key).tocsc())
            return self._lu[key].solve(R.ravel()).reshape(R.shape)
        A, B = self.factors(key)
        p = self.p
        Y = sla.solve_banded((p, p), to_banded(B, p), R)  # along y: every column of R
        return sla.solve_banded((p, p), to_banded(A, p), Y.T).T  # along x: every row

    def load(self, T, phi):
        F, Phi = load_vectors(self.tx, self.ty, T, phi, self.prm, self.dt, self.wind_factors)
        if self.forcing is not None:
            F = F + self.forcing.load(self.tx, self.ty, self.t, self.c, self.wind)
        return F, Phi

    # ---- schemes -----------------------------------------------------------------
    def step(self, T, phi):
        if self.scheme == "explicit":
            out = self.explicit_step(T, phi)
        elif self.scheme == "pr":
            out = self.pr_step(T, phi)
        else:
            out = self.strang_step(T, phi)
        self.t += self.dt
        return out

    def pr_step(self, T, phi):
        th = 0.5 * self.dt
        F, Phi = self.load(T, phi)
        R1 = self.apply(("y", th, -1.0), T) + th * F
        Ts = self.solve(("x", th, 1.0), R1)
        F2 = F if self.prm.F_timing == "once" else self.load(Ts, phi)[0]
        R2 = self.apply(("x", th, -1.0), Ts) + th * F2
        Tn = self.solve(("y", th, 1.0), R2)
        phin = self.solve(("m",), Phi)
        return Tn, phin

    def strang_step(self, T, phi):
        tau = self.dt
        qx = 0.25 * tau
        hy = 0.5 * tau
        F, Phi = self.load(T, phi)
        Ts = self.solve(("x", qx, 1.0), self.apply(("x", qx, -1.0), T) + 0.5 * tau * F)
        Tss = self.solve(("y", hy, 1.0), self.apply(("y", hy, -1.0), Ts))
        F3, _ = self.load(Tss, phi)
        Tn = self.solve(("x", qx, 1.0), self.apply(("x", qx, -1.0), Tss) + 0.5 * tau * F3)
        phin = self.solve(("m",), Phi)
        return Tn, phin

    def explicit_step(self, T, phi):
        tau = self.dt
        F, Phi = self.load(T, phi)
        R = (self.apply(("x", tau, -1.0), T) + self.apply(("y", tau, -1.0), T) - self.apply(("m",), T)
             + tau * F)
        return self.solve(("m",), R), self.solve(("m",), Phi)

    def run(self, T, phi, steps):
        T = np.array(T, dtype=np.float64)
        phi = np.array(phi, dtype=np.float64)
        for _ in range(steps):
            T, phi = self.step(T, phi)
        return T, phi
