"""Pin of the oracle's load vectors by brute force on a tiny grid.

The expected F and Phi are integrated point by point with pure-Python
loops, basis functions from scipy's own B-spline evaluator (every basis
function evaluated everywhere, no element-local indexing) and source terms
recomputed from the raw Table constants with the formulas of the paper's
right-hand-side listing (Sec. 7): R_C = -1e4 rho c_h h_c (M/M1) r,
r = delta A_r T exp(-T_a/T), Q_conv = chi (T_amb - T) with -chi T moved to
the implicit operator, Q_rz = sigma eps/delta_z (T_amb^4 - T^4),
q_r = -4 sigma eps delta_x T^3 grad T, fuel rate -delta 300 r fuel, all
divided by rho c_p.
"""
import math

import numpy as np
import pytest
from scipy.interpolate import BSpline

from oracle.bspline import ElementTables, gauss01
from oracle.physics import Params
from oracle.rhs import load_vectors


def _raw_source(T, phi, prm):
    inv = 1.0 / (prm.rho * prm.cp)
    delta = 1.0 if (T > prm.T_ig and phi > prm.fuel_thresh + prm.thresh_guard) else 0.0
    r = delta * prm.A_r * T * math.exp(-prm.T_a / T)
    Rc = -1e4 * prm.rho * prm.ch * prm.hc * prm.M_ratio * r * (phi if prm.scale_heat_by_fuel else 1.0)
    Qconv_explicit = prm.chi * prm.T_amb
    Qrz = prm.sigma * prm.eps / prm.delta_z * (prm.T_amb ** 4 - T ** 4)
    s = (Rc + Qconv_explicit + Qrz) * inv
    flux_coef = -4.0 * prm.sigma * prm.eps * prm.delta_x * T ** 3 * inv
    fval = -delta * 3e2 * r * phi
    return s, flux_coef, fval


@pytest.mark.parametrize("p,heat_by_fuel", [(1, False), (2, False), (3, False), (2, True)])
def test_load_vectors_brute_force(p, heat_by_fuel):
    nx, ny = 3, 2
    Lx, Ly = 4.6875, 3.125
    Nx, Ny = nx + p, ny + p
    tx, ty = ElementTables(nx, p, Lx), ElementTables(ny, p, Ly)
    rng = np.random.default_rng(3)
    T = 300.0 + 900.0 * rng.random((Ny, Nx))
    phi = rng.random((Ny, Nx))
    R = 2
    fx, gx = rng.normal(size=(R, Nx)), rng.normal(size=(R, Ny))
    fy, gy = rng.normal(size=(R, Nx)), rng.normal(size=(R, Ny))
    prm = Params(scale_heat_by_fuel=heat_by_fuel)
    tau = 1e-3
    F, Phi = load_vectors(tx, ty, T, phi, prm, tau, (fx, gx, fy, gy))

    bx = [BSpline(tx.t, np.eye(Nx)[i], p) for i in range(Nx)]
    by = [BSpline(ty.t, np.eye(Ny)[j], p) for j in range(Ny)]
    dbx = [b.derivative() for b in bx]
    dby = [b.derivative() for b in by]
    xi, w = gauss01(p + 1)
    Fe = np.zeros((Ny, Nx))
    Pe = np.zeros((Ny, Nx))
    for ey in range(ny):
        for ex in range(nx):
            for b in range(p + 1):
                for a in range(p + 1):
                    x = (ex + xi[a]) * tx.h
                    y = (ey + xi[b]) * ty.h
                    W = w[a] * w[b] * tx.h * ty.h
                    Bx = np.array([f(x) for f in bx])
                    By = np.array([f(y) for f in by])
                    Dx = np.array([f(x) for f in dbx])
                    Dy = np.array([f(y) for f in dby])
                    Tv = By @ T @ Bx
                    Tx = By @ T @ Dx
                    Ty = Dy @ T @ Bx
                    Pv = By @ phi @ Bx
                    bpx = sum((fx[r] @ Bx) * (gx[r] @ By) for r in range(R))
                    bpy = sum((fy[r] @ Bx) * (gy[r] @ By) for r in range(R))
                    s, qc, fval = _raw_source(Tv, Pv, prm)
                    s -= prm.cW * (bpx * Tx + bpy * Ty)
                    for j in range(Ny):
                        for i in range(Nx):
                            Fe[j, i] += W * (s * Bx[i] * By[j] + qc * (Tx * Dx[i] * By[j] + Ty * Bx[i] * Dy[j]))
                            Pe[j, i] += W * (Pv + tau * fval) * Bx[i] * By[j]
    assert np.allclose(F, Fe, rtol=1e-12, atol=1e-12 * np.abs(Fe).max())
    assert np.allclose(Phi, Pe, rtol=1e-12, atol=1e-12 * np.abs(Pe).max())


def test_params_match_paper_table(repo_root):
    vals = {}
    with open(f"{repo_root}/tests/golden/table_parameters.txt") as f:
        for line in f:
            line = line.split("#")[0].split()
            if len(line) >= 2:
                vals[line[0]] = line[1]
    prm = Params()
    eps = float(vals["epsilon"])
    assert prm.cp == float(vals["c_p"]) and prm.rho == float(vals["rho"])
    assert prm.kappa == float(vals["kappa"]) and prm.sigma == float(vals["sigma"])
    assert prm.eps == eps and prm.ch == float(vals["c_h"]) and prm.hc == float(vals["h_c"])
    assert prm.cW == float(vals["c_W"]) and prm.chi == float(vals["chi"])
    assert prm.T_amb == float(vals["T_amb"]) and prm.T_ig == float(vals["T_ig"])
    assert abs(prm.delta_x - 3.5e-2 / eps) < 1e-15 and abs(prm.delta_z - 1.5 * eps) < 1e-15
    assert prm.heat_scale == float(vals["heat_scale"]) and prm.fuel_rate == float(vals["fuel_rate"])
    assert prm.fuel_thresh == float(vals["fuel_thresh"]) and prm.T_a == float(vals["T_a"])


def test_source_terms_match_hand_table(repo_root):
    # s(T, phi), the reaction rate E and the fuel rate against values worked by hand from the
    # Table constants (tests/golden/source_values.txt): catches a dropped or mis-signed term, a
    # wrong constant or a wrong threshold on either side of T_ig and of the fuel threshold
    from oracle.physics import derived_constants, source_terms

    rows = []
    with open(f"{repo_root}/tests/golden/source_values.txt") as f:
        for line in f:
            line = line.split("#")[0].split()
            if len(line) == 6:
                rows.append([float(v) for v in line])
    assert len(rows) == 9
    prm = Params()
    kf = derived_constants(prm)["k_f"]
    for T, phi, delta, s_ref, E_ref, rate_ref in rows:
        s, E, _ = source_terms(np.array([T]), np.array([phi]), prm)
        assert abs(s[0] - s_ref) <= 1e-13 * abs(s_ref), (T, phi)
        assert abs(E[0] - E_ref) <= 1e-13 * max(abs(E_ref), 1.0), (T, phi)
        assert (E[0] > 0) == bool(delta)
        assert abs(-kf * E[0] * phi - rate_ref) <= 1e-13 * max(abs(rate_ref), 1.0), (T, phi)
