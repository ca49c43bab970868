"""Pins of the oracle's time steps (PR, Sec. 3.1; Strang/Crank-Nicolson, Sec. 3.2).

* 'ads' (1-D line solves, Sec. 4) equals 'direct' (assembled 2-D system) to 1e-12;
  'direct' equals a dense numpy solve of the same system on tiny grids.
* Closed-form decay of discrete eigenmodes (pure diffusion, F off): one PR step
  multiplies v_x (x) v_y by (1 - th C_d l_y)(1 - th C_d l_x) / ((1 + th C_d l_x)(1 + th C_d l_y)),
  th = tau/2; one Strang step by [(1 - tau C_d l_x/4)/(1 + tau C_d l_x/4)]^2 (1 - tau C_d l_y/2)/(1 + tau C_d l_y/2);
  one explicit L2-projection step by 1 - tau C_d (l_x + l_y).
* A spatially uniform state follows the scalar recurrences derived from the schemes
  (source recomputed from raw Table constants, not from the oracle), for PR also with the
  second substep's F evaluated at T*.
* The ambient state T = T_amb is steady for any wind and fuel.
* With zero wind and only diffusion (linear and T^3), the heat content
  1^T (M (x) M) T is conserved.
* Mirror symmetry of the paper's verification problem (Sec. 5: zero wind,
  uniform fuel, centred ignition).
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from oracle.physics import Params
from oracle.step import Problem
from scenarios import make_scenario


def _raw_s(T, phi, prm):
    inv = 1.0 / (prm.rho * prm.cp)
    delta = 1.0 if (T > prm.T_ig and phi > prm.fuel_thresh + prm.thresh_guard) else 0.0
    r = delta * prm.A_r * T * math.exp(-prm.T_a / T)
    Rc = -1e4 * prm.rho * prm.ch * prm.hc * prm.M_ratio * r
    s = (Rc + prm.chi * prm.T_amb + prm.sigma * prm.eps / prm.delta_z * (prm.T_amb ** 4 - T ** 4)) * inv
    return s, r


def _uniform_pr(T, phi, prm, tau):
    c_chi = prm.chi / (prm.rho * prm.cp)
    th = tau / 2
    s, r = _raw_s(T, phi, prm)
    Ts = (T + th * s) / (1 + th * c_chi)
    Tn = (1 - th * c_chi) * Ts + th * s
    return Tn, phi * (1 - tau * 3e2 * r)


def _uniform_pr_per_substep(T, phi, prm, tau):
    # the second substep's F is evaluated at T* (with the step's starting fuel)
    c_chi = prm.chi / (prm.rho * prm.cp)
    th = tau / 2
    s, r = _raw_s(T, phi, prm)
    Ts = (T + th * s) / (1 + th * c_chi)
    s2, _ = _raw_s(Ts, phi, prm)
    Tn = (1 - th * c_chi) * Ts + th * s2
    return Tn, phi * (1 - tau * 3e2 * r)


def _uniform_explicit(T, phi, prm, tau):
    c_chi = prm.chi / (prm.rho * prm.cp)
    s, r = _raw_s(T, phi, prm)
    return T - tau * c_chi * T + tau * s, phi * (1 - tau * 3e2 * r)


def _uniform_strang(T, phi, prm, tau):
    c_chi = prm.chi / (prm.rho * prm.cp)
    q = tau / 4
    s, r = _raw_s(T, phi, prm)
    Ts = ((1 - q * c_chi) * T + tau / 2 * s) / (1 + q * c_chi)
    s3, _ = _raw_s(Ts, phi, prm)
    Tn = ((1 - q * c_chi) * Ts + tau / 2 * s3) / (1 + q * c_chi)
    return Tn, phi * (1 - tau * 3e2 * r)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("scheme", ["pr", "strang", "explicit"])
@pytest.mark.parametrize("p,n", [(2, 1), (2, 6), (3, 5), (3, 13)])
def test_ads_equals_direct(scheme, p, n):
    sc = make_scenario("t", n, p, 1e-3, 3, 11 + n, wind=(1.2, -0.4), fuel_sigma=1.0)
    T0 = sc.T0 + 400.0 * np.random.default_rng(n).random(sc.T0.shape)
    Pd = Problem.from_scenario(sc, scheme=scheme, mode="direct")
    Pa = Problem.from_scenario(sc, scheme=scheme, mode="ads")
    Td, pd = Pd.run(T0, sc.fuel0, 3)
    Ta, pa = Pa.run(T0, sc.fuel0, 3)
    assert _rel(Ta, Td) < 1e-12
    assert _rel(pa, pd) < 1e-12
    R = np.random.default_rng(5).normal(size=T0.shape)
    for key in [("x", 5e-4, 1.0), ("y", 5e-4, 1.0), ("m",)]:
        assert _rel(Pa.solve(key, R), Pd.solve(key, R)) < 1e-12
        assert _rel(Pa.apply(key, R), Pd.apply(key, R)) < 1e-13


@pytest.mark.parametrize("p", [1, 2, 3])
def test_direct_equals_dense_solve(p):
    P = Problem(2, 3, p, 3.125, 4.6875, 1e-3, wind=(0.7, 2.0), mode="direct")
    R = np.random.default_rng(p).normal(size=(3 + p, 2 + p))
    for key in [("x", 5e-4, 1.0), ("y", 5e-4, 1.0), ("m",)]:
        dense = np.linalg.solve(P.op2d(key).toarray(), R.ravel()).reshape(R.shape)
        assert _rel(P.solve(key, R), dense) < 1e-13


def _diffusion_only():
    return Params(sigma=0.0, chi=0.0, heat_scale=0.0)


@pytest.mark.parametrize("mode", ["direct", "ads"])
@pytest.mark.parametrize("p", [2, 3])
def test_eigenmode_decay_pr_and_strang(mode, p):
    nx, ny, Lx, Ly = 9, 7, 14.0, 10.0
    dt = 0.8  # large enough that the factors differ visibly from 1
    prm = _diffusion_only()
    C_d = prm.kappa / (prm.rho * prm.cp)
    for scheme in ("pr", "strang", "explicit"):
        P = Problem(nx, ny, p, Lx, Ly, dt, prm=prm, scheme=scheme, mode=mode)
        lx, Vx = sla.eigh(P.Kx.toarray(), P.Mx.toarray())
        ly, Vy = sla.eigh(P.Ky.toarray(), P.My.toarray())
        for kx, ky in [(3, 2), (1, 5), (6, 0)]:
            T0 = np.outer(Vy[:, ky], Vx[:, kx])
            T1, _ = P.step(T0, np.ones_like(T0))
            if scheme == "pr":
                th = dt / 2
                rho = ((1 - th * C_d * ly[ky]) * (1 - th * C_d * lx[kx])
                       / ((1 + th * C_d * lx[kx]) * (1 + th * C_d * ly[ky])))
            elif scheme == "explicit":
                rho = 1 - dt * C_d * (lx[kx] + ly[ky])
            else:
                ax = (1 - dt * C_d * lx[kx] / 4) / (1 + dt * C_d * lx[kx] / 4)
                ay = (1 - dt * C_d * ly[ky] / 2) / (1 + dt * C_d * ly[ky] / 2)
                rho = ax * ax * ay
            assert _rel(T1, rho * T0) < 1e-12, (scheme, kx, ky)


@pytest.mark.parametrize("scheme", ["pr", "strang", "explicit"])
@pytest.mark.parametrize("T,phi", [(1000.0, 0.8), (1000.0, 0.1), (500.0, 0.9), (1400.0, 0.2 + 5e-7)])
def test_uniform_state_recurrence(scheme, T, phi):
    sc = make_scenario("u", 5, 2, 2e-3, 1, 3, wind=(1.0, 0.5))  # wind and its perturbation on
    prm = Params()
    P = Problem.from_scenario(sc, prm=prm, scheme=scheme, mode="direct")
    shape = sc.T0.shape
    Tn, pn = P.step(np.full(shape, T), np.full(shape, phi))
    f = {"pr": _uniform_pr, "strang": _uniform_strang, "explicit": _uniform_explicit}[scheme]
    Te, pe = f(T, phi, prm, sc.dt)
    assert np.abs(Tn / Te - 1).max() < 1e-12
    assert np.abs(pn / pe - 1).max() < 1e-12


@pytest.mark.parametrize("T,phi", [(1000.0, 0.8), (790.0, 0.8), (500.0, 0.9)])
def test_uniform_state_recurrence_f_per_substep(T, phi):
    # (burning, just below ignition, and cool)
    sc = make_scenario("u", 5, 2, 2e-3, 1, 3, wind=(1.0, 0.5))
    prm = Params(F_timing="per_substep")
    P = Problem.from_scenario(sc, prm=prm, scheme="pr", mode="direct")
    shape = sc.T0.shape
    Tn, pn = P.step(np.full(shape, T), np.full(shape, phi))
    Te, pe = _uniform_pr_per_substep(T, phi, prm, sc.dt)
    assert np.abs(Tn / Te - 1).max() < 1e-12
    assert np.abs(pn / pe - 1).max() < 1e-12
    # and it differs from the one-F step (the T^4 loss and the reaction change with T)
    To, _ = _uniform_pr(T, phi, Params(), sc.dt)
    assert abs(Te - To) > 0


@pytest.mark.parametrize("scheme", ["pr", "strang", "explicit"])
def test_ambient_state_is_steady(scheme):
    sc = make_scenario("a", 8, 3, 1e-3, 1, 21, wind=(2.0, -1.0))
    P = Problem.from_scenario(sc, scheme=scheme, mode="ads")
    T, phi = P.run(np.full(sc.T0.shape, 300.0), sc.fuel0, 4)
    assert np.abs(T / 300.0 - 1).max() < 1e-12


@pytest.mark.parametrize("scheme", ["pr", "strang", "explicit"])
def test_heat_content_conserved_without_sources(scheme):
    # linear and T^3 diffusion on, every source and the wind off
    prm = Params(chi=0.0, heat_scale=0.0, delta_z=1e300)
    sc = make_scenario("h", 10, 2, 1e-3, 1, 4, wind=(0.0, 0.0))
    P = Problem.from_scenario(sc, prm=prm, scheme=scheme, mode="ads")
    wx = P.Mx @ np.ones(sc.Nx)
    wy = P.My @ np.ones(sc.Ny)
    H0 = wy @ sc.T0 @ wx
    T, _ = P.run(sc.T0, sc.fuel0, 5)
    assert abs(wy @ T @ wx - H0) < 1e-13 * abs(H0)
    assert np.abs(T - sc.T0).max() > 1e-3  # the state did evolve


@pytest.mark.parametrize("scheme", ["pr", "strang", "explicit"])
def test_mirror_symmetry_of_verification_problem(scheme):
    sc = make_scenario("v", 12, 2, 1e-3, 1, 9, wind=(0.0, 0.0), uniform_fuel=1.0, centred_ignition=True)
    P = Problem.from_scenario(sc, scheme=scheme, mode="ads")
    T, phi = P.run(sc.T0, sc.fuel0, 6)
    assert _rel(T[:, ::-1], T) < 1e-13 and _rel(T[::-1, :], T) < 1e-13
    assert _rel(phi[:, ::-1], phi) < 1e-13 and _rel(phi[::-1, :], phi) < 1e-13
    assert phi.min() < 0.99  # fuel burned near the centre


def _transport_only():
    return Params(kappa=0.0, sigma=0.0, chi=0.0, heat_scale=0.0)


def _centroid(T, xg, yg, bg=300.0):
    d = T - bg
    return (d * xg[None, :]).sum() / d.sum(), (d * yg[:, None]).sum() / d.sum()


@pytest.mark.parametrize("implicit", [True, False])
def test_wind_transports_heat_downwind(implicit):
    # pure advection dT/dt + c_W b.grad T = 0 moves a smooth bump by c_W b t
    from scenarios import greville

    n, p, L = 48, 2, 48 * 100 / 64
    sc = make_scenario("w", n, p, 0.02, 1, 5, wind=(0.0, 0.0), uniform_fuel=0.0, centred_ignition=True,
                       sigma_ign=4.0)
    b = (2.0, -1.0)
    N = n + p
    if implicit:
        P = Problem(n, n, p, L, L, sc.dt, wind=b, prm=_transport_only(), mode="ads")
    else:  # the same wind as a rank-1 explicit variation: b'_x = 2 * 1, b'_y = -1 * 1
        wf = (np.ones((1, N)), b[0] * np.ones((1, N)), np.ones((1, N)), b[1] * np.ones((1, N)))
        P = Problem(n, n, p, L, L, sc.dt, wind=(0.0, 0.0), wind_factors=wf, prm=_transport_only(), mode="ads")
    xg = greville(n, p, L)
    x0, y0 = _centroid(sc.T0, xg, xg)
    steps = 25
    T, _ = P.run(sc.T0, sc.fuel0, steps)
    x1, y1 = _centroid(T, xg, xg)
    t = steps * sc.dt
    assert abs((x1 - x0) - 0.5 * b[0] * t) < 0.03 * abs(0.5 * b[0] * t)
    assert abs((y1 - y0) - 0.5 * b[1] * t) < 0.03 * abs(0.5 * b[1] * t)
