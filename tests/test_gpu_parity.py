"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bars (gpu_helpers.BARS):
  FP64 path: relative L2 of T and of phi <= 1e-10 after all steps, and element by element
  max |T - To| <= 1e-10 max |To - T_amb|, max |phi - phi_o| <= 1e-10;
  FP32 path: relative L2 of T <= 1e-4, max |T - To| <= 1e-4 max |To - T_amb|,
  max |phi - phi_o| <= 1e-5, and the 800 K isotherm within one element
  (symmetric Hausdorff distance over elements, Chebyshev metric).
Cases span several tiles (16 x 16 coefficient tiles of the quadrature
kernel) with ragged tails, several chunks per line (32 coefficients per
chunk in FP32, 64 in FP64), p = 1, 2, 3, non-square grids, the smallest
grids (one element) and the full 1024 x 1024 workload for a few steps.
"""
import numpy as np
import pytest

from gpu_helpers import assert_parity, gpu_run, hausdorff_elements, isotherm_elements, need_gpu, oracle_run, rel
from oracle.physics import Params
from scenarios import config_c1, config_c2, make_scenario

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wf():
    return need_gpu()


def test_c1_fp64_pr(wf):
    sc = config_c1()
    T, phi = gpu_run(wf, sc, sc.steps, wf.WF_FP64)
    To, po = oracle_run(sc, sc.steps)
    assert_parity(T, phi, To, po, "fp64")


def test_c1_fp32_pr(wf):
    sc = config_c1()
    # the C1 ignition sits on thin fuel: its 800 K front exists for about 40 steps (3 elements at
    # step 20) and has died by step 100; the isotherm is compared while it exists, the state after
    # all steps
    sim = wf.simulation_from_scenario(sc, precision=wf.WF_FP32)
    sim.step(20)
    T20, _ = sim.state()
    sim.step(sc.steps - 20)
    assert sim.sync() == wf.WF_OK
    T, phi = sim.state()
    sim.close()
    P = oracle_run(sc, 20)
    To20 = P[0]
    To, po = oracle_run(sc, sc.steps - 20, T0=P[0], phi0=P[1])
    assert_parity(T, phi, To, po, "fp32")
    iso_g = isotherm_elements(T20, sc.nx, sc.p, sc.Lx)
    iso_o = isotherm_elements(To20, sc.nx, sc.p, sc.Lx)
    assert len(iso_o) > 0
    assert hausdorff_elements(iso_g, iso_o) <= 1


def _ring(n, steps):
    # the paper's verification problem (Sec. 5): zero wind, uniform fuel 1, centred ignition
    return make_scenario("ring", n, 2, 1e-3, steps, 9, wind=(0.0, 0.0), uniform_fuel=1.0, centred_ignition=True)


def test_ring_of_fire_fp32_isotherm(wf):
    sc = _ring(64, 60)
    T, phi = gpu_run(wf, sc, sc.steps, wf.WF_FP32)
    To, po = oracle_run(sc, sc.steps)
    assert_parity(T, phi, To, po, "fp32")
    iso_g = isotherm_elements(T, sc.nx, sc.p, sc.Lx)
    iso_o = isotherm_elements(To, sc.nx, sc.p, sc.Lx)
    assert len(iso_o) > 0
    assert hausdorff_elements(iso_g, iso_o) <= 1


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-6)])
def test_full_size_ring_mirror_symmetry(wf, prec, tol):
    # a property that holds at any size: the verification problem stays mirror symmetric
    sc = _ring(1024, 8)
    T, phi = gpu_run(wf, sc, sc.steps, wf.WF_FP64 if prec == "fp64" else wf.WF_FP32)
    assert rel(T[:, ::-1], T) <= tol and rel(T[::-1, :], T) <= tol
    assert rel(phi[:, ::-1], phi) <= tol and rel(phi[::-1, :], phi) <= tol
    assert T.max() > 1000.0


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-4)])
def test_c1_strang(wf, prec, tol):
    sc = config_c1()
    steps = 40
    T, phi = gpu_run(wf, sc, steps, wf.WF_FP64 if prec == "fp64" else wf.WF_FP32, scheme=wf.WF_STRANG_CN)
    To, po = oracle_run(sc, steps, scheme="strang")
    assert_parity(T, phi, To, po, prec, rel_bar=tol)


def test_pr_f_per_substep_fp64(wf):
    sc = config_c1()
    steps = 30
    T, phi = gpu_run(wf, sc, steps, wf.WF_FP64, F_timing=wf.WF_F_PER_SUBSTEP)
    To, po = oracle_run(sc, steps, F_timing="per_substep")
    assert_parity(T, phi, To, po, "fp64")


SHAPES = [(1, 1, 2), (2, 3, 1), (1, 4, 3), (37, 29, 2), (23, 41, 3), (150, 70, 2), (70, 150, 3), (130, 5, 1),
          (300, 260, 2)]


@pytest.mark.parametrize("nx,ny,p", SHAPES)
@pytest.mark.parametrize("scheme", ["pr", "strang"])
def test_shapes_fp64(wf, nx, ny, p, scheme):
    sc = _rect(make_scenario("s", max(nx, ny), p, 1e-3, 4, 100 + nx + ny + p, wind=(1.3, -0.6), fuel_sigma=2.0),
               nx, ny)
    T0 = sc.T0 + 500.0 * np.random.default_rng(nx * ny).random(sc.T0.shape)  # burning almost everywhere
    code = wf.WF_PR if scheme == "pr" else wf.WF_STRANG_CN
    T, phi = gpu_run(wf, sc, sc.steps, wf.WF_FP64, scheme=code, T0=T0)
    To, po = oracle_run(sc, sc.steps, scheme=scheme, T0=T0)
    assert_parity(T, phi, To, po, "fp64")


@pytest.mark.parametrize("nx,ny,p", SHAPES)
def test_shapes_fp32(wf, nx, ny, p):
    sc = _rect(make_scenario("s", max(nx, ny), p, 1e-3, 4, 200 + nx + ny + p, wind=(0.4, 1.1), fuel_sigma=2.0),
               nx, ny)
    T, phi = gpu_run(wf, sc, sc.steps, wf.WF_FP32)
    To, po = oracle_run(sc, sc.steps)
    assert_parity(T, phi, To, po, "fp32", rel_bar=1e-5)


def _rect(sc, nx, ny):
    """Cut a square scenario to nx x ny elements (the generator makes squares)."""
    import dataclasses

    from scenarios.generate import H_ELEMENT

    Nx, Ny = nx + sc.p, ny + sc.p
    cut = lambda a, N: a[:, :N].copy() if a is not None else None  # noqa: E731
    return dataclasses.replace(sc, nx=nx, ny=ny, Lx=H_ELEMENT * nx, Ly=H_ELEMENT * ny, T0=sc.T0[:Ny, :Nx].copy(),
                               fuel0=sc.fuel0[:Ny, :Nx].copy(), fx=cut(sc.fx, Nx), gx=cut(sc.gx, Ny),
                               fy=cut(sc.fy, Nx), gy=cut(sc.gy, Ny))


def test_full_size_fp32_pr_two_steps(wf):
    sc = config_c2()
    T, phi = gpu_run(wf, sc, 2, wf.WF_FP32)
    To, po = oracle_run(sc, 2)
    assert_parity(T, phi, To, po, "fp32", rel_bar=1e-5)


def test_full_size_fp64_one_step_and_strang_fp32(wf):
    sc = config_c2()
    T, phi = gpu_run(wf, sc, 1, wf.WF_FP64)
    To, po = oracle_run(sc, 1)
    assert_parity(T, phi, To, po, "fp64")
    T, phi = gpu_run(wf, sc, 1, wf.WF_FP32, scheme=wf.WF_STRANG_CN)
    To, po = oracle_run(sc, 1, scheme="strang")
    assert_parity(T, phi, To, po, "fp32", rel_bar=1e-5)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_uniform_state_matches_scalar_recurrence(wf, prec):
    # a spatially uniform state stays uniform and follows the PR scalar recurrence (closed form)
    sc = make_scenario("u", 40, 2, 1e-3, 1, 5, wind=(1.0, 0.5))
    T0 = np.full(sc.T0.shape, 1000.0)
    phi0 = np.full(sc.T0.shape, 0.8)
    P = wf.WF_FP64 if prec == "fp64" else wf.WF_FP32
    T, phi = gpu_run(wf, sc, 1, P, T0=T0, phi0=phi0)
    prm = Params()
    import math

    inv = 1 / (prm.rho * prm.cp)
    r = prm.A_r * 1000.0 * math.exp(-300.0 / 1000.0)
    s = (-1e4 * prm.rho * prm.ch * prm.hc * r + prm.chi * 300.0 + prm.sigma * prm.eps / prm.delta_z *
         (300.0 ** 4 - 1000.0 ** 4)) * inv
    th = 0.5e-3
    c_chi = prm.chi * inv
    Ts = (1000.0 + th * s) / (1 + th * c_chi)
    Te = (1 - th * c_chi) * Ts + th * s
    pe = 0.8 * (1 - 1e-3 * 300 * r)
    # FP32: the state is T + increment; rounding of the increment (|dT| ~ 23 K) through the
    # inverse 2-D mass matrix (condition ~ 1e2 to 1e3) stays below ~1e-6 relative to T
    tol = 1e-12 if prec == "fp64" else 1e-6
    assert np.abs(T / Te - 1).max() <= tol
    assert np.abs(phi / pe - 1).max() <= tol


def test_ambient_state_steady_fp32(wf):
    sc = make_scenario("a", 50, 3, 1e-3, 20, 6, wind=(2.0, -1.0))
    T, _ = gpu_run(wf, sc, 20, wf.WF_FP32, T0=np.full(sc.T0.shape, 300.0))
    # increments vanish at the ambient state: only storage rounding of 300 K remains
    assert np.abs(T - 300.0).max() <= 300.0 * 1e-6


def test_guard_reports_unstable(wf):
    sc = make_scenario("g", 20, 2, 1e-3, 1, 8, wind=(1.0, 0.0))
    T0 = sc.T0.copy()
    T0[5, 7] = np.nan
    sim = wf.simulation_from_scenario(sc, precision=wf.WF_FP32)
    sim.set_state(T0, sc.fuel0)
    sim.step(2)
    assert sim.sync() == wf.WF_EUNSTABLE
    assert sim.sync() == wf.WF_OK  # the flag is cleared by the call
    sim.close()


@pytest.mark.parametrize("scheme", ["pr", "strang"])
def test_checkpoint_resume_and_determinism_bitwise(wf, scheme):
    sc = make_scenario("c", 60, 2, 1e-3, 1, 12, wind=(0.5, 1.0))
    code = wf.WF_PR if scheme == "pr" else wf.WF_STRANG_CN
    a = wf.simulation_from_scenario(sc, precision=wf.WF_FP32, scheme=code)
    a.step(11)
    Ta, pa = a.state()
    a.close()
    b = wf.simulation_from_scenario(sc, precision=wf.WF_FP32, scheme=code)
    b.step(5)
    Tb, pb = b.state()
    b.set_state(Tb, pb)
    b.step(6)
    Tb, pb = b.state()
    b.close()
    assert np.array_equal(Ta, Tb) and np.array_equal(pa, pb)
    c = wf.simulation_from_scenario(sc, precision=wf.WF_FP32, scheme=code)
    c.step(11)
    Tc, pc = c.state()
    c.close()
    assert np.array_equal(Ta, Tc) and np.array_equal(pa, pc)


def test_wind_change_between_steps(wf):
    sc = config_c1()
    sim = wf.simulation_from_scenario(sc, precision=wf.WF_FP64)
    sim.step(3)
    sim.set_wind(0)
    sim.step(3)
    T, phi = sim.state()
    sim.close()
    T1, p1 = oracle_run(sc, 3)
    import dataclasses

    sc0 = dataclasses.replace(sc, wind_rank=0)
    To, po = oracle_run(sc0, 3, T0=T1, phi0=p1)
    assert_parity(T, phi, To, po, "fp64")


@pytest.mark.parametrize("wind", [(0.0, 0.0), (1.3, -0.6)])
def test_fp32_hot_rows(wf, wind):
    # 700 K with three coefficient rows partly at 1100 K: only the element rows whose window holds
    # a hot row can reach the ignition temperature (800 K), so warps of the FP32 quadrature take
    # the form that skips the reaction term next to warps that evaluate it point by point.  One
    # step from these values keeps every Gauss point far from the threshold (the oracle's result
    # does not move when T_ig moves by 1e-3 K), while the reaction changes T by about 1 %.
    sc = make_scenario("ign", 96, 2, 1e-3, 1, 611, wind=wind, fuel_sigma=3.0)
    rng = np.random.default_rng(612)
    T0 = np.full(sc.T0.shape, 700.0)
    for r in (20, 47, 71):
        T0[r, rng.random(T0.shape[1]) < 0.3] = 1100.0
    T, phi = gpu_run(wf, sc, 1, wf.WF_FP32, T0=T0)
    To, po = oracle_run(sc, 1, T0=T0)
    assert_parity(T, phi, To, po, "fp32", rel_bar=1e-5)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_state_io_f32_matches_f64(wf, prec):
    # the float32 state calls carry the same values as the float64 ones: set from float32 values
    # (exactly representable in both), step, read both ways
    sc = make_scenario("io", 60, 2, 1e-3, 1, 71, wind=(0.7, -0.4), fuel_sigma=3.0)
    P = wf.WF_FP32 if prec == "fp32" else wf.WF_FP64
    T0 = sc.T0.astype(np.float32)
    F0 = sc.fuel0.astype(np.float32)
    a = wf.simulation_from_scenario(sc, precision=P)
    b = wf.simulation_from_scenario(sc, precision=P)
    wf.wf_set_state(a.h, T0.astype(np.float64), F0.astype(np.float64))
    wf.wf_set_state_f32(b.h, T0, F0)
    a.step(3)
    b.step(3)
    Ta, Fa = wf.wf_get_state(a.h)
    Tb, Fb = wf.wf_get_state(b.h)
    assert np.array_equal(Ta, Tb) and np.array_equal(Fa, Fb)
    T32, F32 = wf.wf_get_state_f32(b.h)
    assert T32.dtype == np.float32
    assert np.array_equal(T32, Tb.astype(np.float32)) and np.array_equal(F32, Fb.astype(np.float32))
    a.close()
    b.close()
