"""Explicit L2-projection scheme on the GPU (the explicit dynamics of Sec. 6): parity with the oracle.

One step is (M^x (x) M^y)(T^{n+1} - T^n) = tau F(T^n) - tau (A_x (x) M^y + M^x (x) A_y) T^n and
the same fuel update as the split schemes; the kernels are the quadrature, one x pass and one
y pass with the mass matrices.  Bars as for the split schemes: FP64 <= 1e-10, FP32 <= 1e-5
after a few steps; shapes cover several chunks per line, ragged tails and p = 1, 2, 3.
"""
import numpy as np
import pytest

from gpu_helpers import assert_parity, gpu_run, need_gpu, oracle_run
from scenarios import config_c1, make_scenario
from test_gpu_parity import _rect

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wf():
    return need_gpu()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_c1_explicit(wf, prec, tol):
    sc = config_c1()
    steps = 40
    P = wf.WF_FP64 if prec == "fp64" else wf.WF_FP32
    T, phi = gpu_run(wf, sc, steps, P, scheme=wf.WF_EXPLICIT)
    To, po = oracle_run(sc, steps, scheme="explicit")
    assert_parity(T, phi, To, po, prec, rel_bar=tol)


@pytest.mark.parametrize("nx,ny,p", [(1, 1, 2), (37, 29, 2), (23, 41, 3), (150, 70, 2), (130, 5, 1)])
def test_shapes_explicit_fp64(wf, nx, ny, p):
    sc = _rect(make_scenario("e", max(nx, ny), p, 1e-3, 4, 300 + nx + ny + p, wind=(0.9, -1.4), fuel_sigma=2.0),
               nx, ny)
    T0 = sc.T0 + 500.0 * np.random.default_rng(nx + 7 * ny).random(sc.T0.shape)
    T, phi = gpu_run(wf, sc, sc.steps, wf.WF_FP64, scheme=wf.WF_EXPLICIT, T0=T0)
    To, po = oracle_run(sc, sc.steps, scheme="explicit", T0=T0)
    assert_parity(T, phi, To, po, "fp64")


def test_explicit_uniform_state(wf):
    # a uniform state follows T' = (1 - tau c_chi) T + tau s(T, phi) exactly (FP64)
    sc = make_scenario("u", 30, 2, 1e-3, 1, 5, wind=(1.0, 0.5))
    T0 = np.full(sc.T0.shape, 1000.0)
    phi0 = np.full(sc.T0.shape, 0.8)
    T, _ = gpu_run(wf, sc, 1, wf.WF_FP64, scheme=wf.WF_EXPLICIT, T0=T0, phi0=phi0)
    To, _ = oracle_run(sc, 1, scheme="explicit", T0=T0, phi0=phi0)
    assert np.abs(T / To - 1).max() <= 1e-12
    assert np.abs(T / T.mean() - 1).max() <= 1e-12
