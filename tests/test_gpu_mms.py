"""Manufactured-solution forcing on the GPU (the convergence study of Sec. 6).

* parity with the oracle (same forcing, same Gauss rule, same start times) for PR (one F
  per step and per substep), Strang/Crank-Nicolson and the explicit scheme, linear and
  with the nonlinear diffusion and radiation, FP64 <= 1e-10 and FP32 <= 1e-5;
* first-order convergence in time of the GPU result towards u* (the paper's conclusion)
  and the device clock at t = 1 after the last step.
"""
import numpy as np
import pytest

from gpu_helpers import need_gpu, rel
from oracle.mms import PAPER_MODES, Manufactured
from oracle.physics import Params
from oracle.step import Problem

pytestmark = pytest.mark.gpu

L = 100.0
WIND = (1.0, 0.5)


@pytest.fixture(scope="module")
def wf():
    return need_gpu()


def _gpu_sim(wf, nx, ny, tau, prec, scheme, F_timing, linear):
    prm = wf.wf_params_default(Lx=L, Ly=L, wind_x=WIND[0], wind_y=WIND[1], precision=prec, scheme=scheme,
                               F_timing=F_timing, heat_scale=0.0, **({"sigma": 0.0} if linear else {}))
    sim = wf.Simulation(nx, ny, 2, tau, prm)
    wf.wf_set_mms(sim.h, [(a, n, m, lam) for a, n, m, lam in PAPER_MODES], 300.0, 0.0)
    return sim


def _oracle(nx, ny, tau, scheme, F_timing, linear, forcing):
    prm = Params(heat_scale=0.0, sigma=0.0, F_timing=F_timing) if linear else Params(heat_scale=0.0, F_timing=F_timing)
    return Problem(nx, ny, 2, L, L, tau, wind=WIND, prm=prm, scheme=scheme, mode="ads", forcing=forcing)


CASES = [("pr", "once"), ("pr", "per_substep"), ("strang", "once"), ("explicit", "once")]


@pytest.mark.parametrize("scheme,F_timing", CASES)
@pytest.mark.parametrize("linear", [True, False])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_forcing_parity(wf, scheme, F_timing, linear, prec, tol):
    nx, ny, tau, steps = 24, 20, 1 / 16, 6
    m = Manufactured()
    P = _oracle(nx, ny, tau, scheme, F_timing, linear, m)
    T0 = m.project(P.tx, P.ty, 0.0)
    phi0 = np.zeros_like(T0)
    To, po = P.run(T0, phi0, steps)
    code = {"pr": wf.WF_PR, "strang": wf.WF_STRANG_CN, "explicit": wf.WF_EXPLICIT}[scheme]
    ft = wf.WF_F_ONCE if F_timing == "once" else wf.WF_F_PER_SUBSTEP
    sim = _gpu_sim(wf, nx, ny, tau, wf.WF_FP64 if prec == "fp64" else wf.WF_FP32, code, ft, linear)
    sim.set_state(T0, phi0)
    sim.step(steps)
    assert sim.sync() == wf.WF_OK
    T, _ = sim.state()
    assert abs(wf.wf_get_time(sim.h) - steps * tau) < 1e-12
    sim.close()
    assert rel(T, To) <= tol


def test_first_order_convergence_on_gpu(wf):
    m = Manufactured()
    errs = []
    for tau in (1 / 16, 1 / 32, 1 / 64):
        P = _oracle(50, 50, tau, "pr", "once", True, m)  # tables and norms only
        T = m.project(P.tx, P.ty, 0.0)
        sim = _gpu_sim(wf, 50, 50, tau, wf.WF_FP64, wf.WF_PR, wf.WF_F_ONCE, True)
        sim.set_state(T, np.zeros_like(T))
        se = sr = 0.0
        steps = int(round(1 / tau))
        for k in range(steps):
            sim.step(1)
            Tk, _ = sim.state()
            e, r = m.l2_norms(P.tx, P.ty, Tk, (k + 1) * tau)
            se += e * e
            sr += r * r
        assert abs(wf.wf_get_time(sim.h) - 1.0) < 1e-12
        sim.close()
        errs.append(np.sqrt(se / sr))
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(0.8 < r < 1.3 for r in rates), (errs, rates)
