"""The large single domain at full size: 4096 x 4096 elements, cubic B-splines (16.8M DOFs), FP32
bulk with FP64 1-D factorisations, Peaceman-Rachford, in the launch configuration of wf_step.

The FP64 oracle cannot step 16.8M DOFs within a test, so two checks stand in for element-by-element
parity at this size:

* sampled outputs: the oracle runs the same steps on a 160 x 160-element window around an ignition
  (same element size, the window's fuel, temperature and wind-factor coefficients).  Every kernel of
  the step is local except the 1-D inverses, whose entries decay by 1e-11 over 40 DOFs for cubic
  splines, so away from the window's edges its result is the full domain's to far below the FP32
  bar; the outputs at least 45 DOFs inside the window are compared;
* a property over every DOF: a uniform state (below ignition) stays uniform under any wind and
  follows the same 0-D update whatever the mesh, so all 16.8M values must equal the oracle's value
  on a small grid.
"""
import dataclasses

import numpy as np
import pytest

from gpu_helpers import assert_parity, gpu_run, need_gpu, oracle_run, rel
from scenarios import config_c3

pytestmark = pytest.mark.gpu

STEPS = 2
WIN = 160  # window elements
EDGE = 45  # DOFs left out at each edge of the window


@pytest.fixture(scope="module")
def wf():
    return need_gpu()


@pytest.fixture(scope="module")
def c3():
    return config_c3()


def _window(sc, e0x, e0y, n):
    N = n + sc.p
    h = sc.Lx / sc.nx
    cut = lambda a: a[e0y:e0y + N, e0x:e0x + N].copy()  # noqa: E731
    kw = {}
    if sc.wind_rank:
        kw = dict(fx=sc.fx[:, e0x:e0x + N].copy(), gx=sc.gx[:, e0y:e0y + N].copy(),
                  fy=sc.fy[:, e0x:e0x + N].copy(), gy=sc.gy[:, e0y:e0y + N].copy())
    return dataclasses.replace(sc, name=sc.name + "_window", nx=n, ny=n, Lx=n * h, Ly=n * h,
                               T0=cut(sc.T0), fuel0=cut(sc.fuel0), **kw)


def test_c3_sampled_window(wf, c3):
    sc = c3
    assert sc.nx == 4096 and sc.p == 3 and sc.wind_rank > 0
    T, phi = gpu_run(wf, sc, STEPS, wf.WF_FP32)
    assert T.shape == (4099, 4099) and np.all(np.isfinite(T))
    # window centred on the hottest coefficient (an ignition), kept inside the domain's interior
    j, i = np.unravel_index(np.argmax(sc.T0), sc.T0.shape)
    e0x = int(np.clip(i - WIN // 2, 8, sc.nx - WIN - 8))
    e0y = int(np.clip(j - WIN // 2, 8, sc.ny - WIN - 8))
    sub = _window(sc, e0x, e0y, WIN)
    To, po = oracle_run(sub, STEPS)
    N = WIN + sc.p
    inner = (slice(EDGE, N - EDGE), slice(EDGE, N - EDGE))
    Tg = T[e0y:e0y + N, e0x:e0x + N][inner]
    pg = phi[e0y:e0y + N, e0x:e0x + N][inner]
    # the window holds the ignition: the reaction term is exercised
    assert Tg.max() > 800.0
    assert_parity(Tg, pg, To[inner], po[inner], "fp32", rel_bar=1e-5)


def test_c3_uniform_state_every_dof(wf, c3):
    sc = c3
    T0 = np.full(sc.T0.shape, 500.0)
    phi0 = np.full(sc.T0.shape, 0.6)
    T, phi = gpu_run(wf, sc, STEPS, wf.WF_FP32, T0=T0, phi0=phi0)
    small = _window(dataclasses.replace(sc, T0=T0, fuel0=phi0), 100, 100, 8)
    To, po = oracle_run(small, STEPS)
    t_ref = To.mean()
    assert np.abs(To / t_ref - 1).max() <= 1e-12  # the oracle's state is uniform too
    assert np.abs(T / t_ref - 1).max() <= 1e-5
    assert np.abs(phi / po.mean() - 1).max() <= 1e-5
