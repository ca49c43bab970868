"""Kernels per time step, as counted by wf_launch_count (the bench's gpu_launches).

A PR step with one F per step launches the quadrature (FP32 with interior elements: an
interior launch and a boundary launch), the first x and y passes and the second x and y
passes; the count is the same in eager mode and, replayed, in the captured graph.
"""
import pytest

from gpu_helpers import need_gpu
from scenarios import make_scenario

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wf():
    return need_gpu()


@pytest.mark.parametrize("prec,n,per_step", [("fp32", 200, 6), ("fp64", 200, 5), ("fp32", 6, 5)])
def test_launches_per_step(wf, prec, n, per_step):
    sc = make_scenario("l", n, 2, 1e-3, 1, 5)
    sim = wf.simulation_from_scenario(sc, precision=wf.WF_FP32 if prec == "fp32" else wf.WF_FP64)
    wf.wf_set_profiling(sim.h, True)
    n0 = wf.wf_launch_count()
    sim.step(3)
    n1 = wf.wf_launch_count()
    assert sim.sync() == wf.WF_OK
    wf.wf_kernel_times(sim.h)
    sim.close()
    assert n1 - n0 == 3 * per_step
