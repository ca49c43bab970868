"""Kernels per time step, as counted by wf_launch_count (the bench's gpu_launches).

Per-pass form: a PR step with one F per step launches the quadrature (FP32 with interior
elements: an interior launch, a launch for the boundary strips and one for the boundary segments),
the first x and y passes, the substep-2 right-hand side and the second x and y passes.  Persistent form: one quadrature launch, then one launch for every line pass,
whatever the number of slots.  The library counts the kernels it launches (eager steps, and captures once); a replayed
step graph runs the captured kernels without counting them again.
"""
import pytest

from gpu_helpers import need_gpu
from scenarios import make_scenario

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wf():
    return need_gpu()


@pytest.mark.parametrize("prec,n,form,per_step", [("fp32", 200, 1, 7), ("fp64", 200, 1, 5), ("fp32", 6, 1, 5), ("fp32", 200, 3, 7),
                                                  ("fp32", 200, 2, 2), ("fp32", 6, 2, 2), ("fp64", 200, 2, 2)])
@pytest.mark.parametrize("graph", [False, True])
def test_launches_per_step(wf, prec, n, form, per_step, graph):
    sc = make_scenario("l", n, 2, 1e-3, 1, 5)
    sim = wf.simulation_from_scenario(sc, precision=wf.WF_FP32 if prec == "fp32" else wf.WF_FP64)
    wf.wf_set_tuning(sim.h, (0, 0, 0, 0, 0, 0, form, 0))
    if graph:
        sim.step(1)  # captures the step graphs (the capture counts its launches once)
        assert sim.sync() == wf.WF_OK
    else:
        wf.wf_set_profiling(sim.h, True)
    n0 = wf.wf_launch_count()
    sim.step(3)
    n1 = wf.wf_launch_count()
    assert sim.sync() == wf.WF_OK
    wf.wf_kernel_times(sim.h)
    sim.close()
    if graph:
        # graph replays launch the captured kernels without passing through the counter
        assert n1 - n0 == 0
    else:
        assert n1 - n0 == 3 * per_step
