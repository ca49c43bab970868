"""Bounded device waits give up, report WF_ETIMEOUT and leave the device usable.

The wait limit (wf_set_wait_limit) is set to 0 seconds, so every bounded wait of a step
gives up at its first check instead of waiting for its barrier: the kernel drains its
copies in flight, sets the timeout bit of its slot and returns.  Nothing faults or
hangs; wf_sync reports WF_ETIMEOUT (it outranks the guard, since the step's output is
invalid), the flags are cleared, and with the default limit restored the handle steps
exactly as a fresh one does.
"""
import numpy as np
import pytest

from gpu_helpers import need_gpu
from scenarios import make_scenario

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wf():
    return need_gpu()


@pytest.mark.parametrize("capacity", [1, 3])
def test_wait_limit_zero_reports_timeout_and_recovers(wf, capacity):
    sc = make_scenario("to", 120, 2, 1e-3, 1, 41, wind=(0.8, 0.3), fuel_sigma=3.0)
    prm = wf.wf_params_default(Lx=sc.Lx, Ly=sc.Ly, wind_x=sc.wind[0], wind_y=sc.wind[1], precision=wf.WF_FP32)
    b = wf.Batch(sc.nx, sc.ny, sc.p, sc.dt, prm, capacity=capacity)
    for k in range(capacity):
        b.load_scenario(k, sc)
    wf.wf_set_wait_limit(b.h, 0.0)
    b.step(2)
    assert wf.wf_sync(b.h) == wf.WF_ETIMEOUT
    st = wf.wf_batch_status(b.h)  # cleared by the call above
    assert not st.any()
    wf.wf_set_wait_limit(b.h, 1.0)
    for k in range(capacity):
        b.load_scenario(k, sc)
    b.step(3)
    assert wf.wf_sync(b.h) == wf.WF_OK
    ref = wf.simulation_from_scenario(sc, precision=wf.WF_FP32)
    ref.step(3)
    assert ref.sync() == wf.WF_OK
    Tr, Pr = ref.state()
    ref.close()
    for k in range(capacity):
        T, P = b.state(k)
        assert np.array_equal(T, Tr) and np.array_equal(P, Pr)
    b.close()


def test_wait_limit_arguments(wf):
    sc = make_scenario("to2", 16, 2, 1e-3, 1, 42, wind=(0.0, 0.0))
    s = wf.simulation_from_scenario(sc, precision=wf.WF_FP32)
    for bad in (-1.0, 61.0, float("nan")):
        with pytest.raises(wf.WFError):
            wf.wf_set_wait_limit(s.h, bad)
    s.close()
