"""wf_batch_run: states from host arrays, steps, states back, pipelined over slot groups.

The slots are taken in groups whose uploads, steps and downloads overlap on three streams; each
group's steps are the per-pass launches over its slots.  Every slot is independent, so the result
must equal wf_batch_set_states + wf_step + wf_batch_get_states bit for bit, for every group count,
in both host precisions, with inactive slots and step budgets, and with the output arrays equal to
the input arrays.
"""
import numpy as np
import pytest
import torch

from gpu_helpers import need_gpu
from scenarios import make_scenario

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wf():
    return need_gpu()


def _batch(wf, k, prec, inactive=(), budgets=None):
    winds = [(1.0, 0.5), (0.0, 0.0), (-2.0, 1.5), (0.3, -2.7), (2.5, 0.0)]
    scs = [make_scenario(f"r{i}", 40, 2, 1e-3, 1, 1200 + i, wind=winds[i % 5], fuel_sigma=3.0) for i in range(k)]
    sc0 = scs[0]
    prm = wf.wf_params_default(Lx=sc0.Lx, Ly=sc0.Ly, precision=prec)
    b = wf.Batch(sc0.nx, sc0.ny, sc0.p, sc0.dt, prm, capacity=k)
    for i, sc in enumerate(scs):
        b.load_scenario(i, sc, active=i not in inactive)
    if budgets is not None:
        for i, n in enumerate(budgets):
            wf.wf_batch_set_budget(b.h, i, n)
    return b, scs


def _host(scs, dt):
    T = torch.empty(len(scs) * scs[0].T0.size, dtype=dt, pin_memory=True)
    P = torch.empty_like(T, pin_memory=True)
    n = scs[0].T0.size
    for i, sc in enumerate(scs):
        T.numpy()[i * n:(i + 1) * n] = sc.T0.ravel()
        P.numpy()[i * n:(i + 1) * n] = sc.fuel0.ravel()
    return T, P


@pytest.mark.parametrize("f32", [True, False])
@pytest.mark.parametrize("groups", [1, 2, 3, 8])
def test_run_equals_set_step_get(wf, f32, groups):
    prec = wf.WF_FP32 if f32 else wf.WF_FP64
    dt = torch.float32 if f32 else torch.float64
    k, steps = 5, 3
    inactive, budgets = (3,), [-1, 2, -1, -1, 1]
    # reference: one upload, the steps, one download
    a, scs = _batch(wf, k, prec, inactive, budgets)
    Ta, Pa = _host(scs, dt)
    n = Ta.numel()
    wf.wf_batch_states_ptr(a.h, Ta.data_ptr(), Pa.data_ptr(), n, f32, True)
    a.step(steps)
    wf.wf_batch_states_ptr(a.h, Ta.data_ptr(), Pa.data_ptr(), n, f32, False)
    assert wf.wf_sync(a.h) == wf.WF_OK
    a.close()
    # the pipelined call, in place
    b, _ = _batch(wf, k, prec, inactive, budgets)
    Tb, Pb = _host(scs, dt)
    wf.wf_batch_run_ptr(b.h, Tb.data_ptr(), Pb.data_ptr(), Tb.data_ptr(), Pb.data_ptr(), n, steps, groups, f32)
    assert wf.wf_sync(b.h) == wf.WF_OK
    b.close()
    assert torch.equal(Ta, Tb) and torch.equal(Pa, Pb)


def test_run_twice_separate_outputs(wf):
    # two calls of one step each give the state of two steps; separate output arrays leave the input
    a, scs = _batch(wf, 4, wf.WF_FP32)
    T0, P0 = _host(scs, torch.float32)
    T1, P1 = torch.empty_like(T0, pin_memory=True), torch.empty_like(P0, pin_memory=True)
    n = T0.numel()
    wf.wf_batch_run_ptr(a.h, T0.data_ptr(), P0.data_ptr(), T1.data_ptr(), P1.data_ptr(), n, 1, 2, True)
    wf.wf_batch_run_ptr(a.h, T1.data_ptr(), P1.data_ptr(), T1.data_ptr(), P1.data_ptr(), n, 1, 2, True)
    a.close()
    b, _ = _batch(wf, 4, wf.WF_FP32)
    b.step(2)
    Tb = np.concatenate([b.state(i)[0].ravel() for i in range(4)])
    b.close()
    T0c, _ = _host(scs, torch.float32)
    assert torch.equal(T0, T0c)  # the input arrays were not written
    assert np.array_equal(T1.numpy().astype(np.float64), Tb)


def test_run_argument_checks(wf):
    a, scs = _batch(wf, 2, wf.WF_FP32)
    T, P = _host(scs, torch.float32)
    L = wf.lib()
    fp = wf.ctypes.POINTER(wf.ctypes.c_float)
    tp, pp = wf.ctypes.cast(T.data_ptr(), fp), wf.ctypes.cast(P.data_ptr(), fp)
    n = T.numel()
    assert L.wf_batch_run_f32(a.h, tp, pp, tp, pp, n + 1, 1, 1) == wf.WF_EINVAL
    assert L.wf_batch_run_f32(a.h, tp, pp, tp, pp, n, -1, 1) == wf.WF_EINVAL
    assert L.wf_batch_run_f32(a.h, tp, pp, tp, pp, n, 1, 0) == wf.WF_EINVAL
    assert L.wf_batch_run_f32(a.h, tp, pp, tp, pp, n, 1, 9) == wf.WF_EINVAL
    assert L.wf_batch_run_f32(a.h, None, pp, tp, pp, n, 1, 1) == wf.WF_EINVAL
    assert L.wf_batch_run_f32(a.h, tp, pp, tp, pp, n, 0, 2) == wf.WF_OK  # no steps: a round trip
    a.close()
