"""Batches of scenarios in one launch: each slot's result equals the same scenario run alone.

A batch steps every active slot with one launch per kernel (slots are the third
grid dimension); slots carry their own state, mean wind (hence operators) and wind
variation.  The computation of a slot does not depend on the other slots, so a
slot's result must be bit-for-bit the single-scenario result, and within the
parity bar of the FP64 oracle.
"""
import numpy as np
import pytest

from gpu_helpers import assert_parity, gpu_run, need_gpu, oracle_run, rel
from scenarios import make_scenario

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wf():
    return need_gpu()


def _scenarios(n, p, k, base_seed):
    out = []
    for i in range(k):
        wind = [(1.0, 0.5), (0.0, 0.0), (-2.0, 1.5), (0.3, -2.7), (2.5, 0.0)][i % 5]
        out.append(make_scenario(f"b{i}", n, p, 1e-3, 1, base_seed + i, wind=wind, fuel_sigma=3.0,
                                 wind_perturbation=0.1 if i % 2 == 0 else 0.0))
    return out


def _batch_params(wf, sc, prec, scheme):
    return wf.wf_params_default(Lx=sc.Lx, Ly=sc.Ly, precision=prec, scheme=scheme)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("scheme", ["pr", "strang", "explicit"])
def test_batch_slots_equal_single_runs(wf, prec, scheme):
    P = wf.WF_FP32 if prec == "fp32" else wf.WF_FP64
    code = {"pr": wf.WF_PR, "strang": wf.WF_STRANG_CN, "explicit": wf.WF_EXPLICIT}[scheme]
    scs = _scenarios(40, 2, 5, 700)
    steps = 4
    b = wf.Batch(scs[0].nx, scs[0].ny, 2, 1e-3, _batch_params(wf, scs[0], P, code), capacity=6)
    for i, sc in enumerate(scs):
        b.load_scenario(i, sc)
    b.step(steps)
    assert not b.status().any()
    for i, sc in enumerate(scs):
        Tb, pb = b.state(i)
        Ts, ps = gpu_run(wf, sc, steps, P, scheme=code)
        assert np.array_equal(Tb, Ts) and np.array_equal(pb, ps), i
    # one slot against the oracle
    To, po = oracle_run(scs[2], steps, scheme=scheme)
    Tb, pb = b.state(2)
    assert_parity(Tb, pb, To, po, prec, rel_bar=1e-10 if prec == "fp64" else 1e-5)
    # the unused slot stayed zero
    Tz, pz = b.state(5)
    assert not Tz.any() and not pz.any()
    b.close()


def test_slots_join_and_leave_between_steps(wf):
    # continuous batching: slot 1 joins after 3 steps, slot 0 leaves after 5
    scs = _scenarios(30, 2, 2, 900)
    b = wf.Batch(30, 30, 2, 1e-3, _batch_params(wf, scs[0], wf.WF_FP32, wf.WF_PR), capacity=2)
    b.load_scenario(0, scs[0])
    b.step(3)
    b.load_scenario(1, scs[1])
    b.step(2)
    b.activate(0, False)
    b.step(4)
    T0, p0 = b.state(0)
    T1, p1 = b.state(1)
    b.close()
    Ta, pa = gpu_run(wf, scs[0], 5, wf.WF_FP32)
    Tb, pb = gpu_run(wf, scs[1], 6, wf.WF_FP32)
    assert np.array_equal(T0, Ta) and np.array_equal(p0, pa)
    assert np.array_equal(T1, Tb) and np.array_equal(p1, pb)


def test_batch_guard_is_per_slot(wf):
    scs = _scenarios(20, 2, 3, 950)
    b = wf.Batch(20, 20, 2, 1e-3, _batch_params(wf, scs[0], wf.WF_FP32, wf.WF_PR), capacity=3)
    for i, sc in enumerate(scs):
        T0 = sc.T0.copy()
        if i == 1:
            T0[3, 4] = np.inf
        b.set_slot(i, T0, sc.fuel0, sc.wind, sc.wind_rank, sc.wind_packed())
        b.activate(i, True)
    b.step(2)
    st = b.status()
    assert list(st) == [0, 1, 0]
    assert not b.status().any()  # cleared by the call
    b.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_whole_batch_state_io(wf, prec):
    # one call for every slot's state (float64 and float32 host arrays) equals slot-by-slot transfers
    scs = _scenarios(40, 2, 3, 800)
    P = wf.WF_FP32 if prec == "fp32" else wf.WF_FP64
    prm = _batch_params(wf, scs[0], P, wf.WF_PR)
    a = wf.Batch(40, 40, 2, 1e-3, prm, capacity=3)
    b = wf.Batch(40, 40, 2, 1e-3, prm, capacity=3)
    for i, sc in enumerate(scs):
        a.load_scenario(i, sc)
        b.load_scenario(i, sc)
    n = scs[0].T0.size
    T32 = np.stack([sc.T0 for sc in scs]).astype(np.float32).ravel()
    F32 = np.stack([sc.fuel0 for sc in scs]).astype(np.float32).ravel()
    for i, sc in enumerate(scs):  # same values through the per-slot float64 call
        wf.wf_batch_set_slot(a.h, i, T32[i * n:(i + 1) * n].astype(np.float64),
                             F32[i * n:(i + 1) * n].astype(np.float64), sc.wind[0], sc.wind[1],
                             sc.wind_rank, sc.wind_packed())
    wf.wf_batch_states_ptr(b.h, T32.ctypes.data, F32.ctypes.data, 3 * n, True, True)
    a.step(2)
    b.step(2)
    T64 = np.empty(3 * n)
    F64 = np.empty(3 * n)
    wf.wf_batch_states_ptr(b.h, T64.ctypes.data, F64.ctypes.data, 3 * n, False, False)
    To32 = np.empty(3 * n, dtype=np.float32)
    wf.wf_batch_states_ptr(b.h, To32.ctypes.data, 0, 3 * n, True, False)
    for i in range(3):
        Ta, Fa = a.state(i)
        assert np.array_equal(T64[i * n:(i + 1) * n], Ta.ravel()), i
        assert np.array_equal(F64[i * n:(i + 1) * n], Fa.ravel()), i
        assert np.array_equal(To32[i * n:(i + 1) * n], Ta.ravel().astype(np.float32)), i
    with pytest.raises(wf.WFError):
        wf.wf_batch_states_ptr(b.h, T64.ctypes.data, F64.ctypes.data, 3 * n - 1, False, True)
    a.close()
    b.close()
