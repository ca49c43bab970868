"""The persistent form (the quadrature launch, then one launch over every line pass of every active
slot) against the per-pass launches.

The persistent kernel runs the tiles of the per-pass kernels (the same device functions or the
same operations in the same order) under a different schedule: work items claimed from a
ticket counter in a wavefront over groups of slots, with per-slot arrival counters between the
passes.  Its results must therefore equal the per-pass launches bit for bit whatever the
schedule (group size, lines per tile, slots joining and leaving), in FP32 and FP64, p = 1..3,
and sit within the parity bars of the FP64 oracle.  A zero wait limit makes its counter waits
give up: the step reports WF_ETIMEOUT, nothing hangs, and the handle steps normally afterwards.
"""
import numpy as np
import pytest

from gpu_helpers import assert_parity, need_gpu, oracle_run
from scenarios import make_scenario

pytestmark = pytest.mark.gpu

PER_PASS, PERSIST = 1, 2


@pytest.fixture(scope="module")
def wf():
    return need_gpu()


def _run(wf, scs, steps, form, shape=(0, 0, 0, 0, 0, 0, 0, 0), active=None, prec=None):
    sc0 = scs[0]
    prec = wf.WF_FP32 if prec is None else prec
    prm = wf.wf_params_default(Lx=sc0.Lx, Ly=sc0.Ly, wind_x=sc0.wind[0], wind_y=sc0.wind[1], precision=prec)
    b = wf.Batch(sc0.nx, sc0.ny, sc0.p, sc0.dt, prm, capacity=len(scs))
    for k, sc in enumerate(scs):
        b.load_scenario(k, sc, active=True if active is None else bool(active[k]))
    s = list(shape)
    s[6] = form
    wf.wf_set_tuning(b.h, s)
    b.step(steps)
    st = wf.wf_sync(b.h)
    out = [b.state(k) for k in range(len(scs))]
    b.close()
    return st, out


def _scs(n, p, k, seed, rank=True):
    winds = [(1.0, 0.5), (0.0, 0.0), (-2.0, 1.5), (0.3, -2.7), (2.5, 0.0)]
    return [make_scenario(f"pp{i}", n, p, 1e-3, 1, seed + i, wind=winds[i % 5], fuel_sigma=3.0,
                          wind_perturbation=0.1 if (rank and i % 2 == 0) else 0.0) for i in range(k)]


@pytest.mark.parametrize("n,p,k,prec", [(40, 2, 1, "fp32"), (96, 2, 3, "fp32"), (150, 2, 2, "fp32"), (61, 1, 3, "fp32"),
                                        (7, 2, 2, "fp32"), (300, 2, 1, "fp32"), (70, 3, 3, "fp32"), (90, 2, 3, "fp64"),
                                        (50, 3, 2, "fp64"), (33, 1, 2, "fp64")])
def test_persistent_equals_per_pass_bitwise(wf, n, p, k, prec):
    scs = _scs(n, p, k, 900 + n + p)
    P = wf.WF_FP32 if prec == "fp32" else wf.WF_FP64
    st1, a = _run(wf, scs, 4, PER_PASS, prec=P)
    st2, b = _run(wf, scs, 4, PERSIST, prec=P)
    assert st1 == wf.WF_OK and st2 == wf.WF_OK
    for i in range(k):
        assert np.array_equal(a[i][0], b[i][0]) and np.array_equal(a[i][1], b[i][1]), i


@pytest.mark.parametrize("shape", [(0, 0, 16, 0, 0, 0, 0, 1), (8, 4, 32, 1, 0, 0, 0, 2), (2, 16, 128, 2, 0, 0, 0, 5),
                                   (32, 1, 20, 4, 0, 0, 0, 3), (4, 2, 0, 0, 0, 0, 0, 64)])
def test_persistent_schedules_bitwise(wf, shape):
    # group size, lines per tile and lines per warp change the schedule only
    scs = _scs(120, 2, 5, 950, rank=False)
    st1, ref = _run(wf, scs, 3, PER_PASS)
    st2, got = _run(wf, scs, 3, PERSIST, shape=shape)
    assert st1 == wf.WF_OK and st2 == wf.WF_OK
    for i in range(len(scs)):
        assert np.array_equal(ref[i][0], got[i][0]) and np.array_equal(ref[i][1], got[i][1]), (shape, i)


def test_persistent_slots_join_and_leave(wf):
    # the item list follows the active slots between steps; inactive slots stay untouched
    scs = _scs(80, 2, 4, 970)
    sc0 = scs[0]
    res = {}
    for form in (PER_PASS, PERSIST):
        prm = wf.wf_params_default(Lx=sc0.Lx, Ly=sc0.Ly, wind_x=sc0.wind[0], wind_y=sc0.wind[1],
                                   precision=wf.WF_FP32)
        b = wf.Batch(sc0.nx, sc0.ny, 2, 1e-3, prm, capacity=4)
        wf.wf_set_tuning(b.h, (0, 0, 0, 0, 0, 0, form, 0))
        for k, sc in enumerate(scs):
            b.load_scenario(k, sc, active=k != 2)
        b.step(2)
        b.activate(2, True)
        b.activate(0, False)
        b.step(3)
        b.activate(0, True)
        b.step(1)
        assert wf.wf_sync(b.h) == wf.WF_OK
        res[form] = [b.state(k) for k in range(4)]
        b.close()
    for k in range(4):
        assert np.array_equal(res[PER_PASS][k][0], res[PERSIST][k][0]), k
        assert np.array_equal(res[PER_PASS][k][1], res[PERSIST][k][1]), k


def test_persistent_against_oracle(wf):
    sc = make_scenario("po", 130, 2, 1e-3, 6, 991, wind=(1.3, -0.6), fuel_sigma=3.0)
    _, out = _run(wf, [sc], sc.steps, PERSIST)
    T, phi = out[0]
    To, po = oracle_run(sc, sc.steps)
    assert_parity(T, phi, To, po, "fp32", rel_bar=1e-5)


@pytest.mark.parametrize("k", [1, 4])
def test_persistent_wait_limit_zero(wf, k):
    scs = _scs(100, 2, k, 1010)
    sc0 = scs[0]
    prm = wf.wf_params_default(Lx=sc0.Lx, Ly=sc0.Ly, wind_x=sc0.wind[0], wind_y=sc0.wind[1], precision=wf.WF_FP32)
    b = wf.Batch(sc0.nx, sc0.ny, 2, 1e-3, prm, capacity=k)
    wf.wf_set_tuning(b.h, (0, 0, 0, 0, 0, 0, PERSIST, 0))
    for i, sc in enumerate(scs):
        b.load_scenario(i, sc)
    wf.wf_set_wait_limit(b.h, 0.0)
    b.step(3)
    assert wf.wf_sync(b.h) == wf.WF_ETIMEOUT
    wf.wf_set_wait_limit(b.h, 1.0)
    for i, sc in enumerate(scs):
        b.load_scenario(i, sc)
    b.step(2)
    assert wf.wf_sync(b.h) == wf.WF_OK
    got = [b.state(i) for i in range(k)]
    b.close()
    _, ref = _run(wf, scs, 2, PER_PASS)
    for i in range(k):
        assert np.array_equal(got[i][0], ref[i][0]) and np.array_equal(got[i][1], ref[i][1]), i
