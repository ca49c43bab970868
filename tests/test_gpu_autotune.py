"""Launch-shape autotuner: shapes change the schedule, never the arithmetic.

* every launch shape (x lines per CTA, y lines per CTA, quadrature segment rows,
  x lines per warp, second-x-pass lines per CTA, second-x-pass right-hand side fused or in a
  separate matvec) gives bit-for-bit the trajectory of the launchers' own rule, single and
  batched, FP32 and FP64, PR and Strang;
* wf_autotune leaves the device state exactly as it found it and picks shapes
  from its candidate lists;
* the tuned handle then matches the FP64 oracle within the parity bar.
"""
import numpy as np
import pytest

from gpu_helpers import assert_parity, need_gpu, oracle_run, rel
from scenarios import make_scenario

pytestmark = pytest.mark.gpu

SHAPES = [(0, 0, 0, 0, 0, 0), (1, 1, 16, 1, 2, 2), (8, 32, 128, 2, 1, 1), (2, 4, 32, 4, 32, 2),
          (4, 2, 64, 0, 8, 0), (32, 8, 16, 4, 16, 2)]


@pytest.fixture(scope="module")
def wf():
    return need_gpu()


def _sim(wf, sc, prec, scheme):
    return wf.simulation_from_scenario(sc, precision=prec, scheme=scheme)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("scheme", ["pr", "strang"])
def test_shapes_do_not_change_results(wf, prec, scheme):
    P = wf.WF_FP32 if prec == "fp32" else wf.WF_FP64
    code = wf.WF_PR if scheme == "pr" else wf.WF_STRANG_CN
    # rectangular, several chunks per line and several quadrature segments
    sc = make_scenario("shape", 150, 2, 1e-3, 1, 91, wind=(1.2, -0.7), fuel_sigma=3.0)
    ref = None
    # every shape in every step form (per-pass launches; the persistent launch where it applies; the
    # slot-group form, which a single slot runs as per-pass launches)
    for shape in [tuple(s6) + (form, 0) for s6 in SHAPES for form in (1, 2, 3)]:
        sim = _sim(wf, sc, P, code)
        wf.wf_set_tuning(sim.h, shape)
        assert wf.wf_get_tuning(sim.h) == shape
        sim.step(5)
        assert sim.sync() == wf.WF_OK
        T, phi = sim.state()
        sim.close()
        if ref is None:
            ref = (T, phi)
        else:
            assert np.array_equal(T, ref[0]) and np.array_equal(phi, ref[1]), shape


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("p", [1, 3])
def test_shapes_do_not_change_results_p1_p3(wf, prec, p):
    # p = 1 and p = 3: the matvec's items (16 rows; 8 in FP64 at p = 1) and the fused right-hand
    # side give the same bits
    P = wf.WF_FP32 if prec == "fp32" else wf.WF_FP64
    sc = make_scenario(f"shape{p}", 120, p, 1e-3, 1, 95, wind=(-0.9, 1.1), fuel_sigma=3.0)
    ref = None
    for shape in [(0, 0, 0, 0, 0, 0), (8, 16, 32, 2, 4, 2), (1, 4, 16, 1, 2, 1), (4, 2, 64, 0, 8, 2)]:
        sim = _sim(wf, sc, P, wf.WF_PR)
        wf.wf_set_tuning(sim.h, shape)
        sim.step(4)
        assert sim.sync() == wf.WF_OK
        T, phi = sim.state()
        sim.close()
        if ref is None:
            ref = (T, phi)
        else:
            assert np.array_equal(T, ref[0]) and np.array_equal(phi, ref[1]), shape


def test_autotune_keeps_state_and_parity(wf):
    sc = make_scenario("tune", 96, 2, 1e-3, 1, 92, wind=(0.8, 0.4), fuel_sigma=3.0)
    sim = _sim(wf, sc, wf.WF_FP32, wf.WF_PR)
    sim.step(2)
    T0, p0 = sim.state()
    shape = wf.wf_autotune(sim.h, 2)
    assert shape[0] in (0, 32, 16, 8, 4, 2, 1) and shape[1] in (0, 32, 16, 8, 4, 2, 1)
    assert shape[2] in (0, 128, 96, 80, 64, 56, 48, 40, 32, 28, 24, 21, 20, 16, 12) and shape[3] in (0, 1, 2, 4)
    assert shape[4] in (0, 32, 16, 8, 4, 2, 1) and shape[5] in (0, 2)
    assert shape[6] in (0, 1, 2) and shape[7] in (0, 1, 2, 4, 8, 16, 32, 64)
    T1, p1 = sim.state()
    assert np.array_equal(T0, T1) and np.array_equal(p0, p1)
    sim.step(4)
    assert sim.sync() == wf.WF_OK
    T, phi = sim.state()
    sim.close()
    To, po = oracle_run(sc, 6)
    assert_parity(T, phi, To, po, "fp32", rel_bar=1e-5)


def test_autotune_batch_keeps_every_slot(wf):
    scs = [make_scenario(f"tb{i}", 48, 2, 1e-3, 1, 930 + i, wind=((1.0, 0.5), (-2.0, 1.5), (0.0, 0.0))[i],
                         fuel_sigma=3.0) for i in range(3)]
    prm = wf.wf_params_default(Lx=scs[0].Lx, Ly=scs[0].Ly, precision=wf.WF_FP32)
    b = wf.Batch(48, 48, 2, 1e-3, prm, capacity=4)
    for i, sc in enumerate(scs):
        b.load_scenario(i, sc)
    b.step(1)
    before = [b.state(i) for i in range(3)]
    wf.wf_autotune(b.h, 1)
    for i in range(3):
        T, phi = b.state(i)
        assert np.array_equal(T, before[i][0]) and np.array_equal(phi, before[i][1]), i
    b.step(3)
    assert not b.status().any()
    ref = wf.Batch(48, 48, 2, 1e-3, prm, capacity=4)
    for i, sc in enumerate(scs):
        ref.load_scenario(i, sc)
    ref.step(4)
    for i in range(3):
        assert np.array_equal(b.state(i)[0], ref.state(i)[0]), i
    b.close()
    ref.close()


def test_tuning_argument_checks(wf):
    sc = make_scenario("chk", 16, 2, 1e-3, 1, 93)
    sim = _sim(wf, sc, wf.WF_FP32, wf.WF_PR)
    L = wf.lib()
    assert L.wf_autotune(sim.h, 0) == wf.WF_EINVAL
    bad = (wf.ctypes.c_int * 8)(1, -1, 0, 0, 0, 0, 0, 0)
    assert L.wf_set_tuning(sim.h, bad) == wf.WF_EINVAL
    bad = (wf.ctypes.c_int * 8)(0, 0, 0, 0, 0, 3, 0, 0)
    assert L.wf_set_tuning(sim.h, bad) == wf.WF_EINVAL
    bad = (wf.ctypes.c_int * 8)(0, 0, 0, 0, 0, 0, 4, 0)
    assert L.wf_set_tuning(sim.h, bad) == wf.WF_EINVAL
    ok = (wf.ctypes.c_int * 8)(0, 0, 0, 0, 0, 0, 3, 0)
    assert L.wf_set_tuning(sim.h, ok) == wf.WF_OK
    sim.close()


def test_autotune_keeps_forcing_time(wf):
    # every step advances the manufactured solution's time; the tuner's steps must not
    sc = make_scenario("mt", 40, 2, 1e-3, 1, 94)
    sim = _sim(wf, sc, wf.WF_FP64, wf.WF_PR)
    wf.wf_set_mms(sim.h, [(10.0, 1.0, 1.0, 0.5)], 300.0, 0.25)
    sim.step(2)
    t0 = wf.wf_get_time(sim.h)
    T0, _ = sim.state()
    wf.wf_autotune(sim.h, 1)
    assert wf.wf_get_time(sim.h) == t0
    T1, _ = sim.state()
    assert np.array_equal(T0, T1)
    sim.close()
