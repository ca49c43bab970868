"""Step form 3: the per-pass launches over two groups of slots on two streams.

The first half of the slots runs on the handle's stream, the second half on a second stream whose
quadrature of each step waits for the first group's, so one group's quadrature overlaps the other
group's line passes.  Every slot is independent of the others, so each slot's result must equal
the per-pass form bit for bit: with graphs (several steps per call, groups half a step apart),
eagerly, with odd slot counts, inactive slots, step budgets and every scheme.
"""
import numpy as np
import pytest

from gpu_helpers import assert_parity, need_gpu, oracle_run
from scenarios import make_scenario

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wf():
    return need_gpu()


def _scenarios(n, p, k, base_seed):
    winds = [(1.0, 0.5), (0.0, 0.0), (-2.0, 1.5), (0.3, -2.7), (2.5, 0.0)]
    return [make_scenario(f"g{i}", n, p, 1e-3, 1, base_seed + i, wind=winds[i % 5], fuel_sigma=3.0,
                          wind_perturbation=0.1 if i % 2 == 0 else 0.0) for i in range(k)]


def _run(wf, scs, cap, prec, scheme, form, calls, inactive=(), budgets=None):
    sc0 = scs[0]
    prm = wf.wf_params_default(Lx=sc0.Lx, Ly=sc0.Ly, precision=prec, scheme=scheme)
    b = wf.Batch(sc0.nx, sc0.ny, sc0.p, sc0.dt, prm, capacity=cap)
    for i, sc in enumerate(scs):
        b.load_scenario(i, sc, active=i not in inactive)
    if budgets is not None:
        for i, n in enumerate(budgets):
            wf.wf_batch_set_budget(b.h, i, n)
    wf.wf_set_tuning(b.h, (0, 0, 0, 0, 0, 0, form, 0))
    for n in calls:
        b.step(n)
    st = b.status()
    out = [b.state(i) for i in range(len(scs))]
    assert wf.wf_get_tuning(b.h)[6] == form
    b.close()
    return out, st


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("scheme", ["pr", "strang", "explicit"])
@pytest.mark.parametrize("k,cap", [(5, 5), (4, 7)])
def test_groups_equal_per_pass_bitwise(wf, prec, scheme, k, cap):
    P = wf.WF_FP32 if prec == "fp32" else wf.WF_FP64
    code = {"pr": wf.WF_PR, "strang": wf.WF_STRANG_CN, "explicit": wf.WF_EXPLICIT}[scheme]
    scs = _scenarios(48, 2, k, 900)
    calls = (1, 9, 3)  # one-step graph, an eight-step graph and one more, eager-sized remainders
    a, sa = _run(wf, scs, cap, P, code, 1, calls)
    b, sb = _run(wf, scs, cap, P, code, 3, calls)
    assert not sa.any() and not sb.any()
    for i in range(k):
        assert np.array_equal(a[i][0], b[i][0]) and np.array_equal(a[i][1], b[i][1]), i


def test_groups_with_inactive_slots_and_budgets(wf):
    scs = _scenarios(40, 2, 6, 950)
    calls = (2, 8)
    budgets = [-1, 3, 0, 7, -1, 1]
    a, _ = _run(wf, scs, 6, wf.WF_FP32, wf.WF_PR, 1, calls, inactive=(1, 4), budgets=budgets)
    b, _ = _run(wf, scs, 6, wf.WF_FP32, wf.WF_PR, 3, calls, inactive=(1, 4), budgets=budgets)
    for i in range(6):
        assert np.array_equal(a[i][0], b[i][0]) and np.array_equal(a[i][1], b[i][1]), i
    # an inactive slot and a slot with no budget kept their initial state
    for i in (1, 2, 4):
        T0 = scs[i].T0.astype(np.float32).astype(np.float64)
        f0 = scs[i].fuel0.astype(np.float32).astype(np.float64)
        assert np.array_equal(b[i][0].reshape(T0.shape), T0) and np.array_equal(b[i][1].reshape(f0.shape), f0), i


def test_groups_against_oracle(wf):
    scs = _scenarios(40, 2, 3, 970)
    out, st = _run(wf, scs, 3, wf.WF_FP32, wf.WF_PR, 3, (5,))
    assert not st.any()
    To, po = oracle_run(scs[2], 5, scheme="pr")
    assert_parity(out[2][0], out[2][1], To, po, "fp32")


def test_group_form_on_one_slot_is_per_pass(wf):
    # a single slot has no second group: the per-pass launches run
    sc = _scenarios(40, 2, 1, 990)
    a, _ = _run(wf, sc, 1, wf.WF_FP32, wf.WF_PR, 1, (4,))
    b, _ = _run(wf, sc, 1, wf.WF_FP32, wf.WF_PR, 3, (4,))
    assert np.array_equal(a[0][0], b[0][0]) and np.array_equal(a[0][1], b[0][1])
