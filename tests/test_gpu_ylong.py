"""The long-line y pass (k_ysolve_long) against the strip kernel, bit for bit.

Lines of more than eight chunks take the long-line kernel when the launch has enough 32-column
blocks (a batch of several slots of 400^2 elements here); one slot alone takes the shared-memory
strip kernel.  Both perform the same operations in the same order, so every slot of the batch must
equal the same scenario run alone, in every scheme and precision, and one slot the oracle.
"""
import numpy as np
import pytest

from gpu_helpers import assert_parity, gpu_run, need_gpu, oracle_run
from scenarios import make_scenario

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wf():
    return need_gpu()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("scheme", ["pr", "strang", "explicit"])
def test_long_lines_batch_equals_single(wf, prec, scheme):
    P = wf.WF_FP32 if prec == "fp32" else wf.WF_FP64
    code = {"pr": wf.WF_PR, "strang": wf.WF_STRANG_CN, "explicit": wf.WF_EXPLICIT}[scheme]
    winds = [(1.0, 0.5), (-2.0, 1.5), (0.3, -2.7), (2.5, 0.0)]
    scs = [make_scenario(f"yl{i}", 400, 2, 1e-3, 1, 1300 + i, wind=winds[i], fuel_sigma=6.0) for i in range(4)]
    steps = 3
    sc0 = scs[0]
    prm = wf.wf_params_default(Lx=sc0.Lx, Ly=sc0.Ly, precision=P, scheme=code)
    b = wf.Batch(sc0.nx, sc0.ny, sc0.p, sc0.dt, prm, capacity=4)
    for i, sc in enumerate(scs):
        b.load_scenario(i, sc)
    b.step(steps)
    assert not b.status().any()
    for i, sc in enumerate(scs):
        Tb, pb = b.state(i)
        Ts, ps = gpu_run(wf, sc, steps, P, scheme=code)
        assert np.array_equal(Tb, Ts) and np.array_equal(pb, ps), i
    if scheme == "pr":
        To, po = oracle_run(scs[1], steps, scheme="pr")
        Tb, pb = b.state(1)
        assert_parity(Tb, pb, To, po, prec)
    b.close()
