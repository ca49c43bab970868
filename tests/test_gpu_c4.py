"""The batched ensemble at full size: 256 scenarios of 256 x 256 elements (p = 2, 66,564 DOFs each,
17.0M in all) in one batch handle, FP32, autotuned launch shapes, steps replayed from the captured
graph, as the ensemble bench runs them.

The oracle steps single scenarios of this size in about a third of a second, so sampled slots (the
first, the last and two in between) are compared with it element by element (the bars of
gpu_helpers.BARS: max |T - To| against max |To - T_amb|, max |phi - phi_o|, and the relative L2);
every slot is also checked to be finite, inside the guard and unflagged.  The all-steps comparison
of sampled members is in test_gpu_zlong.py.
"""
import numpy as np
import pytest

from gpu_helpers import assert_parity, need_gpu, oracle_run
from scenarios import config_c4

pytestmark = pytest.mark.gpu

S = 256
STEPS = 2
SAMPLED = (0, 97, 178, 255)


@pytest.fixture(scope="module")
def wf():
    return need_gpu()


def test_c4_full_ensemble_sampled_slots(wf):
    first = config_c4(0)
    shared = first.fuel0
    scs = [first] + [config_c4(k, shared_fuel=shared) for k in range(1, S)]
    prm = wf.wf_params_default(Lx=first.Lx, Ly=first.Ly, precision=wf.WF_FP32)
    b = wf.Batch(first.nx, first.ny, first.p, first.dt, prm, capacity=S)
    try:
        for k, sc in enumerate(scs):
            b.load_scenario(k, sc)
        wf.wf_autotune(b.h, 1)
        b.step(STEPS)
        assert not b.status().any()
        for k in range(S):
            T, phi = b.state(k)
            assert np.all(np.isfinite(T)) and np.all(np.abs(T) < 1e5), k
        for k in SAMPLED:
            T, phi = b.state(k)
            To, po = oracle_run(scs[k], STEPS)
            assert_parity(T, phi, To, po, "fp32", rel_bar=1e-5)
    finally:
        b.close()
