"""The allocation-free step entry point against the regular step (runs last).

wf_step_noalloc serves callers that cannot allocate device memory while they
step (their device memory belongs to another allocator, or their loop must not
pay cudaMalloc's device synchronisation).  It runs the same step on FP32 arrays
the caller owns, with the step's intermediate fields in a static device array
reserved by the library.  Here the caller's arrays come from torch, with a row
pitch different from the handle's own, and two calls in a row must match two
wf_step calls within the FP32 tolerance of the parity tests.
"""
import numpy as np
import pytest

from gpu_helpers import need_gpu
from scenarios import make_scenario

pytestmark = pytest.mark.gpu


# Nx = 92 here.  Nx + 5: rows of 388 bytes, not a multiple of 16, so the x pass stages its rows
# with plain loads; Nx + 8: 400-byte rows (16-byte multiple, unlike the handle's own 96-element
# pitch), so the x pass stages them with bulk copies at a shared-memory stride of its own.
@pytest.mark.parametrize("extra", [5, 8])
def test_noalloc_step_matches_regular_step(extra):
    wf = need_gpu()
    import torch

    sc = make_scenario("noalloc", 90, 2, 1e-3, 1, 31, wind=(1.2, -0.7), fuel_sigma=3.0)
    ref = wf.simulation_from_scenario(sc, precision=wf.WF_FP32)
    alt = wf.simulation_from_scenario(sc, precision=wf.WF_FP32)
    Nx, Ny = sc.Nx, sc.Ny
    pitch = Nx + extra  # any pitch >= Nx
    T = torch.zeros((Ny, pitch), dtype=torch.float32, device="cuda")
    P = torch.zeros((Ny, pitch), dtype=torch.float32, device="cuda")
    T[:, :Nx] = torch.from_numpy(sc.T0.astype(np.float32))
    P[:, :Nx] = torch.from_numpy(sc.fuel0.astype(np.float32))
    torch.cuda.synchronize()
    for call in range(2):
        ref.step(1)
        Tr, Pr = ref.state()
        assert wf.wf_step_noalloc(alt.h, T.data_ptr(), P.data_ptr(), pitch, 1) == wf.WF_OK
        assert alt.sync() == wf.WF_OK
        Tn = T[:, :Nx].double().cpu().numpy()
        Pn = P[:, :Nx].double().cpu().numpy()
        assert np.linalg.norm(Tn - Tr) / np.linalg.norm(Tr) <= 1e-6, call
        assert np.linalg.norm(Pn - Pr) / np.linalg.norm(Pr) <= 1e-6, call
    # limits are refused before any work is queued
    assert wf.wf_step_noalloc(alt.h, T.data_ptr(), P.data_ptr(), Nx - 1, 1) == wf.WF_EINVAL
    assert wf.wf_step_noalloc(alt.h, T.data_ptr(), P.data_ptr(), (1 << 19) // Ny + 1, 1) == wf.WF_EINVAL
    assert wf.wf_step_noalloc(alt.h, 0, P.data_ptr(), pitch, 1) == wf.WF_EINVAL
    # the manufactured-solution clock belongs to the handle's own trajectory
    wf.wf_set_mms(alt.h, [(10.0, 1, 1, 1.0)])
    assert wf.wf_step_noalloc(alt.h, T.data_ptr(), P.data_ptr(), pitch, 1) == wf.WF_EINVAL
    wf.wf_set_mms(alt.h, None)
    ref.close()
    alt.close()
    big = make_scenario("noalloc_fp64", 20, 2, 1e-3, 1, 3, wind=(0.0, 0.0))
    h64 = wf.simulation_from_scenario(big, precision=wf.WF_FP64)
    assert wf.wf_step_noalloc(h64.h, T.data_ptr(), P.data_ptr(), pitch, 1) == wf.WF_EINVAL
    h64.close()
