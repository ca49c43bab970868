"""Helpers shared by the GPU parity tests: oracle runs, error metrics, the isotherm criterion."""
import numpy as np
import pytest

from oracle.bspline import eval_local, knots
from oracle.physics import Params
from oracle.step import Problem


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_19370_gb300.build import build_library

    build_library()
    from paper_2604_19370_gb300 import wf

    wf.lib()
    return wf


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def oracle_run(sc, steps, scheme="pr", F_timing="once", prm=None, T0=None, phi0=None):
    prm = prm if prm is not None else Params(F_timing=F_timing)
    P = Problem.from_scenario(sc, prm=prm, scheme=scheme, mode="ads")
    return P.run(sc.T0 if T0 is None else T0, sc.fuel0 if phi0 is None else phi0, steps)


def gpu_run(wf, sc, steps, precision, scheme=None, F_timing=None, T0=None, phi0=None, **kw):
    scheme = wf.WF_PR if scheme is None else scheme
    F_timing = wf.WF_F_ONCE if F_timing is None else F_timing
    sim = wf.simulation_from_scenario(sc, precision=precision, scheme=scheme, F_timing=F_timing, **kw)
    if T0 is not None:
        sim.set_state(T0, sc.fuel0 if phi0 is None else phi0)
    sim.step(steps)
    st = sim.sync()
    T, phi = sim.state()
    sim.close()
    assert st == wf.WF_OK, wf.wf_strerror(st)
    return T, phi


def isotherm_elements(T, n, p, L, level=800.0, sub=2):
    """Elements whose 2x2 sample points straddle the isotherm T = level."""
    t = knots(n, p, L)
    h = L / n
    off = (np.arange(sub) + 0.5) / sub
    e = np.repeat(np.arange(n), sub)
    x = (e + np.tile(off, n)) * h
    B, _ = eval_local(t, p, e, x)  # (n*sub, p+1)
    # dense evaluation matrix (n*sub, N)
    E = np.zeros((n * sub, n + p))
    for l in range(p + 1):
        E[np.arange(n * sub), e + l] = B[:, l]
    V = E @ T @ E.T  # samples [y][x]
    V = V.reshape(n, sub, n, sub)
    lo = V.min(axis=(1, 3))
    hi = V.max(axis=(1, 3))
    return np.argwhere((lo < level) & (hi > level))


def hausdorff_elements(a, b):
    """Symmetric Hausdorff distance between two element index sets (Chebyshev metric)."""
    if len(a) == 0 and len(b) == 0:
        return 0
    if len(a) == 0 or len(b) == 0:
        return np.inf
    d = np.abs(a[:, None, :] - b[None, :, :]).max(axis=2)
    return max(d.min(axis=1).max(), d.min(axis=0).max())
