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


T_AMB = 300.0

#: parity bars of the CUDA path against the FP64 oracle, per precision:
#:   rel   relative L2 of T and of phi over the coefficient vectors;
#:   dT    max |T - To| / max(max |To - T_amb|, 1 K) (element by element, against the fire's departure
#:         from ambient, which the background would otherwise hide in the relative L2; at least 1 K,
#:         so that a domain without fire is held to an absolute bar);
#:   dphi  max |phi - phi_o| (fuel is in [0, 1]).
BARS = {"fp64": dict(rel=1e-10, dT=1e-10, dphi=1e-10), "fp32": dict(rel=1e-4, dT=1e-4, dphi=1e-5)}


def parity_errors(T, phi, To, po):
    T, phi, To, po = (np.asarray(a, dtype=np.float64) for a in (T, phi, To, po))
    dev = max(float(np.abs(To - T_AMB).max()), 1.0)
    return dict(rel_T=rel(T, To), rel_phi=rel(phi, po), dT=float(np.abs(T - To).max()) / dev,
                dphi=float(np.abs(phi - po).max()))


def assert_parity(T, phi, To, po, prec, rel_bar=None, dT_bar=None):
    """Element-wise and relative-L2 parity of (T, phi) with the oracle's (To, po) at the bars of `prec`."""
    b = BARS[prec]
    e = parity_errors(T, phi, To, po)
    rb = b["rel"] if rel_bar is None else rel_bar
    assert e["rel_T"] <= rb and e["rel_phi"] <= rb, e
    assert e["dT"] <= (b["dT"] if dT_bar is None else dT_bar), e
    assert e["dphi"] <= b["dphi"], e
    return e


def window(sc, e0x, e0y, n):
    """The scenario restricted to n x n elements starting at element (e0x, e0y): same element size,
    the window's temperature, fuel and wind-factor coefficients (its edges become domain edges)."""
    import dataclasses

    N = n + sc.p
    h = sc.Lx / sc.nx
    cut = lambda a: a[e0y:e0y + N, e0x:e0x + N].copy()  # noqa: E731
    kw = {}
    if sc.wind_rank:
        kw = dict(fx=sc.fx[:, e0x:e0x + N].copy(), gx=sc.gx[:, e0y:e0y + N].copy(),
                  fy=sc.fy[:, e0x:e0x + N].copy(), gy=sc.gy[:, e0y:e0y + N].copy())
    return dataclasses.replace(sc, name=sc.name + "_window", nx=n, ny=n, Lx=n * h, Ly=n * h,
                               T0=cut(sc.T0), fuel0=cut(sc.fuel0), **kw)


def fire_window(sc, n, margin=8):
    """Origin (e0x, e0y) of an n x n element window centred on the hottest coefficient."""
    j, i = np.unravel_index(np.argmax(sc.T0), sc.T0.shape)
    e0x = int(np.clip(i - n // 2, margin, sc.nx - n - margin))
    e0y = int(np.clip(j - n // 2, margin, sc.ny - n - margin))
    return e0x, e0y


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
