"""Pin of the windowed oracle runs that stand in for full-size parity at 1026^2 and 4099^2 DOFs.

The full-size parity tests run the FP64 oracle on a window of elements around the fire (same
element size; the window's coefficients of temperature, fuel and wind factors; the window's
edges become domain edges with open knots) and compare the interior of the window.  That is
exact up to far below the parity bars when (i) the state near the window's edges is ambient,
where the explicit terms and the increments vanish (T = T_amb is a steady state for any wind
and fuel), and (ii) the window's edges are far enough from the fire that the exponentially
decaying tails of the 1-D inverses (for p = 2 about 0.43 per coefficient) are negligible.
This test checks that claim on a domain the oracle can step in full: the windowed run agrees
with the full run to 1e-12 of the fire's departure from ambient over the window's interior.
"""
import numpy as np

from gpu_helpers import T_AMB, fire_window, window
from oracle.step import Problem
from scenarios import make_scenario

STEPS = 150  # the hottest phase of the fire (the front spreads fastest)


def test_window_run_equals_full_run():
    sc = make_scenario("win", 150, 2, 1e-3, STEPS, 2077, fuel_sigma=20.0, wind_speed_range=(0.0, 3.0))
    assert sc.wind_rank == 2
    P = Problem.from_scenario(sc, mode="ads")
    T, phi = P.run(sc.T0, sc.fuel0, STEPS)
    n = 84
    e0x, e0y = fire_window(sc, n)
    sub = window(sc, e0x, e0y, n)
    Pw = Problem.from_scenario(sub, mode="ads")
    Tw, pw = Pw.run(sub.T0, sub.fuel0, STEPS)
    N = n + sc.p
    edge = 16
    inner = (slice(edge, N - edge), slice(edge, N - edge))
    Tf = T[e0y:e0y + N, e0x:e0x + N][inner]
    pf = phi[e0y:e0y + N, e0x:e0x + N][inner]
    assert Tf.max() > 1500.0  # the fire is inside, burning
    dev = np.abs(Tf - T_AMB).max()
    assert np.abs(Tw[inner] - Tf).max() <= 1e-12 * dev
    assert np.abs(pw[inner] - pf).max() <= 1e-12
    # and outside the window the full run stayed ambient (to the tails)
    mask = np.ones_like(T, dtype=bool)
    mask[e0y:e0y + N, e0x:e0x + N] = False
    assert np.abs(T[mask] - T_AMB).max() <= 1e-9 * dev
