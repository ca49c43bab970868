"""Convergence study with the manufactured solution (Sec. 6), on the GPU through the C ABI.

For meshes 50^2, 100^2, 200^2 (quadratic B-splines on [0, 100]^2) and time steps 1 .. 1/128
covering [0, 1], runs the explicit scheme, Peaceman-Rachford and Strang/Crank-Nicolson with
the forcing of u*, from the L2 projection of u*(., 0), and prints the relative error over
the whole interval, sqrt(sum_n ||u_h(t_n) - u*(t_n)||^2) / sqrt(sum_n ||u*(t_n)||^2), as a
Markdown table ("unstable" where the solution blew up).  The L2 norms come from the oracle's
quadrature of u*; the solver is the CUDA path in FP64.

  python tests/mms_study.py [--meshes 50,100,200] [--nonlinear]
"""
import argparse
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

from oracle.bspline import ElementTables  # noqa: E402
from oracle.mms import PAPER_MODES, Manufactured  # noqa: E402
from paper_2604_19370_gb300 import wf  # noqa: E402
from paper_2604_19370_gb300.build import build_library  # noqa: E402

L = 100.0
WIND = (1.0, 0.5)
TAUS = [1.0 / 2 ** k for k in range(8)]


def run(n, tau, scheme, nonlinear):
    m = Manufactured()
    tx = ElementTables(n, 2, L)
    T = m.project(tx, tx, 0.0)
    extra = {} if nonlinear else {"sigma": 0.0}
    prm = wf.wf_params_default(Lx=L, Ly=L, wind_x=WIND[0], wind_y=WIND[1], precision=wf.WF_FP64, scheme=scheme,
                               heat_scale=0.0, **extra)
    sim = wf.Simulation(n, n, 2, tau, prm)
    wf.wf_set_mms(sim.h, list(PAPER_MODES), 300.0, 0.0)
    sim.set_state(T, np.zeros_like(T))
    se = sr = 0.0
    steps = int(round(1.0 / tau))
    for k in range(steps):
        sim.step(1)
        Tk, _ = sim.state()
        if not np.all(np.isfinite(Tk)) or np.abs(Tk).max() > 1e6:
            sim.close()
            return None
        e, r = m.l2_norms(tx, tx, Tk, (k + 1) * tau)
        se += e * e
        sr += r * r
    sim.close()
    return float(np.sqrt(se / sr))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--meshes", default="50,100,200")
    ap.add_argument("--nonlinear", action="store_true")
    args = ap.parse_args()
    build_library()
    schemes = [("explicit", wf.WF_EXPLICIT), ("PR", wf.WF_PR), ("Strang-CN", wf.WF_STRANG_CN)]
    print(f"problem: {'nonlinear (T^3 diffusion, radiation)' if args.nonlinear else 'linear'}; "
          f"wind {WIND}; relative error over [0, 1]")
    print("| mesh | scheme | " + " | ".join(f"tau=1/{int(round(1 / t))}" for t in TAUS) + " |")
    print("|---|---|" + "---|" * len(TAUS))
    for n in [int(v) for v in args.meshes.split(",")]:
        for name, code in schemes:
            cells = []
            for tau in TAUS:
                e = run(n, tau, code, args.nonlinear)
                cells.append("unstable" if e is None else f"{e:.3e}")
            print(f"| {n}x{n} | {name} | " + " | ".join(cells) + " |", flush=True)


if __name__ == "__main__":
    main()
