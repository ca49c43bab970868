"""Oracle runs behind the all-steps parity tests at full size, in background processes.

The FP64 oracle steps a 130^2-coefficient window for 1000 steps in about a minute, and the
full-size GPU runs take seconds; so the oracle runs are started (in spawned processes, which
inherit no GPU state) as soon as pytest has collected a test that needs them, and run while the
other GPU tests run.  Each run is a window of elements around the fire of a full-size scenario
(see tests/test_oracle_window.py for why a window stands in for the whole domain), with
snapshots of (T, phi) after the listed step counts.
"""
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

# name -> (configuration, member, window elements, snapshot steps)
JOBS = {
    "c2": ("c2", 0, 128, (150, 1000)),
    "c4_0": ("c4", 0, 100, (100, 2000)),
    "c4_178": ("c4", 178, 100, (100, 2000)),
}

_pool = None
_res = {}


def scenario(kind, member):
    sys.path.insert(0, ROOT)
    from scenarios import config_c2, config_c4

    if kind == "c2":
        return config_c2()
    return config_c4(member, shared_fuel=config_c4(0).fuel0)


def _run(job):
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    sys.path.insert(0, HERE)
    sys.path.insert(0, ROOT)
    from gpu_helpers import fire_window, window
    from oracle.step import Problem

    kind, member, n, snaps = job
    sc = scenario(kind, member)
    e0x, e0y = fire_window(sc, n)
    sub = window(sc, e0x, e0y, n)
    P = Problem.from_scenario(sub, mode="ads")
    T, phi = sub.T0.copy(), sub.fuel0.copy()
    out = {"origin": (e0x, e0y), "n": n}
    done = 0
    for s in snaps:
        for _ in range(s - done):
            T, phi = P.step(T, phi)
        done = s
        out[s] = (T.copy(), phi.copy())
    return out


def start():
    """Start every job (once per process)."""
    global _pool
    if _pool is not None:
        return
    ctx = mp.get_context("spawn")
    env = os.environ.get("CUDA_VISIBLE_DEVICES")
    os.environ["CUDA_VISIBLE_DEVICES"] = ""
    try:
        _pool = ctx.Pool(len(JOBS))
    finally:
        if env is None:
            os.environ.pop("CUDA_VISIBLE_DEVICES", None)
        else:
            os.environ["CUDA_VISIBLE_DEVICES"] = env
    for name, job in JOBS.items():
        _res[name] = _pool.apply_async(_run, (job,))


def result(name, timeout=1500):
    start()
    return _res[name].get(timeout)
