"""Serving with continuous batching: every result is the same alone and in the mix.

Requests of different grid sizes, degrees, precisions, schemes, winds and step
counts are submitted in two waves (the second while the first is running, so its
requests join running batches).  Each result must match the same scenario run
alone through a single-scenario handle (bit for bit where the two runs share
their chunk lengths; within 1e-6 relative in FP32 and 1e-12 in FP64 in any case)
and report a positive latency.
"""
import time

import numpy as np
import pytest

from gpu_helpers import gpu_run, need_gpu, rel
from scenarios import make_scenario

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wf():
    return need_gpu()


def _mix():
    out = []
    specs = [(24, 2, "fp32", "pr", 7), (24, 2, "fp32", "pr", 12), (40, 3, "fp32", "pr", 9), (24, 2, "fp64", "pr", 5),
             (40, 3, "fp32", "strang", 6), (24, 2, "fp32", "pr", 30), (40, 3, "fp64", "strang", 4),
             (24, 2, "fp32", "pr", 3)]
    for i, (n, p, prec, scheme, steps) in enumerate(specs):
        wind = [(1.0, 0.5), (-1.5, 2.0), (0.0, 0.0), (2.2, -0.4)][i % 4]
        sc = make_scenario(f"r{i}", n, p, 1e-3, steps, 600 + i, wind=wind, fuel_sigma=2.0,
                           wind_perturbation=0.1 if i % 3 else 0.0)
        out.append((sc, prec, scheme))
    return out


def test_server_results_match_single_runs(wf):
    mix = _mix()
    code = {"fp32": wf.WF_FP32, "fp64": wf.WF_FP64, "pr": wf.WF_PR, "strang": wf.WF_STRANG_CN}
    results = {}
    with wf.Server(2 << 30, max_slots=4) as srv:
        tickets = {}
        for i, (sc, prec, scheme) in enumerate(mix[:4]):
            tickets[srv.submit(sc, precision=code[prec], scheme=code[scheme])] = i
        time.sleep(0.05)
        for i, (sc, prec, scheme) in enumerate(mix[4:], start=4):
            tickets[srv.submit(sc, precision=code[prec], scheme=code[scheme])] = i
        t0 = time.time()
        while tickets and time.time() - t0 < 120:
            for t in list(tickets):
                r = srv.poll(t)
                if r is not None:
                    results[tickets.pop(t)] = r
            time.sleep(0.002)
        assert not tickets, "requests did not finish"
        dof_steps, completed, used = srv.stats()
        assert completed == len(mix) and dof_steps > 0 and used > 0
    for i, (sc, prec, scheme) in enumerate(mix):
        status, res, T, phi = results[i]
        assert status == wf.WF_OK and res.latency_s > 0 and res.run_s >= 0
        Ts, ps = gpu_run(wf, sc, sc.steps, code[prec], scheme=code[scheme])
        tol = 1e-6 if prec == "fp32" else 1e-12
        assert rel(T, Ts) <= tol and rel(phi, ps) <= tol, (i, rel(T, Ts))


def test_server_zero_steps_and_bad_requests(wf):
    sc = make_scenario("z", 16, 2, 1e-3, 0, 3, wind=(1.0, 0.0))
    with wf.Server(1 << 30, max_slots=2) as srv:
        t = srv.submit(sc, steps=0)
        st, res, T, phi = srv.poll(t)
        assert st == wf.WF_OK and np.array_equal(T, sc.T0) and np.array_equal(phi, sc.fuel0)
        with pytest.raises(wf.WFError):
            srv.poll(t)  # reported once
        # a request too large for the budget is refused, not stalled
    with wf.Server(1 << 20, max_slots=1) as srv:
        big = make_scenario("big", 200, 2, 1e-3, 3, 4, wind=(0.0, 0.0))
        t = srv.submit(big)
        t0 = time.time()
        r = None
        while r is None and time.time() - t0 < 30:
            r = srv.poll(t)
            time.sleep(0.01)
        assert r is not None and r[0] == wf.WF_ENOMEM


def test_served_results_against_oracle(wf):
    # a sample of served requests, FP32 and FP64, checked element by element against the oracle
    from gpu_helpers import assert_parity, oracle_run

    reqs = [(make_scenario("so0", 48, 2, 1e-3, 17, 801, wind=(1.0, -0.5), fuel_sigma=3.0), "fp32"),
            (make_scenario("so1", 48, 2, 1e-3, 9, 802, wind=(-2.0, 0.7), fuel_sigma=3.0), "fp32"),
            (make_scenario("so2", 36, 2, 1e-3, 11, 803, wind=(0.4, 1.9), fuel_sigma=3.0), "fp64"),
            (make_scenario("so3", 30, 3, 1e-3, 6, 804, wind=(0.0, 0.0), fuel_sigma=3.0), "fp64")]
    code = {"fp32": wf.WF_FP32, "fp64": wf.WF_FP64}
    out = {}
    with wf.Server(1 << 30, max_slots=4) as srv:
        tickets = {srv.submit(sc, precision=code[prec]): i for i, (sc, prec) in enumerate(reqs)}
        t0 = time.time()
        while tickets and time.time() - t0 < 120:
            for t in list(tickets):
                r = srv.poll(t)
                if r is not None:
                    out[tickets.pop(t)] = r
            time.sleep(0.002)
        assert not tickets
    for i, (sc, prec) in enumerate(reqs):
        st, res, T, phi = out[i]
        assert st == wf.WF_OK
        To, po = oracle_run(sc, sc.steps)
        assert_parity(T, phi, To, po, prec, rel_bar=1e-10 if prec == "fp64" else 1e-5)


@pytest.mark.parametrize("form", [1, 2])
def test_step_budgets_give_each_slot_its_own_count(wf, form):
    # one wf_step(n) with per-slot budgets advances each slot by min(n, its budget); in both step
    # forms; a slot re-armed afterwards continues from where it stopped
    scs = [make_scenario(f"bg{i}", 64, 2, 1e-3, 1, 820 + i, wind=((1.0, 0.5), (0.0, -1.0), (2.0, 2.0))[i],
                         fuel_sigma=3.0) for i in range(3)]
    counts = [3, 8, 5]
    prm = wf.wf_params_default(Lx=scs[0].Lx, Ly=scs[0].Ly, wind_x=1.0, wind_y=0.5, precision=wf.WF_FP32)
    b = wf.Batch(64, 64, 2, 1e-3, prm, capacity=3)
    wf.wf_set_tuning(b.h, (0, 0, 0, 0, 0, 0, form, 0))
    for i, sc in enumerate(scs):
        b.load_scenario(i, sc)
        wf.wf_batch_set_budget(b.h, i, counts[i])
    b.step(10)
    assert wf.wf_sync(b.h) == wf.WF_OK
    got = [b.state(i) for i in range(3)]
    wf.wf_batch_set_budget(b.h, 0, 2)
    wf.wf_batch_activate(b.h, 0, True)
    b.step(4)
    T0b, _ = b.state(0)
    b.close()
    for i, sc in enumerate(scs):
        T, phi = gpu_run(wf, sc, counts[i], wf.WF_FP32)
        assert np.array_equal(got[i][0], T) and np.array_equal(got[i][1], phi), i
    T, _ = gpu_run(wf, scs[0], counts[0] + 2, wf.WF_FP32)
    assert np.array_equal(T0b, T)
