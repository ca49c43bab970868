"""Runs of the kind of Sec. 7: a mean wind that changes part-way, and fuel from a raster file.

* two wind phases on the GPU (wf_set_mean_wind between steps) equal the oracle run with
  the same phases, FP64 <= 1e-10 and FP32 <= 1e-5, and a batch slot with the same phases
  equals the single run bit for bit;
* a scenario whose fuel comes from a CSV raster (the listing's fuel_init rule, scale 0.725)
  matches the oracle.
"""
import dataclasses

import numpy as np
import pytest

from gpu_helpers import assert_parity, gpu_run, need_gpu, oracle_run
from oracle.step import Problem
from scenarios import fuel_from_map, gaussian_blur, make_scenario, read_fuel_csv

pytestmark = pytest.mark.gpu

WIND_A = (1.5, 1.5)    # from the south-west
WIND_B = (2.0, -0.3)   # from the west, slightly north


@pytest.fixture(scope="module")
def wf():
    return need_gpu()


def _oracle_two_phase(sc, k, m):
    P = Problem.from_scenario(dataclasses.replace(sc, wind=WIND_A), mode="ads")
    T, phi = P.run(sc.T0, sc.fuel0, k)
    P2 = Problem.from_scenario(dataclasses.replace(sc, wind=WIND_B), mode="ads")
    return P2.run(T, phi, m)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_two_wind_phases(wf, prec, tol):
    sc = make_scenario("w2", 60, 2, 1e-3, 1, 41, wind=WIND_A, fuel_sigma=3.0, wind_perturbation=0.0)
    k, m = 7, 9
    sim = wf.simulation_from_scenario(sc, precision=wf.WF_FP64 if prec == "fp64" else wf.WF_FP32)
    sim.step(k)
    wf.wf_set_mean_wind(sim.h, *WIND_B)
    sim.step(m)
    assert sim.sync() == wf.WF_OK
    T, phi = sim.state()
    sim.close()
    To, po = _oracle_two_phase(sc, k, m)
    assert_parity(T, phi, To, po, prec, rel_bar=tol)


def test_two_wind_phases_in_a_batch_slot(wf):
    sc = make_scenario("w3", 40, 2, 1e-3, 1, 42, wind=WIND_A, fuel_sigma=3.0, wind_perturbation=0.0)
    other = make_scenario("w4", 40, 2, 1e-3, 1, 43, wind=(0.0, 1.0), fuel_sigma=3.0, wind_perturbation=0.0)
    prm = wf.wf_params_default(Lx=sc.Lx, Ly=sc.Ly, precision=wf.WF_FP32)
    b = wf.Batch(40, 40, 2, 1e-3, prm, capacity=2)
    b.load_scenario(0, other)
    b.load_scenario(1, sc)
    b.step(5)
    wf.wf_set_mean_wind(b.h, *WIND_B, slot=1)
    b.step(6)
    Tb, pb = b.state(1)
    b.close()
    sim = wf.simulation_from_scenario(sc, precision=wf.WF_FP32)
    sim.step(5)
    wf.wf_set_mean_wind(sim.h, *WIND_B)
    sim.step(6)
    Ts, ps = sim.state()
    sim.close()
    assert np.array_equal(Tb, Ts) and np.array_equal(pb, ps)


def test_fuel_from_csv_raster(wf, tmp_path):
    rng = np.random.default_rng(7)
    raster = gaussian_blur(rng.random((90, 120)), 3.0)
    raster = np.where(raster > np.median(raster), 1.0, 0.3)  # two fuel classes, as a classified map
    path = tmp_path / "map.csv"
    np.savetxt(path, raster, delimiter=",", fmt="%.3f")
    sc = make_scenario("m", 48, 2, 1e-3, 1, 44, wind=(1.0, 0.5), centred_ignition=True)
    fuel = fuel_from_map(read_fuel_csv(str(path)), sc.nx, sc.ny, sc.p, sc.Lx, sc.Ly)
    sc = dataclasses.replace(sc, fuel0=fuel)
    T, phi = gpu_run(wf, sc, 12, wf.WF_FP64)
    To, po = oracle_run(sc, 12)
    assert_parity(T, phi, To, po, "fp64")
    assert set(np.unique(np.round(fuel, 6))) <= {0.3 * 0.725, 0.725}
