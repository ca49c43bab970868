"""Host checks of the seeded scenario generators (shared input module)."""
import numpy as np

from scenarios import config_c1, greville, make_scenario, splitmix64, uniform01


def test_splitmix64_deterministic_and_uniform():
    a = splitmix64(42, 1000)
    b = splitmix64(42, 1000)
    assert (a == b).all()
    assert (splitmix64(42, 10, offset=5) == a[5:15]).all()
    u = uniform01(7, 200000)
    assert 0.0 <= u.min() and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.005 and abs(u.var() - 1 / 12) < 0.002


def test_greville_symmetric_and_inside():
    for p in (1, 2, 3):
        g = greville(10, p, 15.625)
        assert np.allclose(g + g[::-1], 15.625)
        assert g[0] == 0.0 and g[-1] == 15.625 and (np.diff(g) > 0).all()


def test_c1_recipe():
    sc = config_c1()
    assert (sc.Nx, sc.Ny) == (66, 66) and sc.Lx == 100.0 and sc.wind == (1.0, 0.5)
    assert 0.0 <= sc.fuel0.min() and sc.fuel0.max() <= 1.0
    assert abs(sc.T0.max() - 1000.0) < 50.0 and abs(sc.T0.min() - 300.0) < 1e-9
    assert sc.wind_rank == 2 and sc.wind_packed().size == 2 * 2 * (66 + 66)
    sc2 = config_c1()
    assert np.array_equal(sc.T0, sc2.T0) and np.array_equal(sc.fuel0, sc2.fuel0)


def test_fuel_classes_and_gaps():
    sc = make_scenario("c", 64, 3, 1e-3, 1, 3001, ignitions=3, fuel_sigma=5.0, fuel_classes=True,
                       wind_speed_range=(0.0, 3.0))
    vals = set(np.unique(sc.fuel0).tolist())
    assert vals <= {0.0, 0.2, 1.0} and 0.0 in vals
