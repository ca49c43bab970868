"""Fuel rasters (the Sec. 7 listing's fuel_init): orientation, cell rule, scale, CSV reading."""
import numpy as np
import pytest

from scenarios import FUEL_MAP_SCALE, fuel_from_map, greville, read_fuel_csv, sample_fuel_map


def _raster():
    # 4 rows (north first) x 5 columns, every cell distinct
    return np.arange(20, dtype=np.float64).reshape(4, 5) / 20.0


def test_orientation_and_cells():
    r = _raster()
    Lx, Ly = 50.0, 40.0  # cells are 10 x 10
    assert FUEL_MAP_SCALE == 0.725
    # north-west corner cell is row 0, column 0; south-east is the last row and column
    assert sample_fuel_map(r, 1.0, 39.0, Lx, Ly) == pytest.approx(r[0, 0] * 0.725)
    assert sample_fuel_map(r, 49.0, 1.0, Lx, Ly) == pytest.approx(r[3, 4] * 0.725)
    # x = 25 falls in column 2; y = 25 is 15 below the northern edge: row 1
    assert sample_fuel_map(r, 25.0, 25.0, Lx, Ly) == pytest.approx(r[1, 2] * 0.725)
    # the closed edges x = Lx and y = 0 read the last column / row
    assert sample_fuel_map(r, 50.0, 0.0, Lx, Ly) == pytest.approx(r[3, 4] * 0.725)
    with pytest.raises(ValueError):
        sample_fuel_map(r, 50.1, 10.0, Lx, Ly)


def test_fuel_from_map_samples_greville_points():
    r = _raster()
    nx, ny, p, Lx, Ly = 7, 6, 2, 50.0, 40.0
    F = fuel_from_map(r, nx, ny, p, Lx, Ly)
    assert F.shape == (ny + p, nx + p)
    gx, gy = greville(nx, p, Lx), greville(ny, p, Ly)
    for j in (0, 3, ny + p - 1):
        for i in (0, 4, nx + p - 1):
            assert F[j, i] == sample_fuel_map(r, gx[i], gy[j], Lx, Ly)


def test_csv_round_trip(tmp_path):
    r = _raster()
    path = tmp_path / "fuel.csv"
    np.savetxt(path, r, delimiter=",")
    assert np.array_equal(read_fuel_csv(str(path)), r)
    bad = tmp_path / "bad.csv"
    bad.write_text("1,2\n3,nan\n")
    with pytest.raises(ValueError):
        read_fuel_csv(str(bad))
