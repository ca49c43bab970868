"""Fuel maps from raster files (inputs only).

The paper's runs read a satellite-derived fuel raster and initialise the fuel from it
(Sec. 7 listing, "fuel_init"): a point (x, y) of the domain [0, L_x] x [0, L_y] reads the
raster cell (row floor(rows (L_y - y) / L_y), column floor(cols x / L_x)) -- row 0 is the
northern edge -- and the value is scaled by 0.725.  The real maps are not available here;
these functions read any comma-separated raster of that layout.

Reading: the fuel coefficients are the map sampled at the Greville abscissae (as every
other initial field here); the closed domain edges x = L_x and y = 0, which the listing's
floor maps one cell past the raster, read the last cell.
"""
from __future__ import annotations

import numpy as np

from .generate import greville

FUEL_MAP_SCALE = 0.725


def read_fuel_csv(path: str) -> np.ndarray:
    """Raster rows (north first) of a comma-separated file, as float64."""
    a = np.loadtxt(path, delimiter=",", dtype=np.float64, ndmin=2)
    if a.size == 0 or not np.all(np.isfinite(a)):
        raise ValueError(f"{path}: empty or non-finite fuel raster")
    return a


def sample_fuel_map(raster: np.ndarray, x, y, Lx: float, Ly: float, scale: float = FUEL_MAP_SCALE):
    """Fuel at points (x, y) of [0, Lx] x [0, Ly] by the listing's nearest-cell rule."""
    rows, cols = raster.shape
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    if np.any(x < 0) or np.any(x > Lx) or np.any(y < 0) or np.any(y > Ly):
        raise ValueError("fuel map sampled outside the domain")
    mx = np.minimum(np.floor(cols / Lx * x).astype(np.int64), cols - 1)
    my = np.minimum(np.floor(rows / Ly * (Ly - y)).astype(np.int64), rows - 1)
    return raster[my, mx] * scale


def fuel_from_map(raster: np.ndarray, nx: int, ny: int, p: int, Lx: float, Ly: float,
                  scale: float = FUEL_MAP_SCALE) -> np.ndarray:
    """Fuel coefficient grid (Ny, Nx) of the spline space: the map at the Greville abscissae."""
    gx = greville(nx, p, Lx)
    gy = greville(ny, p, Ly)
    return sample_fuel_map(raster, gx[None, :], gy[:, None], Lx, Ly, scale)
