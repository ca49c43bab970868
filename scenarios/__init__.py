"""Seeded synthetic fire scenarios (inputs only).

This package produces the initial temperature and fuel coefficient grids,
the mean wind and the separable wind-perturbation factors that both the CUDA
path and the FP64 CPU oracle consume.  It holds none of the time-step
arithmetic of the method: no quadrature, no matrices, no solves.
"""
from .generate import (  # noqa: F401
    Scenario,
    splitmix64,
    uniform01,
    greville,
    gaussian_blur,
    make_scenario,
    config_c1,
    config_c2,
    config_c3,
    config_c4,
    request_stream_c5,
    element_size,
)
from .fuelmap import FUEL_MAP_SCALE, fuel_from_map, read_fuel_csv, sample_fuel_map  # noqa: F401,E402
