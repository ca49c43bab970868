"""Python binding of libwf (include/wf.h): argument marshalling only.

Every function keeps the C name and forwards to the shared library through
ctypes; all arithmetic of the time step runs in the library's CUDA kernels.
There is no fallback: if libwf.so has not been built, importing the
library raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Tuple

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libwf.so")

WF_OK = 0
WF_PENDING = 1
WF_EINVAL = -1
WF_ENOMEM = -2
WF_ESINGULAR = -3
WF_EUNSTABLE = -4
WF_ETIMEOUT = -5
WF_ECUDA = -6
WF_ETRUNC = -7
WF_ENOTFOUND = -8
WF_PR = 0
WF_STRANG_CN = 1
WF_FP32 = 0
WF_FP64 = 1
WF_F_ONCE = 0
WF_F_PER_SUBSTEP = 1


class wf_params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "Lx", "Ly", "rho", "cp", "kappa", "sigma", "eps", "ch", "hc", "cW", "chi", "T_amb", "T_ig",
        "delta_x", "delta_z", "A_r", "M_ratio", "T_a", "heat_scale", "fuel_rate", "fuel_thresh",
        "thresh_guard", "wind_x", "wind_y")] + [(n, ctypes.c_int) for n in (
        "scheme", "precision", "F_timing", "scale_heat_by_fuel")]


class WFError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {wf_strerror(code)} ({code})")


_lib = None


def lib() -> ctypes.CDLL:
    """Load libwf.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libwf.so is not built ({LIB_PATH}); run paper_2604_19370_gb300.build")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
        dp = ctypes.POINTER(ctypes.c_double)
        L.wf_params_default.argtypes = [ctypes.POINTER(wf_params)]
        L.wf_create.argtypes = [i, i, i, d, ctypes.POINTER(wf_params), ctypes.POINTER(vp)]
        L.wf_set_state.argtypes = [vp, dp, dp, sz]
        L.wf_set_wind.argtypes = [vp, i, dp]
        L.wf_step.argtypes = [vp, i]
        L.wf_sync.argtypes = [vp]
        L.wf_get_state.argtypes = [vp, dp, dp, sz]
        L.wf_get_dims.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]
        L.wf_set_stream.argtypes = [vp, vp]
        L.wf_set_profiling.argtypes = [vp, i]
        L.wf_kernel_times.argtypes = [vp, dp, ctypes.POINTER(i), ctypes.c_void_p, i]
        L.wf_step_noalloc.argtypes = [vp, vp, vp, i, i]
        L.wf_destroy.argtypes = [vp]
        L.wf_destroy.restype = None
        L.wf_strerror.argtypes = [i]
        L.wf_strerror.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(code: int, where: str) -> int:
    if code < 0:
        raise WFError(code, where)
    return code


def _dptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _host(a, n: int) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64).ravel()
    if a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def wf_strerror(code: int) -> str:
    return lib().wf_strerror(code).decode()


def wf_params_default(**overrides) -> wf_params:
    p = wf_params()
    _check(lib().wf_params_default(ctypes.byref(p)), "wf_params_default")
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def wf_create(nx: int, ny: int, p: int, dt: float, params: wf_params) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().wf_create(nx, ny, p, dt, ctypes.byref(params), ctypes.byref(h)), "wf_create")
    return h


def wf_get_dims(h) -> Tuple[int, int, int, int]:
    a, b, c, d = (ctypes.c_int() for _ in range(4))
    _check(lib().wf_get_dims(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)), "wf_get_dims")
    return a.value, b.value, c.value, d.value


def wf_set_state(h, T, fuel) -> None:
    Nx, Ny, _, _ = wf_get_dims(h)
    n = Nx * Ny
    Ta, Fa = _host(T, n), _host(fuel, n)
    _check(lib().wf_set_state(h, _dptr(Ta), _dptr(Fa), n), "wf_set_state")


def wf_set_state_ptr(h, T_ptr: int, fuel_ptr: int, n: int) -> None:
    """Same call with raw host addresses (e.g. pinned buffers owned by the caller)."""
    dp = ctypes.POINTER(ctypes.c_double)
    _check(lib().wf_set_state(h, ctypes.cast(T_ptr, dp), ctypes.cast(fuel_ptr, dp), n), "wf_set_state")


def wf_set_wind(h, rank: int, factors=None) -> None:
    arr = None if factors is None else np.ascontiguousarray(factors, dtype=np.float64).ravel()
    _check(lib().wf_set_wind(h, rank, _dptr(arr)), "wf_set_wind")


def wf_step(h, nsteps: int) -> None:
    _check(lib().wf_step(h, nsteps), "wf_step")


def wf_sync(h) -> int:
    """Returns the status code (WF_OK or WF_EUNSTABLE); raises on other errors."""
    code = lib().wf_sync(h)
    if code < 0 and code != WF_EUNSTABLE:
        raise WFError(code, "wf_sync")
    return code


def wf_get_state(h) -> Tuple[np.ndarray, np.ndarray]:
    Nx, Ny, _, _ = wf_get_dims(h)
    T = np.empty((Ny, Nx))
    F = np.empty((Ny, Nx))
    _check(lib().wf_get_state(h, _dptr(T), _dptr(F), Nx * Ny), "wf_get_state")
    return T, F


def wf_get_state_ptr(h, T_ptr: int, fuel_ptr: int, n: int) -> None:
    dp = ctypes.POINTER(ctypes.c_double)
    _check(lib().wf_get_state(h, ctypes.cast(T_ptr, dp), ctypes.cast(fuel_ptr, dp), n), "wf_get_state")


def wf_set_stream(h, stream_ptr: Optional[int]) -> None:
    _check(lib().wf_set_stream(h, ctypes.c_void_p(stream_ptr or 0)), "wf_set_stream")


def wf_set_profiling(h, on: bool) -> None:
    _check(lib().wf_set_profiling(h, 1 if on else 0), "wf_set_profiling")


def wf_kernel_times(h, max_k: int = 16):
    ms = (ctypes.c_double * max_k)()
    cnt = (ctypes.c_int * max_k)()
    names = (ctypes.c_char * (48 * max_k))()
    k = _check(lib().wf_kernel_times(h, ms, cnt, ctypes.cast(names, ctypes.c_void_p), max_k), "wf_kernel_times")
    out = {}
    for j in range(min(k, max_k)):
        nm = bytes(names[48 * j:48 * (j + 1)]).split(b"\0")[0].decode()
        out[nm] = (ms[j], cnt[j])
    return out


def wf_step_noalloc(h, T_dev_ptr: int, fuel_dev_ptr: int, pitch: int, nsteps: int) -> int:
    """Allocation-free steps on caller-owned FP32 device arrays (returns the status code)."""
    return lib().wf_step_noalloc(h, ctypes.c_void_p(T_dev_ptr), ctypes.c_void_p(fuel_dev_ptr), pitch, nsteps)


def wf_destroy(h) -> None:
    if h:
        lib().wf_destroy(h)


class Simulation:
    """Owning wrapper around one handle (same calls, Python life cycle)."""

    def __init__(self, nx, ny, p, dt, params: wf_params):
        self.h = wf_create(nx, ny, p, dt, params)
        self.Nx, self.Ny, self.p, self.precision = wf_get_dims(self.h)

    def set_state(self, T, fuel):
        wf_set_state(self.h, T, fuel)

    def set_wind(self, rank, factors=None):
        wf_set_wind(self.h, rank, factors)

    def step(self, n=1):
        wf_step(self.h, n)

    def sync(self):
        return wf_sync(self.h)

    def state(self):
        return wf_get_state(self.h)

    def close(self):
        if self.h:
            wf_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def simulation_from_scenario(sc, precision=WF_FP32, scheme=WF_PR, F_timing=WF_F_ONCE, **overrides) -> Simulation:
    """Create a handle for a `scenarios.Scenario`, load its state and wind variation."""
    prm = wf_params_default(Lx=sc.Lx, Ly=sc.Ly, wind_x=sc.wind[0], wind_y=sc.wind[1], precision=precision,
                            scheme=scheme, F_timing=F_timing, **overrides)
    sim = Simulation(sc.nx, sc.ny, sc.p, sc.dt, prm)
    sim.set_state(sc.T0, sc.fuel0)
    if sc.wind_rank:
        sim.set_wind(sc.wind_rank, sc.wind_packed())
    return sim
