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
WF_EXPLICIT = 2
WF_FP32 = 0
WF_FP64 = 1
WF_F_ONCE = 0
WF_F_PER_SUBSTEP = 1
WF_STATUS_UNSTABLE = 1
WF_STATUS_TIMEOUT = 4


class wf_params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "Lx", "Ly", "rho", "cp", "kappa", "sigma", "eps", "ch", "hc", "cW", "chi", "T_amb", "T_ig",
        "delta_x", "delta_z", "A_r", "M_ratio", "T_a", "heat_scale", "fuel_rate", "fuel_thresh",
        "thresh_guard", "wind_x", "wind_y")] + [(n, ctypes.c_int) for n in (
        "scheme", "precision", "F_timing", "scale_heat_by_fuel")]


class wf_request(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("p", ctypes.c_int), ("steps", ctypes.c_int),
                ("dt", ctypes.c_double), ("params", wf_params), ("T0", ctypes.POINTER(ctypes.c_double)),
                ("fuel0", ctypes.POINTER(ctypes.c_double)), ("wind_rank", ctypes.c_int),
                ("wind_factors", ctypes.POINTER(ctypes.c_double)), ("T_out", ctypes.POINTER(ctypes.c_double)),
                ("fuel_out", ctypes.POINTER(ctypes.c_double))]


class wf_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("latency_s", ctypes.c_double), ("queue_s", ctypes.c_double),
                ("run_s", ctypes.c_double)]


class WFError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {wf_strerror(code)} ({code})")


_lib = None


class wf_mms(ctypes.Structure):
    _fields_ = [("nmodes", ctypes.c_int), ("amp", ctypes.c_double * 4), ("kx", ctypes.c_double * 4),
                ("ky", ctypes.c_double * 4), ("lambda_", ctypes.c_double * 4), ("base", ctypes.c_double),
                ("t0", ctypes.c_double)]


def lib() -> ctypes.CDLL:
    """Load libwf.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libwf.so is not built ({LIB_PATH}); run paper_2604_19370_gb300.build")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
        dp = ctypes.POINTER(ctypes.c_double)
        fp = ctypes.POINTER(ctypes.c_float)
        L.wf_params_default.argtypes = [ctypes.POINTER(wf_params)]
        L.wf_create.argtypes = [i, i, i, d, ctypes.POINTER(wf_params), ctypes.POINTER(vp)]
        L.wf_set_state.argtypes = [vp, dp, dp, sz]
        L.wf_set_state_f32.argtypes = [vp, fp, fp, sz]
        L.wf_set_wind.argtypes = [vp, i, dp]
        L.wf_step.argtypes = [vp, i]
        L.wf_sync.argtypes = [vp]
        L.wf_get_state.argtypes = [vp, dp, dp, sz]
        L.wf_get_state_f32.argtypes = [vp, fp, fp, sz]
        L.wf_batch_set_states.argtypes = [vp, dp, dp, sz]
        L.wf_batch_set_states_f32.argtypes = [vp, fp, fp, sz]
        L.wf_batch_get_states.argtypes = [vp, dp, dp, sz]
        L.wf_batch_get_states_f32.argtypes = [vp, fp, fp, sz]
        L.wf_batch_run.argtypes = [vp, dp, dp, dp, dp, sz, i, i]
        L.wf_batch_run_f32.argtypes = [vp, fp, fp, fp, fp, sz, i, i]
        L.wf_get_dims.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]
        L.wf_set_stream.argtypes = [vp, vp]
        L.wf_set_profiling.argtypes = [vp, i]
        L.wf_kernel_times.argtypes = [vp, dp, ctypes.POINTER(i), ctypes.c_void_p, i]
        L.wf_step_noalloc.argtypes = [vp, vp, vp, i, i]
        L.wf_autotune.argtypes = [vp, i]
        L.wf_launch_count.argtypes = [ctypes.POINTER(ctypes.c_ulonglong)]
        L.wf_set_mms.argtypes = [vp, ctypes.POINTER(wf_mms)]
        L.wf_set_mean_wind.argtypes = [vp, i, d, d]
        L.wf_get_time.argtypes = [vp, ctypes.POINTER(d)]
        L.wf_get_tuning.argtypes = [vp, ctypes.POINTER(i)]
        L.wf_set_tuning.argtypes = [vp, ctypes.POINTER(i)]
        L.wf_batch_create.argtypes = [i, i, i, d, ctypes.POINTER(wf_params), i, ctypes.POINTER(vp)]
        L.wf_batch_set_slot.argtypes = [vp, i, dp, dp, d, d, i, dp]
        L.wf_batch_get_slot.argtypes = [vp, i, dp, dp]
        L.wf_batch_activate.argtypes = [vp, i, i]
        L.wf_batch_set_budget.argtypes = [vp, i, i]
        L.wf_batch_status.argtypes = [vp, ctypes.POINTER(i), i]
        L.wf_batch_capacity.argtypes = [vp]
        L.wf_device_bytes.argtypes = [vp, ctypes.POINTER(sz)]
        L.wf_batch_bytes.argtypes = [i, i, i, d, ctypes.POINTER(wf_params), i, ctypes.POINTER(sz)]
        L.wf_set_wait_limit.argtypes = [vp, d]
        L.wf_measure_fma_peak.argtypes = [i, dp]
        L.wf_measure_host_link.argtypes = [vp, vp, sz, dp, dp, dp]
        L.wf_server_create.argtypes = [sz, i, ctypes.POINTER(vp)]
        L.wf_submit.argtypes = [vp, ctypes.POINTER(wf_request), ctypes.POINTER(ctypes.c_uint64)]
        L.wf_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(wf_result)]
        L.wf_server_stats.argtypes = [vp, dp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(sz)]
        L.wf_server_destroy.argtypes = [vp]
        L.wf_server_destroy.restype = None
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


def wf_set_state_f32(h, T, fuel) -> None:
    """wf_set_state with float32 host arrays (half the bytes over the host link)."""
    Nx, Ny, _, _ = wf_get_dims(h)
    n = Nx * Ny
    Ta = np.ascontiguousarray(T, dtype=np.float32).ravel()
    Fa = np.ascontiguousarray(fuel, dtype=np.float32).ravel()
    if Ta.size != n or Fa.size != n:
        raise ValueError(f"wf_set_state_f32: expected {n} values per field")
    fp = ctypes.POINTER(ctypes.c_float)
    _check(lib().wf_set_state_f32(h, Ta.ctypes.data_as(fp), Fa.ctypes.data_as(fp), n), "wf_set_state_f32")


def wf_set_state_f32_ptr(h, T_ptr: int, fuel_ptr: int, n: int) -> None:
    """Same call with raw float32 host addresses (e.g. pinned buffers owned by the caller)."""
    fp = ctypes.POINTER(ctypes.c_float)
    _check(lib().wf_set_state_f32(h, ctypes.cast(T_ptr, fp), ctypes.cast(fuel_ptr, fp), n), "wf_set_state_f32")


def wf_set_wind(h, rank: int, factors=None) -> None:
    arr = None if factors is None else np.ascontiguousarray(factors, dtype=np.float64).ravel()
    _check(lib().wf_set_wind(h, rank, _dptr(arr)), "wf_set_wind")


def wf_step(h, nsteps: int) -> None:
    _check(lib().wf_step(h, nsteps), "wf_step")


def wf_sync(h) -> int:
    """Returns the status code (WF_OK, WF_EUNSTABLE or WF_ETIMEOUT); raises on other errors."""
    code = lib().wf_sync(h)
    if code < 0 and code not in (WF_EUNSTABLE, WF_ETIMEOUT):
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


def wf_get_state_f32(h) -> Tuple[np.ndarray, np.ndarray]:
    Nx, Ny, _, _ = wf_get_dims(h)
    T = np.empty((Ny, Nx), dtype=np.float32)
    F = np.empty((Ny, Nx), dtype=np.float32)
    fp = ctypes.POINTER(ctypes.c_float)
    _check(lib().wf_get_state_f32(h, T.ctypes.data_as(fp), F.ctypes.data_as(fp), Nx * Ny), "wf_get_state_f32")
    return T, F


def wf_get_state_f32_ptr(h, T_ptr: int, fuel_ptr: int, n: int) -> None:
    fp = ctypes.POINTER(ctypes.c_float)
    _check(lib().wf_get_state_f32(h, ctypes.cast(T_ptr, fp), ctypes.cast(fuel_ptr, fp), n), "wf_get_state_f32")


def wf_batch_states_ptr(h, T_ptr: int, fuel_ptr: int, n: int, f32: bool, set_: bool) -> None:
    """Every slot's state in (set_) or out through raw host addresses ([S][Ny][Nx] per field)."""
    tp = ctypes.POINTER(ctypes.c_float if f32 else ctypes.c_double)
    name = ("wf_batch_set_states" if set_ else "wf_batch_get_states") + ("_f32" if f32 else "")
    fn = getattr(lib(), name)
    _check(fn(h, ctypes.cast(T_ptr, tp) if T_ptr else None, ctypes.cast(fuel_ptr, tp) if fuel_ptr else None, n),
           name)


def wf_batch_run_ptr(h, T_in: int, fuel_in: int, T_out: int, fuel_out: int, n: int, steps: int, groups: int,
                     f32: bool) -> None:
    """End-to-end run through raw host addresses: states in, `steps` steps, states out ([S][Ny][Nx])."""
    tp = ctypes.POINTER(ctypes.c_float if f32 else ctypes.c_double)
    name = "wf_batch_run_f32" if f32 else "wf_batch_run"
    _check(getattr(lib(), name)(h, ctypes.cast(T_in, tp), ctypes.cast(fuel_in, tp), ctypes.cast(T_out, tp),
                                ctypes.cast(fuel_out, tp), n, steps, groups), name)


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


def wf_set_mean_wind(h, wind_x: float, wind_y: float, slot: int = 0) -> None:
    _check(lib().wf_set_mean_wind(h, slot, wind_x, wind_y), "wf_set_mean_wind")


def wf_set_mms(h, modes=None, base: float = 300.0, t0: float = 0.0) -> None:
    """Manufactured-solution forcing: modes = [(amp, kx, ky, lambda), ...] (at most 4); None: off."""
    if modes is None:
        _check(lib().wf_set_mms(h, None), "wf_set_mms")
        return
    m = wf_mms()
    m.nmodes = len(modes)
    for k, (a, kx, ky, lam) in enumerate(modes):
        m.amp[k], m.kx[k], m.ky[k], m.lambda_[k] = a, kx, ky, lam
    m.base = base
    m.t0 = t0
    _check(lib().wf_set_mms(h, ctypes.byref(m)), "wf_set_mms")


def wf_get_time(h) -> float:
    t = ctypes.c_double()
    _check(lib().wf_get_time(h, ctypes.byref(t)), "wf_get_time")
    return t.value


def wf_launch_count() -> int:
    n = ctypes.c_ulonglong()
    _check(lib().wf_launch_count(ctypes.byref(n)), "wf_launch_count")
    return int(n.value)


def wf_autotune(h, reps: int = 3) -> Tuple[int, ...]:
    """Tune the launch shapes of a handle on its active slots.

    Returns the eight tuning values (see wf_get_tuning); 0 is the launchers' rule.
    """
    _check(lib().wf_autotune(h, reps), "wf_autotune")
    return wf_get_tuning(h)


#: names of the eight tuning values of wf_get_tuning / wf_set_tuning
TUNING_NAMES = ("x_lines_per_cta", "y_lines_per_cta", "quadrature_segment_rows", "x_lines_per_warp",
                "x2_lines_per_cta", "x2_rhs", "step_form", "persistent_group_slots")


def wf_get_tuning(h) -> Tuple[int, ...]:
    """(x lines per CTA, y lines per CTA, quadrature segment rows, x lines per warp, second-x-pass
    lines per CTA, second-x-pass right-hand side (1 fused, 2 separate matvec), step form (1 per-pass
    launches, 2 persistent), slots per group of the persistent order)."""
    out = (ctypes.c_int * 8)()
    _check(lib().wf_get_tuning(h, out), "wf_get_tuning")
    return tuple(int(v) for v in out)


def wf_set_tuning(h, shape) -> None:
    """Set the tuning values (six values leave the last two at 0, the rule)."""
    vals = [int(v) for v in shape]
    if len(vals) == 6:
        vals += [0, 0]
    if len(vals) != 8:
        raise ValueError("wf_set_tuning: six or eight values")
    arr = (ctypes.c_int * 8)(*vals)
    _check(lib().wf_set_tuning(h, arr), "wf_set_tuning")


def wf_step_noalloc(h, T_dev_ptr: int, fuel_dev_ptr: int, pitch: int, nsteps: int) -> int:
    """Allocation-free steps on caller-owned FP32 device arrays (returns the status code)."""
    return lib().wf_step_noalloc(h, ctypes.c_void_p(T_dev_ptr), ctypes.c_void_p(fuel_dev_ptr), pitch, nsteps)


def wf_batch_create(nx: int, ny: int, p: int, dt: float, params: wf_params, capacity: int) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().wf_batch_create(nx, ny, p, dt, ctypes.byref(params), capacity, ctypes.byref(h)), "wf_batch_create")
    return h


def wf_batch_set_slot(h, slot: int, T, fuel, wind_x: float, wind_y: float, wind_rank: int = 0, factors=None) -> None:
    Nx, Ny, _, _ = wf_get_dims(h)
    n = Nx * Ny
    Ta, Fa = _host(T, n), _host(fuel, n)
    fa = None if factors is None else np.ascontiguousarray(factors, dtype=np.float64).ravel()
    _check(lib().wf_batch_set_slot(h, slot, _dptr(Ta), _dptr(Fa), float(wind_x), float(wind_y), wind_rank, _dptr(fa)),
           "wf_batch_set_slot")


def wf_batch_get_slot(h, slot: int) -> Tuple[np.ndarray, np.ndarray]:
    Nx, Ny, _, _ = wf_get_dims(h)
    T = np.empty((Ny, Nx))
    F = np.empty((Ny, Nx))
    _check(lib().wf_batch_get_slot(h, slot, _dptr(T), _dptr(F)), "wf_batch_get_slot")
    return T, F


def wf_batch_activate(h, slot: int, on: bool) -> None:
    _check(lib().wf_batch_activate(h, slot, 1 if on else 0), "wf_batch_activate")


def wf_batch_set_budget(h, slot: int, steps: int) -> None:
    _check(lib().wf_batch_set_budget(h, slot, steps), "wf_batch_set_budget")


def wf_batch_status(h) -> np.ndarray:
    S = wf_batch_capacity(h)
    st = (ctypes.c_int * S)()
    _check(lib().wf_batch_status(h, st, S), "wf_batch_status")
    return np.array(st[:], dtype=np.int32)


def wf_batch_capacity(h) -> int:
    return _check(lib().wf_batch_capacity(h), "wf_batch_capacity")


def wf_device_bytes(h) -> int:
    b = ctypes.c_size_t()
    _check(lib().wf_device_bytes(h, ctypes.byref(b)), "wf_device_bytes")
    return b.value


def wf_batch_bytes(nx: int, ny: int, p: int, dt: float, params: wf_params, capacity: int) -> int:
    """Upper bound of the device bytes a batch handle with these arguments allocates (host-only)."""
    b = ctypes.c_size_t()
    _check(lib().wf_batch_bytes(nx, ny, p, dt, ctypes.byref(params), capacity, ctypes.byref(b)), "wf_batch_bytes")
    return b.value


def wf_measure_fma_peak(precision: int) -> float:
    """Measured FMA rate of this GPU in TFLOP/s (WF_FP32 or WF_FP64)."""
    t = ctypes.c_double()
    _check(lib().wf_measure_fma_peak(precision, ctypes.byref(t)), "wf_measure_fma_peak")
    return t.value


def wf_measure_host_link_ptr(host_in: int, host_out: int, nbytes: int):
    """Copy rates (GB/s) between pinned host arrays (raw addresses) and the GPU:
    (host to device, device to host, both directions at once)."""
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().wf_measure_host_link(ctypes.c_void_p(host_in), ctypes.c_void_p(host_out), nbytes, ctypes.byref(a),
                                      ctypes.byref(b), ctypes.byref(c)), "wf_measure_host_link")
    return a.value, b.value, c.value


def wf_set_wait_limit(h, seconds: float) -> None:
    _check(lib().wf_set_wait_limit(h, float(seconds)), "wf_set_wait_limit")


def wf_server_create(hbm_budget_bytes: int, max_slots: int) -> ctypes.c_void_p:
    s = ctypes.c_void_p()
    _check(lib().wf_server_create(hbm_budget_bytes, max_slots, ctypes.byref(s)), "wf_server_create")
    return s


def wf_server_destroy(s) -> None:
    if s:
        lib().wf_server_destroy(s)


def wf_server_stats(s):
    d = ctypes.c_double()
    c = ctypes.c_uint64()
    b = ctypes.c_size_t()
    _check(lib().wf_server_stats(s, ctypes.byref(d), ctypes.byref(c), ctypes.byref(b)), "wf_server_stats")
    return d.value, c.value, b.value


class Server:
    """Owning wrapper around wf_server: keeps every request's arrays alive until it is polled."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 16):
        self.s = wf_server_create(hbm_budget_bytes, max_slots)
        self.live = {}

    def submit(self, sc, steps=None, precision=WF_FP32, scheme=WF_PR, F_timing=WF_F_ONCE) -> int:
        """Queue scenario `sc` (a scenarios.Scenario); returns its ticket."""
        prm = wf_params_default(Lx=sc.Lx, Ly=sc.Ly, wind_x=sc.wind[0], wind_y=sc.wind[1], precision=precision,
                                scheme=scheme, F_timing=F_timing)
        T0 = np.ascontiguousarray(sc.T0, dtype=np.float64)
        f0 = np.ascontiguousarray(sc.fuel0, dtype=np.float64)
        wfac = sc.wind_packed()
        wfac = None if wfac is None else np.ascontiguousarray(wfac, dtype=np.float64)
        Tout = np.empty_like(T0)
        fout = np.empty_like(f0)
        r = wf_request(nx=sc.nx, ny=sc.ny, p=sc.p, steps=sc.steps if steps is None else steps, dt=sc.dt, params=prm,
                       T0=_dptr(T0), fuel0=_dptr(f0), wind_rank=sc.wind_rank, wind_factors=_dptr(wfac),
                       T_out=_dptr(Tout), fuel_out=_dptr(fout))
        t = ctypes.c_uint64()
        _check(lib().wf_submit(self.s, ctypes.byref(r), ctypes.byref(t)), "wf_submit")
        self.live[t.value] = (Tout, fout, T0, f0, wfac)
        return t.value

    def poll(self, ticket: int):
        """None while pending; else (status, wf_result, T, fuel)."""
        res = wf_result()
        code = lib().wf_poll(self.s, ticket, ctypes.byref(res))
        if code == WF_PENDING:
            return None
        if code == WF_ENOTFOUND:
            raise WFError(code, "wf_poll")
        Tout, fout = self.live.pop(ticket)[:2]
        return code, res, Tout, fout

    def stats(self):
        return wf_server_stats(self.s)

    def close(self):
        if self.s:
            wf_server_destroy(self.s)
            self.s = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


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


class Batch:
    """Owning wrapper around a batch handle (capacity scenario slots of one grid)."""

    def __init__(self, nx, ny, p, dt, params: wf_params, capacity: int):
        self.h = wf_batch_create(nx, ny, p, dt, params, capacity)
        self.Nx, self.Ny, self.p, self.precision = wf_get_dims(self.h)
        self.capacity = capacity

    def set_slot(self, slot, T, fuel, wind, wind_rank=0, factors=None):
        wf_batch_set_slot(self.h, slot, T, fuel, wind[0], wind[1], wind_rank, factors)

    def load_scenario(self, slot, sc, active=True):
        self.set_slot(slot, sc.T0, sc.fuel0, sc.wind, sc.wind_rank, sc.wind_packed())
        wf_batch_activate(self.h, slot, active)

    def activate(self, slot, on=True):
        wf_batch_activate(self.h, slot, on)

    def step(self, n=1):
        wf_step(self.h, n)

    def status(self):
        return wf_batch_status(self.h)

    def state(self, slot):
        return wf_batch_get_slot(self.h, slot)

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
