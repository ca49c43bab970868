"""Seeded scenario generators for the wildfire time step.

Every random number comes from SplitMix64 (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014): the stream for a
seed s is z_k = mix(s + (k+1)*0x9E3779B97F4A7C15), k = 0, 1, ...  with the
published mix function, and a uniform double is (z >> 11) * 2^-53.

Scenario recipe (shapes follow the paper's setting, Sec. 5 and Sec. 6):

* domain: a square of side L = h*n with the fixed element size h = 100/64 m,
  so the 64x64 case is exactly the paper's [0,100]^2 m domain (Sec. 5);
* temperature: T0 = 300 + 700 * max_k exp(-|x - x_k|^2 / (2 sigma^2)),
  sigma = 3 m, ignition points x_k uniform in [0.2, 0.8] L (the paper's
  Gaussian-smoothed ignition mask, Sec. 2.1 "Ignition initialization");
* fuel: uniform noise on the coefficient grid, separable Gaussian blur with
  reflecting boundary, min-max normalised to [0, 1] (a synthetic stand-in for
  the NDVI-derived fuel availability of Sec. 2.1; the satellite maps are not
  available);
* wind: a constant mean (b_x, b_y) plus an optional separable perturbation
  b'_c(x, y) = sum_r f_{c,r}(x) g_{c,r}(y) whose factors are 1-D spline
  coefficient vectors obtained by sampling seeded 4-mode cosine series at the
  Greville abscissae; the amplitude is 10 % of |b| in total.

Coefficients of a spline are set by sampling the target function at the
Greville abscissae (Schoenberg's variation-diminishing approximation), which
keeps a field that lies in [a, b] inside [a, b] pointwise.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

#: element size of every configuration (m): the paper's 100 m square on 64 elements
H_ELEMENT = 100.0 / 64.0


def element_size() -> float:
    return H_ELEMENT


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Return `count` SplitMix64 outputs of stream `seed`, starting at index `offset`."""
    k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the SplitMix64 stream `seed`."""
    z = splitmix64(seed, count, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


class _Stream:
    """Sequential reader over one SplitMix64 stream."""

    def __init__(self, seed: int):
        self.seed = seed
        self.pos = 0

    def uniform(self, count: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = uniform01(self.seed, count, self.pos)
        self.pos += count
        return lo + (hi - lo) * u


def greville(n: int, p: int, L: float) -> np.ndarray:
    """Greville abscissae of the open uniform knot vector with n elements of degree p on [0, L]."""
    h = L / n
    t = np.concatenate([np.zeros(p), np.arange(n + 1) * h, np.full(p, L)])
    t[p + n] = L
    if p == 0:
        return 0.5 * (t[:-1] + t[1:])
    return np.array([t[i + 1:i + p + 1].mean() for i in range(n + p)])


def gaussian_blur(a: np.ndarray, sigma: float) -> np.ndarray:
    """Separable Gaussian blur (kernel truncated at 4 sigma) with reflecting boundaries."""
    if sigma <= 0:
        return a.copy()
    r = int(math.ceil(4.0 * sigma))
    d = np.arange(-r, r + 1, dtype=np.float64)
    k = np.exp(-0.5 * (d / sigma) ** 2)
    k /= k.sum()
    out = a.astype(np.float64)
    for axis in (0, 1):
        pad = [(0, 0), (0, 0)]
        pad[axis] = (r, r)
        ap = np.pad(out, pad, mode="symmetric")
        acc = np.zeros_like(out)
        for j, w in enumerate(k):
            sl = [slice(None), slice(None)]
            sl[axis] = slice(j, j + out.shape[axis])
            acc += w * ap[tuple(sl)]
        out = acc
    return out


@dataclasses.dataclass
class Scenario:
    """One fire scenario: grid, time step and initial coefficient fields.

    Arrays are row-major [Ny][Nx] with Nx = nx + p (x index fastest).
    `wind_factors` is None or an array of shape (4, rank, N) laid out as
    [fx (rank, Nx), gx (rank, Ny), fy (rank, Nx), gy (rank, Ny)] packed into
    `wind_packed()`.
    """

    name: str
    nx: int
    ny: int
    p: int
    Lx: float
    Ly: float
    dt: float
    steps: int
    wind: tuple
    T0: np.ndarray
    fuel0: np.ndarray
    wind_rank: int = 0
    fx: Optional[np.ndarray] = None
    gx: Optional[np.ndarray] = None
    fy: Optional[np.ndarray] = None
    gy: Optional[np.ndarray] = None
    seed: int = 0

    @property
    def Nx(self) -> int:
        return self.nx + self.p

    @property
    def Ny(self) -> int:
        return self.ny + self.p

    @property
    def dofs(self) -> int:
        return self.Nx * self.Ny

    def wind_packed(self) -> Optional[np.ndarray]:
        """Factors packed as [fx(rank*Nx), gx(rank*Ny), fy(rank*Nx), gy(rank*Ny)], or None."""
        if self.wind_rank == 0:
            return None
        return np.concatenate([self.fx.ravel(), self.gx.ravel(), self.fy.ravel(), self.gy.ravel()])


def _cosine_series(stream: _Stream, x: np.ndarray, L: float, modes: int = 4) -> np.ndarray:
    a = stream.uniform(modes, -1.0, 1.0)
    ph = stream.uniform(modes, 0.0, 2.0 * math.pi)
    v = np.zeros_like(x)
    for m in range(modes):
        v += a[m] * np.cos((m + 1) * math.pi * x / L + ph[m])
    return v / max(np.abs(a).sum(), 1e-300)


def make_scenario(
    name: str,
    n: int,
    p: int,
    dt: float,
    steps: int,
    seed: int,
    *,
    ignitions: int = 1,
    sigma_ign: float = 3.0,
    fuel_sigma: float = 4.0,
    fuel_classes: bool = False,
    wind: Optional[tuple] = None,
    wind_speed_range: Optional[tuple] = None,
    wind_perturbation: float = 0.1,
    wind_rank: int = 2,
    uniform_fuel: Optional[float] = None,
    centred_ignition: bool = False,
    shared_fuel: Optional[np.ndarray] = None,
) -> Scenario:
    """Build one seeded scenario on an n x n element grid of element size 100/64 m."""
    L = H_ELEMENT * n
    N = n + p
    s = _Stream(seed)
    xg = greville(n, p, L)
    # ignition points
    if centred_ignition:
        pts = [(0.5 * L, 0.5 * L)]
    else:
        u = s.uniform(2 * ignitions, 0.2 * L, 0.8 * L)
        pts = [(u[2 * k], u[2 * k + 1]) for k in range(ignitions)]
    X, Y = np.meshgrid(xg, xg)  # [j][i]: Y varies along rows
    bump = np.zeros_like(X)
    for (cx, cy) in pts:
        bump = np.maximum(bump, np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2.0 * sigma_ign ** 2)))
    T0 = 300.0 + 700.0 * bump
    # fuel
    if shared_fuel is not None:
        fuel0 = shared_fuel.copy()
    elif uniform_fuel is not None:
        fuel0 = np.full((N, N), float(uniform_fuel))
    else:
        fseed = _Stream(seed * 7919 + 17)
        noise = fseed.uniform(N * N).reshape(N, N)
        b = gaussian_blur(noise, fuel_sigma)
        lo, hi = b.min(), b.max()
        fuel0 = (b - lo) / (hi - lo) if hi > lo else np.full_like(b, 0.5)
        if fuel_classes:
            med = np.median(fuel0)
            fuel0 = np.where(fuel0 > med, 1.0, 0.2)
            # 5 % unburnable gaps on 8x8-element blocks
            nb = (N + 7) // 8
            gaps = fseed.uniform(nb * nb).reshape(nb, nb) < 0.05
            g = np.kron(gaps, np.ones((8, 8), dtype=bool))[:N, :N]
            fuel0 = np.where(g, 0.0, fuel0)
    # wind
    if wind is None:
        if wind_speed_range is not None:
            sp = s.uniform(1, wind_speed_range[0], wind_speed_range[1])[0]
            th = s.uniform(1, 0.0, 2.0 * math.pi)[0]
            wind = (sp * math.cos(th), sp * math.sin(th))
        else:
            wind = (0.0, 0.0)
    speed = math.hypot(*wind)
    rank = wind_rank if (wind_perturbation > 0 and speed > 0 and wind_rank > 0) else 0
    fx = gx = fy = gy = None
    if rank:
        amp = wind_perturbation * speed / rank
        ws = _Stream(seed * 104729 + 3)
        fx = np.stack([amp * _cosine_series(ws, xg, L) for _ in range(rank)])
        gx = np.stack([_cosine_series(ws, xg, L) for _ in range(rank)])
        fy = np.stack([amp * _cosine_series(ws, xg, L) for _ in range(rank)])
        gy = np.stack([_cosine_series(ws, xg, L) for _ in range(rank)])
    return Scenario(name, n, n, p, L, L, dt, steps, tuple(float(w) for w in wind), T0, fuel0,
                    rank, fx, gx, fy, gy, seed)


def config_c1(seed: int = 1001) -> Scenario:
    """64x64 elements, p=2, dt=1e-3, 100 steps, wind (1, 0.5) + 10 % perturbation."""
    return make_scenario("c1_64x64_p2", 64, 2, 1e-3, 100, seed, fuel_sigma=4.0, wind=(1.0, 0.5))


def config_c2(seed: int = 2001, p: int = 2) -> Scenario:
    """1024x1024 elements, p=2, dt=1e-3, 1000 steps, wind speed U[0,3] with random direction."""
    return make_scenario("c2_1024x1024_p2", 1024, p, 1e-3, 1000, seed, fuel_sigma=20.0,
                         wind_speed_range=(0.0, 3.0))


def config_c3(seed: int = 3001) -> Scenario:
    """4096x4096 elements, p=3, 500 steps, two fuel classes with 5 % gaps, three ignitions."""
    return make_scenario("c3_4096x4096_p3", 4096, 3, 1e-3, 500, seed, ignitions=3, fuel_sigma=20.0,
                         fuel_classes=True, wind_speed_range=(0.0, 3.0))


def config_c4(scenario: int, shared_fuel: Optional[np.ndarray] = None, n: int = 256) -> Scenario:
    """One member of the 256-scenario ensemble: 256x256 elements, p=2, 2000 steps, constant wind."""
    seed = 4000 + scenario
    if shared_fuel is None:
        shared_fuel = make_scenario("fuel", n, 2, 1e-3, 1, 4000, fuel_sigma=20.0,
                                    wind=(0.0, 0.0)).fuel0
    return make_scenario(f"c4_{scenario}", n, 2, 1e-3, 2000, seed, fuel_sigma=20.0,
                         wind_speed_range=(0.0, 3.0), wind_perturbation=0.0,
                         shared_fuel=shared_fuel)


def request_stream_c5(count: int, rate_hz: float, seed: int = 5) -> List[dict]:
    """Poisson request stream: n in {128,256,512,1024}, p in {2,3}, steps U[200,2000], 20 % FP64."""
    s = _Stream(seed)
    out = []
    t = 0.0
    for k in range(count):
        u = s.uniform(5)
        t += -math.log(max(1.0 - u[0], 1e-300)) / rate_hz
        n = (128, 256, 512, 1024)[min(int(u[1] * 4), 3)]
        p = 2 if u[2] < 0.5 else 3
        steps = 200 + min(int(u[3] * 1801), 1800)
        fp64 = bool(u[4] < 0.2)
        out.append(dict(arrival_s=t, n=n, p=p, steps=steps, fp64=fp64, seed=5000 + k))
    return out
