"""Seeded synthetic inputs for the shallow-water workloads.

This module is shared by the CPU oracle, the CUDA path, the tests and the
benchmark.  It only builds initial data (topography, initial water depth and
discharge, soil and scenario parameters); it contains none of the numerical
scheme's arithmetic.

All arrays are float64, shape [ny][nx] (x fastest), cell centres at
x_i = (i + 1/2) dx and y_j = (j + 1/2) dy.  Flow in the valley and hillslope
cases runs toward increasing j (the "north" edge, j = ny - 1, is the outflow).

Workloads follow the test cases the paper uses or points at:
  * dam_break  - the textbook dam-break Riemann problem on a flat strip
    (Stoker wet bed / Ritter dry bed), the SWASHES-style validation the paper
    cites in Sec. 4.1;
  * valley     - a synthetic stand-in for the Malpasset dam-break valley flood
    of Sec. 4.2 (the real DEM is not available): V-shaped valley + fractal
    noise, a level pool behind a dam line;
  * hillslope  - rainfall runoff with Green-Ampt infiltration (Sec. 3.5) on a
    ridge-and-furrow plane slope with lognormal K_s;
  * ensemble_specs - a seeded batch of valley scenarios of uneven sizes;
  * dem        - a float32 DEM for the D8 flow-direction stencil (Sec. 5.2's
    eight-neighbour example): a tilted fractal surface, optionally
    quantised so that many neighbours tie, with no-data holes.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Boundary codes, in W, E, S, N order (x-min, x-max, y-min, y-max).
BC_WALL = 0
BC_OUTFLOW = 1
BC_IMPOSED_H = 2
BC_IMPOSED_Q = 3
BC_IMPOSED_HQ = 4

RAIN_MM_PER_H = 1.0e-3 / 3600.0  # m/s per mm/h


@dataclass
class Workload:
    """Everything needed to set up one solver run (no scheme arithmetic)."""

    name: str
    nx: int
    ny: int
    dx: float
    dy: float
    z: np.ndarray
    h: np.ndarray
    qx: np.ndarray
    qy: np.ndarray
    bc: tuple = (BC_WALL, BC_WALL, BC_WALL, BC_WALL)
    friction: int = 0  # 0 none, 1 Manning
    manning_n: float = 0.0
    rain_rate: float = 0.0
    rain_t_on: float = 0.0
    rain_t_off: float = 0.0
    infiltration: int = 0
    ks: np.ndarray | None = None
    psi: float = 0.0
    dtheta: float = 0.0
    cfl: float = 0.5
    h_dry: float = 1.0e-6
    dt_max: float = 0.1
    t_end: float = 1.0e30
    steps: int = 0
    extra: dict = field(default_factory=dict)


def dam_break(n: int = 200, dx: float = 0.05, h_left: float = 1.0,
              h_right: float = 0.5, axis: str = "x") -> Workload:
    """Flat-bed dam break on an n x n grid, walls all round, no friction.

    h = h_left where the cell centre lies left of the mid-line (x < L/2),
    h_right elsewhere; the data is uniform along the other axis.  With
    axis="y" the same problem is laid out along y (transposed).
    """
    length = n * dx
    xc = (np.arange(n) + 0.5) * dx
    prof = np.where(xc < 0.5 * length, h_left, h_right).astype(np.float64)
    if axis == "x":
        h = np.tile(prof, (n, 1))
    else:
        h = np.tile(prof[:, None], (1, n))
    z = np.zeros((n, n))
    zero = np.zeros((n, n))
    return Workload(name=f"dam_break_{n}", nx=n, ny=n, dx=dx, dy=dx, z=z, h=h,
                    qx=zero.copy(), qy=zero.copy(), cfl=0.5, t_end=1.0,
                    dt_max=0.1, extra={"x0": 0.5 * length, "h_left": h_left,
                                       "h_right": h_right, "axis": axis})


def fractal_noise(nx: int, ny: int, hurst: float, seed: int,
                  peak: float) -> np.ndarray:
    """Spectral-synthesis fractal surface, power spectrum ~ k^-(2H+2).

    Complex white noise is shaped by k^-(H+1) in Fourier space (DC removed),
    transformed back and rescaled so that max |noise| == peak.
    """
    rng = np.random.default_rng(seed)
    kx = np.fft.rfftfreq(nx)
    ky = np.fft.fftfreq(ny)
    k = np.sqrt(kx[None, :] ** 2 + ky[:, None] ** 2)
    k[0, 0] = 1.0
    amp = k ** (-(hurst + 1.0))
    amp[0, 0] = 0.0
    spec = (rng.standard_normal(amp.shape) + 1j * rng.standard_normal(amp.shape)) * amp
    field_ = np.fft.irfft2(spec, s=(ny, nx))
    return field_ * (peak / np.max(np.abs(field_)))


def valley(n: int = 4096, dx: float = 2.0, seed: int = 1,
           reservoir: float = 40.0, dam_row: int | None = None,
           manning_n: float = 0.033, side_slope: float = 0.15,
           long_slope: float = 0.003, noise_peak: float = 1.5,
           hurst: float = 0.8, rain_mm_h: float = 0.0,
           steps: int = 2000, literal_pool: bool = False) -> Workload:
    """Synthetic dam-break valley flood (stand-in for the Malpasset case).

    z = side_slope |x - x_c| + long_slope (L_y - y) + fractal noise.
    A level pool fills rows j < dam_row up to the free surface
    eta = long_slope (L_y - y_{dam_row-1}) + reservoir (the noise-free
    thalweg elevation of the last reservoir row plus the reservoir depth);
    h = max(0, eta - z) there, dry (h = 0) downstream.  Outflow at the
    downstream edge (j = ny - 1), walls elsewhere.  literal_pool: the
    literal reading instead, h = reservoir in every cell upstream of the dam
    row (water stands on the valley walls).
    """
    if dam_row is None:
        dam_row = 512 if n == 4096 else max(1, n // 8)
    lx = n * dx
    ly = n * dx
    x = (np.arange(n) + 0.5) * dx
    y = (np.arange(n) + 0.5) * dx
    z = (side_slope * np.abs(x[None, :] - 0.5 * lx)
         + long_slope * (ly - y[:, None])
         + fractal_noise(n, n, hurst, seed, noise_peak))
    eta = long_slope * (ly - y[dam_row - 1]) + reservoir
    h = np.zeros((n, n))
    h[:dam_row, :] = reservoir if literal_pool else np.maximum(0.0, eta - z[:dam_row, :])
    zero = np.zeros((n, n))
    return Workload(name=f"valley_{n}", nx=n, ny=n, dx=dx, dy=dx, z=z, h=h,
                    qx=zero.copy(), qy=zero.copy(),
                    bc=(BC_WALL, BC_WALL, BC_WALL, BC_OUTFLOW),
                    friction=1, manning_n=manning_n,
                    rain_rate=rain_mm_h * RAIN_MM_PER_H, rain_t_on=0.0,
                    rain_t_off=1.0e30 if rain_mm_h > 0 else 0.0,
                    cfl=0.5, h_dry=1.0e-6, dt_max=0.1, steps=steps,
                    extra={"dam_row": dam_row, "reservoir": reservoir,
                           "seed": seed})


def hillslope(n: int = 2048, dx: float = 1.0, seed: int = 2, ks_seed: int = 3,
              slope: float = 0.05, furrow_amp: float = 0.1,
              furrow_period: float = 0.75, noise: float = 0.02,
              rain_mm_h: float = 50.0, rain_s: float = 600.0,
              t_end: float = 1200.0, ks_median: float = 1.0e-6,
              ks_sigma: float = 0.5, psi: float = 0.1, dtheta: float = 0.3,
              manning_n: float = 0.05) -> Workload:
    """Rainfall-runoff hillslope with Green-Ampt infiltration.

    z = slope (L_y - y) + furrow_amp sin(2 pi x / furrow_period) + noise N(0,1).
    The sinusoid is sampled at cell centres exactly as stated (at dx = 1 m a
    0.75 m period aliases to a 3 m one).  K_s = ks_median exp(ks_sigma xi),
    xi iid N(0, 1).  Initially dry; outflow at the downslope edge (j = ny-1).
    """
    rng = np.random.default_rng(seed)
    ly = n * dx
    x = (np.arange(n) + 0.5) * dx
    y = (np.arange(n) + 0.5) * dx
    z = (slope * (ly - y[:, None])
         + furrow_amp * np.sin(2.0 * np.pi * x[None, :] / furrow_period)
         + noise * rng.standard_normal((n, n)))
    ks = ks_median * np.exp(ks_sigma * np.random.default_rng(ks_seed).standard_normal((n, n)))
    zero = np.zeros((n, n))
    return Workload(name=f"hillslope_{n}", nx=n, ny=n, dx=dx, dy=dx, z=z,
                    h=zero.copy(), qx=zero.copy(), qy=zero.copy(),
                    bc=(BC_WALL, BC_WALL, BC_WALL, BC_OUTFLOW),
                    friction=1, manning_n=manning_n,
                    rain_rate=rain_mm_h * RAIN_MM_PER_H, rain_t_on=0.0,
                    rain_t_off=rain_s, infiltration=1, ks=ks, psi=psi,
                    dtheta=dtheta, cfl=0.5, h_dry=1.0e-6, dt_max=1.0,
                    t_end=t_end)


def lake_at_rest(n: int = 64, dx: float = 1.0, level: float = 1.0,
                 seed: int = 7, bump: float = 1.4) -> Workload:
    """Still water over uneven bed (including emerged dry bumps), walls."""
    rng = np.random.default_rng(seed)
    x = (np.arange(n) + 0.5) * dx
    X, Y = np.meshgrid(x, x)
    L = n * dx
    z = (0.4 * np.sin(2 * np.pi * X / L) * np.cos(2 * np.pi * Y / L)
         + bump * np.exp(-((X - 0.3 * L) ** 2 + (Y - 0.6 * L) ** 2) / (0.01 * L * L))
         + 0.05 * rng.standard_normal((n, n)))
    h = np.maximum(0.0, level - z)
    zero = np.zeros((n, n))
    return Workload(name=f"lake_{n}", nx=n, ny=n, dx=dx, dy=dx, z=z, h=h,
                    qx=zero.copy(), qy=zero.copy(), cfl=0.5, dt_max=0.1,
                    extra={"level": level})


def random_state(nx: int, ny: int, seed: int, dry_frac: float = 0.2,
                 zamp: float = 0.3, hmean: float = 1.0, vel: float = 0.5,
                 dx: float = 0.1, dy: float | None = None) -> Workload:
    """Rough random wet/dry state for stress and parity tests.

    Smooth-ish bed plus noise, depths with a fraction of exactly-dry cells,
    random velocities; walls W/S, outflow E/N so both boundary kinds run.
    """
    rng = np.random.default_rng(seed)
    dy = dx if dy is None else dy
    z = zamp * rng.standard_normal((ny, nx)).cumsum(axis=1) / np.sqrt(nx)
    z += 0.05 * rng.standard_normal((ny, nx))
    h = hmean * (0.2 + rng.random((ny, nx)))
    h[rng.random((ny, nx)) < dry_frac] = 0.0
    u = vel * rng.standard_normal((ny, nx))
    v = vel * rng.standard_normal((ny, nx))
    return Workload(name=f"random_{nx}x{ny}_{seed}", nx=nx, ny=ny, dx=dx,
                    dy=dy, z=z, h=h, qx=h * u, qy=h * v,
                    bc=(BC_WALL, BC_OUTFLOW, BC_WALL, BC_OUTFLOW),
                    friction=1, manning_n=0.03, cfl=0.5, dt_max=0.1)


@dataclass
class Scenario:
    side: int
    reservoir: float
    manning_n: float
    rain_mm_h: float
    seed: int


ENSEMBLE_SIDES = (128, 256, 384, 512, 768, 1024)


def ensemble_specs(count: int = 256, seed: int = 4) -> list[Scenario]:
    """Seeded batch of valley scenarios: side uniform over ENSEMBLE_SIDES,
    reservoir U(5, 40) m, Manning n U(0.02, 0.06), rain U(0, 80) mm/h."""
    rng = np.random.default_rng(seed)
    sides = rng.choice(np.array(ENSEMBLE_SIDES), size=count)
    res = rng.uniform(5.0, 40.0, size=count)
    nman = rng.uniform(0.02, 0.06, size=count)
    rain = rng.uniform(0.0, 80.0, size=count)
    return [Scenario(int(sides[k]), float(res[k]), float(nman[k]),
                     float(rain[k]), 1000 + k) for k in range(count)]


def ensemble_member(spec: Scenario, dx: float = 2.0) -> Workload:
    """One ensemble scenario: a valley of the given side (dam at row n/8),
    its reservoir depth, Manning n and uniform rain, no infiltration."""
    return valley(n=spec.side, dx=dx, seed=spec.seed, reservoir=spec.reservoir,
                  dam_row=max(1, spec.side // 8), manning_n=spec.manning_n,
                  rain_mm_h=spec.rain_mm_h, steps=1000)


def dem(nx: int, ny: int, seed: int, quantum: float = 0.0, nodata_frac: float = 0.0,
        nodata: float = -9999.0) -> np.ndarray:
    """float32 DEM [ny][nx]: 0.002 (x + 2y) tilt (cell units) + fractal
    noise (H = 0.8, peak 1.5); with quantum > 0 values are rounded to
    multiples of it (ties between neighbours), nodata_frac of the cells set
    to `nodata`."""
    rng = np.random.default_rng(seed + 1000)
    # grids beyond 4096 repeat a 4096-periodic noise field (the synthesis is
    # periodic, so the copies join without seams)
    fx, fy = min(nx, 4096), min(ny, 4096)
    noise = fractal_noise(fx, fy, 0.8, seed, 1.5).astype(np.float32)
    z = np.tile(noise, (-(-ny // fy), -(-nx // fx)))[:ny, :nx]
    z += (np.float32(0.002) * np.arange(nx, dtype=np.float32))[None, :]
    z += (np.float32(0.004) * np.arange(ny, dtype=np.float32))[:, None]
    if quantum > 0:
        z = (np.round(z / np.float32(quantum)) * np.float32(quantum)).astype(np.float32)
    z = np.ascontiguousarray(z, dtype=np.float32)
    if nodata_frac > 0:
        z[rng.random((ny, nx)) < nodata_frac] = np.float32(nodata)
    return z
