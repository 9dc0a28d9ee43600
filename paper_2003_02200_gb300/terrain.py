"""Seeded synthetic inputs: spectral-fractal DEMs and the workload recipes.

This module only draws inputs.  It holds none of the viewshed arithmetic and
imports nothing from the library or the oracle, so both sides (and the
benchmark) can take their inputs from it.

The paper measures on real 10 m DEMs of the Montes de Malaga park (2000^2,
4000^2 and 8000^2 cells, observers 1.5 m above ground; section 5.1, Table 2).
Those rasters are not available, so seeded fractal terrain of the same shapes,
grid step and observer height stands in for them:

* seeded complex Gaussian noise on the rfft2 grid, amplitude |f|^-(hurst+1)
  (power |f|^-(2 hurst + 2)), DC removed, inverse FFT, min-max rescaled to
  [0, relief] metres, float32;
* optional spikes: a seeded fraction of cells, drawn without replacement,
  raised by U(20, 60) m.
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 2003022000


def fractal_dem(rows: int, cols: int, hurst: float, relief: float, seed: int,
                spike_frac: float = 0.0, spike_m: tuple[float, float] = (20.0, 60.0)) -> np.ndarray:
    """Spectral fractal DEM (rows x cols, float32, metres)."""
    rng = np.random.default_rng(seed)
    fy = np.fft.fftfreq(rows)[:, None]
    fx = np.fft.rfftfreq(cols)[None, :]
    f = np.sqrt(fx * fx + fy * fy)
    f[0, 0] = 1.0
    amp = f ** (-(hurst + 1.0))
    amp[0, 0] = 0.0
    shape = (rows, cols // 2 + 1)
    noise = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    field = np.fft.irfft2(noise * amp, s=(rows, cols))
    lo, hi = field.min(), field.max()
    dem = (field - lo) / (hi - lo if hi > lo else 1.0) * relief
    if spike_frac > 0.0:
        count = int(round(spike_frac * rows * cols))
        cells = rng.choice(rows * cols, size=count, replace=False)
        dem.reshape(-1)[cells] += rng.uniform(spike_m[0], spike_m[1], size=count)
    return np.ascontiguousarray(dem, dtype=np.float32)


# The single-DEM workloads: (rows, cols, hurst, relief m, step m, observer m,
# directions, max range m (0 = unlimited), spike fraction, seed offset).
WORKLOADS = {
    "tvs100": dict(rows=100, cols=100, hurst=0.8, relief=500.0, step=10.0, h0=1.5, n=180,
                   max_range=0.0, spike_frac=0.0, seed=SEED_BASE + 0),
    "tvs2000": dict(rows=2000, cols=2000, hurst=0.8, relief=1500.0, step=10.0, h0=1.5, n=180,
                    max_range=0.0, spike_frac=0.0, seed=SEED_BASE + 1),
    "tvs4000": dict(rows=4000, cols=4000, hurst=0.7, relief=2500.0, step=5.0, h0=10.0, n=360,
                    max_range=10000.0, spike_frac=0.05, seed=SEED_BASE + 2),
    # profiling size: the 2000^2 recipe at a quarter of the cells (a few GB of scratch)
    "tvs1000": dict(rows=1000, cols=1000, hurst=0.8, relief=1500.0, step=10.0, h0=1.5, n=180,
                    max_range=0.0, spike_frac=0.0, seed=SEED_BASE + 5),
    # profiling size with the 2000^2 rows: the tvs2000 DEM with 24 of its directions' spacing
    # (the same row lengths and kernels, under 1 GB of scratch)
    "tvs2000n24": dict(rows=2000, cols=2000, hurst=0.8, relief=1500.0, step=10.0, h0=1.5, n=24,
                       max_range=0.0, spike_frac=0.0, seed=SEED_BASE + 1),
}


def workload_dem(name: str) -> np.ndarray:
    w = WORKLOADS[name]
    return fractal_dem(w["rows"], w["cols"], w["hurst"], w["relief"], w["seed"], w["spike_frac"])


def batch_tiles(count: int = 64, seed: int = SEED_BASE + 3, side_lo: int = 256, side_hi: int = 1500,
                n: int = 180) -> list[dict]:
    """Uneven tiles: side log-uniform in [side_lo, side_hi], hurst U(0.6, 0.9),
    step from {5, 10, 30} m, observer U(1.5, 30) m, relief U(200, 2000) m."""
    rng = np.random.default_rng(seed)
    tiles = []
    for q in range(count):
        side = int(round(math.exp(rng.uniform(math.log(side_lo), math.log(side_hi)))))
        tiles.append(dict(rows=side, cols=side, hurst=float(rng.uniform(0.6, 0.9)),
                          relief=float(rng.uniform(200.0, 2000.0)),
                          step=float(rng.choice([5.0, 10.0, 30.0])), h0=float(rng.uniform(1.5, 30.0)),
                          n=n, max_range=0.0, seed=seed * 1000 + q))
    return tiles


def tile_dem(tile: dict) -> np.ndarray:
    return fractal_dem(tile["rows"], tile["cols"], tile["hurst"], tile["relief"], tile["seed"])


def request_stream(count: int, rate_hz: float = 20.0, seed: int = SEED_BASE + 4, side_lo: int = 128,
                   side_hi: int = 2048) -> list[dict]:
    """Poisson arrivals (mean rate_hz) of total-viewshed requests: side
    log-uniform in [side_lo, side_hi], directions from {90, 180, 360}, observer
    U(1.5, 30) m, max range from {unlimited, 5 km}, step from {5, 10, 30} m."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    for q in range(count):
        t += float(rng.exponential(1.0 / rate_hz))
        side = int(round(math.exp(rng.uniform(math.log(side_lo), math.log(side_hi)))))
        reqs.append(dict(arrival=t, rows=side, cols=side, hurst=float(rng.uniform(0.6, 0.9)),
                         relief=float(rng.uniform(200.0, 2000.0)),
                         step=float(rng.choice([5.0, 10.0, 30.0])), h0=float(rng.uniform(1.5, 30.0)),
                         n=int(rng.choice([90, 180, 360])),
                         max_range=float(rng.choice([0.0, 5000.0])), seed=seed * 1000 + q))
    return reqs
