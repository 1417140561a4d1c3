"""Seeded synthetic light curves shaped like the paper's workloads.

This module serves both the oracle and the CUDA path (tests, smoke, bench).
It holds none of the periodogram's arithmetic: it only draws observation
times, signals and noise from numpy's counter-based Philox generator with a
fixed seed per workload, so every caller sees the same arrays.

Workloads (times in days, frequencies in cycles/day, grids half-open):

* ``single_small``   -- one object, N_t=1000 times uniform on [60000, 63650]
  (sorted), y = 0.5 sin(2 pi f0 t + phi) + N(0, 0.1^2), f0 ~ U[0.2, 5],
  phi ~ U[0, 2 pi); grid [0.1, 10) with N_f = 100000.
* ``ragged_survey``  -- N_o objects with N_t ~ U{50..500}; times uniform in
  the observable half of each of 10 years from 60000 (a 6-month seasonal gap
  per year), sorted; y = 0.5 sin(2 pi f0 t + phi) + N(0, sigma^2),
  sigma ~ U[0.02, 0.3], period log-uniform in [2 h, 100 h] (f0 = 24/P_h);
  grid [0.24, 12) with N_f = 100000.  (The paper's ZTF-like asteroid
  population of Section 4.2 is not available; this stands in for it.)
* ``single_large``   -- one object, N_t=100000 times uniform over 10 years,
  y = sin(2 pi f1 t + phi1) + 0.3 sin(2 pi f2 t + phi2) + N(0, 0.2^2),
  f1, f2 ~ U[0.1, 20]; grid [0.05, 25) with N_f = 1000000.
* ``ragged_lognormal`` -- as ``ragged_survey`` but N_o = 100000 and
  N_t = round(exp(U[ln 10, ln 2000])); grid [0.24, 12) with N_f = 50000.
* ``learned_train`` / ``learned_infer`` -- ``ragged_survey``-shaped sets for
  the learned proposal stage (disjoint seeds).

The sinusoid amplitude of the survey-shaped sets is 0.5 (as in the single
object set), since none is given for them.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

T_START = 60000.0
YEAR = 365.25
N_YEARS = 10
SEASON = YEAR / 2.0


@dataclasses.dataclass
class Grid:
    f_min: float
    f_max: float
    n_f: int

    @property
    def df(self) -> float:
        return (self.f_max - self.f_min) / float(self.n_f)


@dataclasses.dataclass
class Batch:
    """CSR batch: object o owns t[offsets[o]:offsets[o+1]]."""
    t: np.ndarray          # float64 [total_nt]
    y: np.ndarray          # float64 [total_nt]
    offsets: np.ndarray    # int64   [n_obj + 1]
    grid: Grid
    f_true: np.ndarray     # float64 [n_obj] injected (dominant) frequency
    sigma: np.ndarray      # float64 [n_obj] noise level

    @property
    def n_obj(self) -> int:
        return self.offsets.size - 1

    @property
    def n_t(self) -> np.ndarray:
        return np.diff(self.offsets)

    @property
    def pairs(self) -> int:
        return int(self.offsets[-1]) * int(self.grid.n_f)

    def subset(self, objs) -> "Batch":
        """A new batch holding only the listed objects (in the given order)."""
        objs = np.asarray(objs, dtype=np.int64)
        lens = self.n_t[objs]
        off = np.zeros(objs.size + 1, dtype=np.int64)
        np.cumsum(lens, out=off[1:])
        idx = np.concatenate([np.arange(self.offsets[o], self.offsets[o + 1]) for o in objs]) \
            if objs.size else np.zeros(0, dtype=np.int64)
        return Batch(self.t[idx], self.y[idx], off, self.grid, self.f_true[objs], self.sigma[objs])


SEEDS = {
    "single_small": 0xC1,
    "ragged_survey": 0xC2,
    "single_large": 0xC3,
    "learned_train": 0xC4000,
    "learned_infer": 0xC4001,
    "ragged_lognormal": 0xC5,
}

GRIDS = {
    "single_small": Grid(0.1, 10.0, 100_000),
    "ragged_survey": Grid(0.24, 12.0, 100_000),
    "single_large": Grid(0.05, 25.0, 1_000_000),
    "learned_train": Grid(0.24, 12.0, 100_000),
    "learned_infer": Grid(0.24, 12.0, 100_000),
    "ragged_lognormal": Grid(0.24, 12.0, 50_000),
}


def rng(seed: int, stream: int = 0) -> np.random.Generator:
    """Philox generator keyed by (seed, stream)."""
    return np.random.Generator(np.random.Philox(key=[seed & 0xFFFFFFFFFFFFFFFF, stream]))


def _single(n_t, grid, seed, t_lo, t_hi, comps, noise):
    g = rng(seed)
    t = np.sort(g.uniform(t_lo, t_hi, n_t))
    y = np.zeros(n_t)
    fs = []
    for amp, f_lo, f_hi in comps:
        f0 = g.uniform(f_lo, f_hi)
        phi = g.uniform(0.0, 2.0 * math.pi)
        y += amp * np.sin(2.0 * math.pi * f0 * t + phi)
        fs.append(f0)
    y += g.normal(0.0, noise, n_t)
    off = np.array([0, n_t], dtype=np.int64)
    return Batch(t, y, off, grid, np.array([fs[0]]), np.array([noise]))


def single_small(seed: int = SEEDS["single_small"], n_t: int = 1000, grid: Grid | None = None) -> Batch:
    return _single(n_t, grid or GRIDS["single_small"], seed, 60000.0, 63650.0,
                   [(0.5, 0.2, 5.0)], 0.1)


def single_large(seed: int = SEEDS["single_large"], n_t: int = 100_000, grid: Grid | None = None) -> Batch:
    return _single(n_t, grid or GRIDS["single_large"], seed, T_START, T_START + N_YEARS * YEAR,
                   [(1.0, 0.1, 20.0), (0.3, 0.1, 20.0)], 0.2)


def _survey_times(g, n_t_per_obj):
    """Seasonal cadence: uniform in the first half of each year, sorted per object."""
    total = int(n_t_per_obj.sum())
    obj = np.repeat(np.arange(n_t_per_obj.size, dtype=np.int64), n_t_per_obj)
    year = g.integers(0, N_YEARS, total)
    t = T_START + year * YEAR + g.uniform(0.0, SEASON, total)
    order = np.lexsort((t, obj))
    return t[order]


def survey_batch(n_obj: int, n_t_per_obj: np.ndarray, grid: Grid, seed: int,
                 amp: float = 0.5, p_hours=(2.0, 100.0), sigma=(0.02, 0.3)) -> Batch:
    g = rng(seed, 1)
    n_t_per_obj = np.asarray(n_t_per_obj, dtype=np.int64)
    off = np.zeros(n_obj + 1, dtype=np.int64)
    np.cumsum(n_t_per_obj, out=off[1:])
    t = _survey_times(g, n_t_per_obj)
    p_h = np.exp(g.uniform(math.log(p_hours[0]), math.log(p_hours[1]), n_obj))
    f0 = 24.0 / p_h
    phi = g.uniform(0.0, 2.0 * math.pi, n_obj)
    sig = g.uniform(sigma[0], sigma[1], n_obj)
    obj = np.repeat(np.arange(n_obj), n_t_per_obj)
    y = amp * np.sin(2.0 * math.pi * f0[obj] * t + phi[obj]) + g.normal(0.0, 1.0, t.size) * sig[obj]
    return Batch(t, y, off, grid, f0, sig)


def ragged_survey(n_obj: int = 10_000, seed: int = SEEDS["ragged_survey"], grid: Grid | None = None,
                  nt_range=(50, 500)) -> Batch:
    g = rng(seed, 0)
    n_t = g.integers(nt_range[0], nt_range[1] + 1, n_obj)
    return survey_batch(n_obj, n_t, grid or GRIDS["ragged_survey"], seed)


def ragged_lognormal(n_obj: int = 100_000, seed: int = SEEDS["ragged_lognormal"],
                     grid: Grid | None = None, nt_range=(10, 2000)) -> Batch:
    g = rng(seed, 0)
    n_t = np.rint(np.exp(g.uniform(math.log(nt_range[0]), math.log(nt_range[1]), n_obj))).astype(np.int64)
    return survey_batch(n_obj, n_t, grid or GRIDS["ragged_lognormal"], seed)


def learned_set(n_obj: int, which: str = "learned_train", part: int = 0, grid: Grid | None = None) -> Batch:
    """Survey-shaped curves for the learned stage; ``part`` selects a disjoint chunk."""
    seed = SEEDS[which] + 7919 * part
    return ragged_survey(n_obj, seed=seed, grid=grid or GRIDS[which])


def by_name(name: str, **kw) -> Batch:
    return {
        "single_small": single_small,
        "single_large": single_large,
        "ragged_survey": ragged_survey,
        "ragged_lognormal": ragged_lognormal,
    }[name](**kw)
