"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random numbers: initial seed positions, per-step integer
displacements, populations of independent simulations and request arrival
times.  It holds none of the method's arithmetic (no distances, no clamping, no
schedules), and both the CUDA path and the CPU oracle consume what it returns.

The paper's experiments (Section VI) place seeds uniformly at random on an n x n
pixel grid and move every seed each step by a uniformly random integer amount
(Section IV and Section V-A); there is no dataset.  The named workloads below
restate those experiments at fixed sizes:

* ``single256``   256 x 256 grid, 64 seeds, 10 steps, moves in [-1, 1]
* ``single2048``  2048 x 2048 grid, 16384 seeds, 100 steps, moves in [-2, 2]
* ``sweep8192``   8192 x 8192 grid, seeds in {2^10, 2^14, 2^18, 2^22},
                  maximum move in {1, 4, 16}, 50 steps
* ``batched256``  256 independent simulations, sides in {256, 512, 1024, 2048},
                  seeds per simulation uniform in [64, side^2 / 64], moves in [-2, 2]
* ``serve1000``   1000 resident simulations, sides in {512, 1024, 2048, 4096},
                  the same density, Poisson request arrivals at 2k-20k per second
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def _rng(seed: int, salt: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([int(seed) & 0xFFFFFFFF, int(salt) & 0xFFFFFFFF]))


def uniform_seeds(w: int, h: int, s: int, seed: int = 0) -> np.ndarray:
    """s seed positions, x uniform in [0, w), y uniform in [0, h); shape (s, 2) int32.

    Positions may coincide (the paper's uniform model does not exclude it)."""
    g = _rng(seed, 1)
    xy = np.empty((s, 2), np.int32)
    xy[:, 0] = g.integers(0, w, size=s, dtype=np.int32)
    xy[:, 1] = g.integers(0, h, size=s, dtype=np.int32)
    return xy


def displacements(s: int, max_disp: int, steps: int, seed: int = 0) -> np.ndarray:
    """Per-step integer moves uniform in [-max_disp, max_disp] per axis; shape (steps, s, 2)."""
    g = _rng(seed, 2)
    return g.integers(-max_disp, max_disp + 1, size=(steps, s, 2), dtype=np.int32)


def step_displacements(s: int, max_disp: int, step: int, seed: int = 0) -> np.ndarray:
    """The moves of one step alone (independent stream per step); shape (s, 2)."""
    g = _rng(seed, 1000 + int(step))
    return g.integers(-max_disp, max_disp + 1, size=(s, 2), dtype=np.int32)


@dataclass(frozen=True)
class SimShape:
    w: int
    h: int
    s: int


def batched_population(n_sims: int, sides=(256, 512, 1024, 2048), seed: int = 0,
                       min_seeds: int = 64, density_div: int = 64) -> list[SimShape]:
    """Independent square simulations: side uniform over ``sides``, seed count
    uniform in [min_seeds, side^2 / density_div]."""
    g = _rng(seed, 3)
    out = []
    for _ in range(n_sims):
        side = int(g.choice(np.asarray(sides)))
        hi = max(min_seeds, side * side // density_div)
        out.append(SimShape(side, side, int(g.integers(min_seeds, hi + 1))))
    return out


def poisson_arrivals(rate_per_s: float, n: int, seed: int = 0) -> np.ndarray:
    """n arrival times (seconds from 0) of a Poisson stream with the given rate."""
    g = _rng(seed, 4)
    return np.cumsum(g.exponential(1.0 / rate_per_s, size=n))


def request_targets(n_requests: int, n_sims: int, seed: int = 0) -> np.ndarray:
    """Which simulation each request steps, uniform over the resident simulations."""
    g = _rng(seed, 5)
    return g.integers(0, n_sims, size=n_requests, dtype=np.int64)


# Named single-simulation workloads: (w, h, seeds, steps, max displacement).
SINGLE = {
    "single256": (256, 256, 64, 10, 1),
    "single2048": (2048, 2048, 16384, 100, 2),
}
SWEEP8192 = {
    "side": 8192,
    "seeds": (1 << 10, 1 << 14, 1 << 18, 1 << 22),
    "max_disp": (1, 4, 16),
    "steps": 50,
}
