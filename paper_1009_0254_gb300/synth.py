"""Seeded synthetic inputs shared by the tests and the benchmark.

Holds no arithmetic of the method: only random draws of given shapes and scales,
and the parameter draws of the ensemble workloads."""
from __future__ import annotations

import numpy as np


def gaussian_field(shape, seed: int, scale: float = 1.0) -> np.ndarray:
    """i.i.d. N(0, scale^2) array (FP64) from numpy's PCG64 with the given seed."""
    return scale * np.random.default_rng(seed).standard_normal(shape)


def uniform(lo: float, hi: float, count: int, seed: int) -> np.ndarray:
    """count i.i.d. draws from U[lo, hi) (FP64)."""
    return np.random.default_rng(seed).uniform(lo, hi, count)


def sample_nodes(nx: int, ny: int, count: int, seed: int) -> np.ndarray:
    """count distinct node numbers y*nx + x, always including the four corners and the
    edge midpoints (where periodic wrap is exercised)."""
    rng = np.random.default_rng(seed)
    fixed = [0, nx - 1, (ny - 1) * nx, ny * nx - 1, nx // 2, (ny // 2) * nx, (ny // 2) * nx + nx - 1,
             (ny - 1) * nx + nx // 2, (ny // 2) * nx + nx // 2]
    extra = rng.choice(nx * ny, size=count, replace=False)
    return np.unique(np.concatenate([np.array(fixed, dtype=np.int64), extra.astype(np.int64)]))


def clipped_gaussian_field(shape, seed: int, scale: float, clip: float) -> np.ndarray:
    """N(0, 1) draws (PCG64, given seed) clipped to [-clip, clip], times scale (FP64)."""
    return scale * np.clip(np.random.default_rng(seed).standard_normal(shape), -clip, clip)
