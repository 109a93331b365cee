"""Seeded synthetic inputs for the Cahn-Hilliard integrators.

This module is the only code that both the CUDA library's tests/bench and the CPU
oracle consume: it draws initial states and batch descriptors and holds none of the
method's arithmetic.  The generator is SplitMix64 (S. Vigna, public domain, the
published 64-bit mixing function), mapped to 53-bit doubles in [0, 1).

Initial data follow the workloads' recipe: i.i.d. uniform values on [lo, hi), then
the FP64 (numpy pairwise) mean is subtracted and a target mean added.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int) -> np.ndarray:
    """First `count` outputs of SplitMix64 started from state `seed` (uint64 array)."""
    with np.errstate(over="ignore"):
        k = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(seed) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, count: int) -> np.ndarray:
    """53-bit uniform doubles in [0, 1)."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def initial_state(n, seed: int, lo: float = -0.05, hi: float = 0.05, mean: float = 0.0) -> np.ndarray:
    """Flat FP64 grid vector (x fastest) of i.i.d. U[lo, hi) values, shifted to `mean`."""
    N = int(np.prod(n))
    y = lo + (hi - lo) * uniform01(seed, N)
    y = y - y.mean()
    if mean != 0.0:
        y = y + mean
    return np.ascontiguousarray(y, dtype=np.float64)


BATCH_SIDES = (64, 96, 128, 192, 256, 384, 512)


def batch_descriptors(count: int, seed: int, sides=BATCH_SIDES, eps_lo=0.01, eps_hi=0.05):
    """Side lengths drawn uniformly from `sides` and eps uniform on [eps_lo, eps_hi),
    one pair per instance, from the batch seed."""
    u = uniform01(seed, 2 * count).reshape(count, 2)
    side_idx = np.minimum((u[:, 0] * len(sides)).astype(np.int64), len(sides) - 1)
    n = np.asarray(sides, dtype=np.int64)[side_idx]
    eps = eps_lo + (eps_hi - eps_lo) * u[:, 1]
    return n, eps


# Workloads of the benchmark configurations (sizes, eps, initial-data recipe, run).
WORKLOADS = {
    "c0_2d64_const": dict(dim=2, n=64, eps=0.05, lo=-0.05, hi=0.05, mean=0.0,
                          T=1e-4, tau0=1e-6, adaptive=False, mmax=30, tol_phi=1e-8, steps=100),
    "c1_2d1024_adaptive": dict(dim=2, n=1024, eps=0.01, lo=-0.05, hi=0.05, mean=0.0,
                               T=1e-3, tau0=1e-7, adaptive=True, tol=1e-6, mmax=30),
    "c2_3d256_adaptive": dict(dim=3, n=256, eps=0.02, lo=-0.1, hi=0.1, mean=0.1,
                              T=5e-4, tau0=1e-7, adaptive=True, tol=1e-5, mmax=30),
    "c3_batch256": dict(dim=2, count=256, lo=-0.05, hi=0.05, mean=0.0, T=1e-4, tau0=1e-7,
                        adaptive=True, tol=1e-6, mmax=30),
    "c4_3d512_adaptive": dict(dim=3, n=512, eps=0.01, lo=-0.05, hi=0.05, mean=0.0,
                              T=1e-4, tau0=1e-7, adaptive=True, tol=1e-6, mmax=30),
}
