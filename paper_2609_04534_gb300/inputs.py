"""Seeded synthetic inputs shared by the CUDA path's callers and the oracle's tests.

Holds none of the method's arithmetic: only a counter-based generator (splitmix64) and
the recipe that turns its draws into vectors.  Draw m of seed s is

    z = splitmix64_mix(s + (m + 1) * 0x9E3779B97F4A7C15),   u = (z >> 11) * 2^-53,
    value = 2 u - 1                                          (uniform on [-1, 1))

and draw m is assigned to unique global node m (lexicographic, x fastest), so a vector
generated this way and copied to the cells is consistent by construction.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Raw 64-bit outputs for draws start .. start+count-1 of the counter-based stream."""
    with np.errstate(over="ignore"):
        m = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed) + m * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_pm1(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Uniform values on [-1, 1) in float64 (53-bit resolution)."""
    z = splitmix64(seed, count, start)
    u = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return 2.0 * u - 1.0


def unique_count(nx: int, ny: int, nz: int, degree: int) -> int:
    return (nx * degree + 1) * (ny * degree + 1) * (nz * degree + 1)


def random_unique(nx: int, ny: int, nz: int, degree: int, seed: int) -> np.ndarray:
    """x uniform[-1,1] on the unique DoFs of the Q_k mesh (consistent once scattered)."""
    return uniform_pm1(seed, unique_count(nx, ny, nz, degree))
