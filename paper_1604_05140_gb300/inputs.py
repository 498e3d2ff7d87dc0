"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

Holds no arithmetic of the transform: only random draws and the index
bookkeeping needed to lay them out (coefficient count and the degree n of each
coefficient slot).  The shapes follow the paper's experiment (Sect. 4: random
SGL coefficients for a bandlimit B) with the distributions of the workloads
this library is benchmarked on.
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 1604051400


def n_coeffs(B: int) -> int:
    """Number of coefficients for bandlimit B (n^2 slots for each n <= B)."""
    return sum(n * n for n in range(1, B + 1))


def degree_of_slot(B: int) -> np.ndarray:
    """n of every coefficient slot, slots grouped by n with n^2 slots each."""
    return np.concatenate([np.full(n * n, n, dtype=np.float64) for n in range(1, B + 1)])


def random_coeffs(B: int, batch: int = 1, seed: int = BASE_SEED, decay: bool = False,
                  dist: str = "normal") -> np.ndarray:
    """Complex coefficients, shape (batch, n_coeffs(B)), complex128.

    dist="normal": real and imaginary parts i.i.d. N(0, 1).
    dist="uniform": real and imaginary parts i.i.d. U[-1, 1] (Sect. 4).
    decay=True divides every slot of degree n by n.
    """
    rng = np.random.default_rng(seed)
    shape = (batch, n_coeffs(B))
    if dist == "normal":
        c = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    elif dist == "uniform":
        c = rng.uniform(-1, 1, shape) + 1j * rng.uniform(-1, 1, shape)
    else:
        raise ValueError(dist)
    if decay:
        c = c / degree_of_slot(B)[None, :]
    return c


def random_samples(B: int, batch: int = 1, seed: int = BASE_SEED, scale: float = 1.0) -> np.ndarray:
    """Complex normal noise on the grid, shape (batch, B, 2B, 2B), complex128."""
    rng = np.random.default_rng(seed)
    shape = (batch, B, 2 * B, 2 * B)
    return scale * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))


def random_real(shape, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(shape)


def uneven_bandlimits(nfn: int = 256, seed: int = BASE_SEED + 4, lo: int = 16, hi: int = 128,
                      step: int = 8) -> np.ndarray:
    """Bandlimits drawn uniformly from {lo, lo+step, ..., hi}."""
    rng = np.random.default_rng(seed)
    choices = np.arange(lo, hi + 1, step)
    return rng.choice(choices, size=nfn).astype(np.int32)
