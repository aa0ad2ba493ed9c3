"""Seeded synthetic workloads (shapes and distributions of the paper's tests).

This module only draws parameters with numpy's PCG64 generator; it contains none
of the method's arithmetic and is shared, as plain arrays, by the oracle-based
tests and by the device path.  Parameter layout per integral: 2*d doubles,
c_1..c_d then w_1..w_d (for the oscillatory family w_1 is the phase u).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Integral:
    family: str
    d: int
    a: int
    n_last: int
    params: np.ndarray  # 2*d float64

    @property
    def c(self):
        return self.params[: self.d]

    @property
    def w(self):
        return self.params[self.d:]


def small_exp(d: int = 4, N: int = 16) -> Integral:
    """f(x) = exp(sum_j x_j / j) on N points per transformed axis (n = N^d)."""
    params = np.concatenate([1.0 / np.arange(1, d + 1), np.zeros(d)])
    return Integral("exp", d, N, N, params)


SMALL_SLR_A = 12345  # Korobov parameter of the plain lattice rule on the small workload


@dataclass
class Batch:
    families: list
    d: np.ndarray
    a: np.ndarray
    n_last: np.ndarray
    offsets: np.ndarray
    pool: np.ndarray

    def __len__(self):
        return len(self.families)

    def integral(self, i: int) -> Integral:
        d = int(self.d[i])
        o = int(self.offsets[i])
        return Integral(self.families[i], d, int(self.a[i]), int(self.n_last[i]), self.pool[o:o + 2 * d])


def batch(count: int = 4096, seed: int = 0, d_range=(6, 20), n_range=(8, 32),
          families=("peak", "gauss")) -> Batch:
    """Many integrals of uneven size: d ~ U{6..20}, N ~ U{8..32} points per
    transformed axis (a = n_last = N); the family alternates product-peak /
    Gaussian; c_j ~ U(0.5, 2), w_j ~ U(0, 1)."""
    rng = np.random.default_rng(seed)
    d = rng.integers(d_range[0], d_range[1] + 1, size=count)
    N = rng.integers(n_range[0], n_range[1] + 1, size=count)
    fams = [families[i % len(families)] for i in range(count)]
    offsets = np.zeros(count, dtype=np.int64)
    offsets[1:] = np.cumsum(2 * d[:-1])
    pool = np.empty(int(2 * d.sum()))
    for i in range(count):
        o, di = offsets[i], int(d[i])
        pool[o:o + di] = rng.uniform(0.5, 2.0, di)
        pool[o + di:o + 2 * di] = rng.uniform(0.0, 1.0, di)
    return Batch(fams, d.astype(np.int32), N.astype(np.int32), N.astype(np.int32), offsets, pool)


def oscillatory(d: int = 50, N: int = 32, seed: int = 0) -> Integral:
    """f(x) = cos(2 pi u + sum_j a_j x_j), u ~ U(0,1), a_j ~ U(0,1)/j."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(0.0, 1.0)
    aj = rng.uniform(0.0, 1.0, d) / np.arange(1, d + 1)
    w = np.zeros(d)
    w[0] = u
    return Integral("osc", d, N, N, np.concatenate([aj, w]))


def gaussian(d: int = 100, N: int = 16, seed: int = 0) -> Integral:
    """f(x) = exp(-sum_j c_j^2 (x_j - w_j)^2), c_j ~ U(0.2, 1.5), w_j ~ U(0, 1)."""
    rng = np.random.default_rng(seed)
    return Integral("gauss", d, N, N, np.concatenate([rng.uniform(0.2, 1.5, d), rng.uniform(0.0, 1.0, d)]))


def scale_exp(d: int = 1000, N: int = 16) -> Integral:
    """f(x) = exp(sum_j x_j / j^2)."""
    return Integral("exp", d, N, N, np.concatenate([1.0 / np.arange(1, d + 1) ** 2, np.zeros(d)]))


def random_product(family: str, d: int, seed: int, c_range=(0.5, 2.0)) -> np.ndarray:
    """2*d parameters for one product-form integral (test cases)."""
    rng = np.random.default_rng(seed)
    return np.concatenate([rng.uniform(c_range[0], c_range[1], d), rng.uniform(0.0, 1.0, d)])
