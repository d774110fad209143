"""Seeded synthetic inputs for the disordered spin chains of Eq. (1).

This module is shared by the CPU oracle (``oracle/``), the tests and the GPU
benchmark as a pure input source.  It holds none of the method's arithmetic:
it only draws random numbers and names the workloads.

Field generator: realization ``r`` of workload ``c`` draws a splitmix64 stream
seeded with ``0x9E3779B97F4A7C15 ^ (1000*c + r)``; ``h_i = W*(2u - 1)`` with
``u = (x >> 11) * 2**-53`` for ``i = 0..L-1``.  This is the uniform
``h_i in [-W, W]`` disorder of the benchmark models (Eq. (1) and the text
after it).  Site ``i`` of the code is site ``i+1`` of the paper and bit ``i``
of a basis state.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

_MASK64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15


def splitmix64_stream(seed: int, n: int) -> List[int]:
    """First ``n`` outputs of splitmix64 (Steele, Lea & Flood 2014) from ``seed``."""
    out = []
    s = seed & _MASK64
    for _ in range(n):
        s = (s + GOLDEN) & _MASK64
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        z = z ^ (z >> 31)
        out.append(z)
    return out


def uniform01(seed: int, n: int) -> np.ndarray:
    """``n`` doubles in [0, 1) with 53 random bits each."""
    return np.array([(x >> 11) * 2.0 ** -53 for x in splitmix64_stream(seed, n)], dtype=np.float64)


def fields(L: int, W: float, config: int, realization: int) -> np.ndarray:
    """Random fields ``h_i ~ U[-W, W]`` for one disorder realization (length L)."""
    seed = GOLDEN ^ (1000 * config + realization)
    u = uniform01(seed, L)
    return W * (2.0 * u - 1.0)


@dataclass
class Model:
    """Parameters of Eq. (1): chain length, couplings, anisotropy, fields, boundary."""
    L: int
    J1: float = 1.0
    J2: float = 0.0
    Delta: float = 1.0
    h: np.ndarray = field(default_factory=lambda: np.zeros(0))
    periodic: bool = True
    W: float = 0.0

    def __post_init__(self):
        self.h = np.asarray(self.h, dtype=np.float64)
        if self.h.size == 0:
            self.h = np.zeros(self.L)
        assert self.h.shape == (self.L,)


def xxz(L: int, W: float, config: int = 0, realization: int = 0, periodic: bool = True) -> Model:
    """XXZ point of Eq. (1): J1=1, J2=0, Delta=1."""
    return Model(L, 1.0, 0.0, 1.0, fields(L, W, config, realization), periodic, W)


def j1j2(L: int, W: float, config: int = 0, realization: int = 0, periodic: bool = True) -> Model:
    """J1-J2 point of Eq. (1): J1=J2=1, Delta=0.55."""
    return Model(L, 1.0, 1.0, 0.55, fields(L, W, config, realization), periodic, W)


def free_fermion(L: int, W: float, config: int = 0, realization: int = 0, periodic: bool = False) -> Model:
    """Delta=0, J2=0 (XX chain): maps to free fermions; used as an exact check at any L."""
    return Model(L, 1.0, 0.0, 0.0, fields(L, W, config, realization), periodic, W)


# Workloads shaped like the paper's runs (middle of the spectrum, eps = 0.5).
WORKLOADS = {
    # name: (builder, L, W, N_ev, n_b)
    "L14_xxz_W3": (xxz, 14, 3.0, 50, 16),
    "L20_j1j2_W4": (j1j2, 20, 4.0, 200, 32),
    "L22_xxz_W3": (xxz, 22, 3.0, 500, 64),
    "L24_j1j2_W5": (j1j2, 24, 5.0, 1000, 64),
}


def block(n_rows: int, n_cols: int, seed: int, dtype=np.float64) -> np.ndarray:
    """Seeded standard-normal block (row-major n_rows x n_cols) used as filter/apply input."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n_rows, n_cols)).astype(dtype)


def sample_rows(n_rows: int, k: int, seed: int) -> np.ndarray:
    """Seeded sorted sample of k distinct row indices (including the first and last row)."""
    rng = np.random.default_rng(seed)
    k = min(k, n_rows)
    picks = rng.choice(n_rows, size=k, replace=False)
    picks[0] = 0
    if k > 1:
        picks[1] = n_rows - 1
    return np.unique(picks)
