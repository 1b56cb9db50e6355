"""Seeded synthetic workloads shared by the tests, the benchmark and the smoke check.

Only random draws and parameter sets live here; none of the method's arithmetic.  The
shapes and distributions stand in for the paper's SUSY / NUS-WIDE samples (Sec. 6).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class SchemeParams:
    log_n: int
    q_bits: tuple
    p_bits: tuple
    dnum: int
    scale: float

    @property
    def n(self) -> int:
        return 1 << self.log_n

    @property
    def slots(self) -> int:
        return self.n // 2

    @property
    def top(self) -> int:
        return len(self.q_bits) - 1


# ring N = 4096, chain [40, 20 | 40], scale 2^20 (one multiply level)
PARAMS_SMALL = SchemeParams(12, (40, 20), (40,), 2, 2.0**20)
# ring N = 8192, chain [60, 40, 40 | 60], scale 2^40, digits of one prime
PARAMS_N8192 = SchemeParams(13, (60, 40, 40), (60,), 3, 2.0**40)
# ring N = 16384, chain [60, 40 x 6 | 60, 60, 60], scale 2^40, dnum 3 (digits of three primes)
PARAMS_N16384 = SchemeParams(14, (60, 40, 40, 40, 40, 40, 40), (60, 60, 60), 3, 2.0**40)


def gradient_small(seed: int = 0):
    """X 64x16 ~ N(0,1), residual r 64 ~ U[-1,1]: the LR gradient X^T [[r]] (m=16, n=64)."""
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(64, 16))
    r = rng.uniform(-1.0, 1.0, 64)
    return X, r


def gradient_and_forward_n8192(seed: int = 0):
    """X 1024x256 ~ N(0,1); r 1024 ~ U[-1,1] (gradient X^T [[r]]); w 256 ~ N(0, var 0.1) (forward X [[w]])."""
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(1024, 256))
    r = rng.uniform(-1.0, 1.0, 1024)
    w = rng.normal(scale=np.sqrt(0.1), size=256)
    return X, r, w


def vfl_nn_layer(seed: int = 0):
    """VFL neural layer: activations A 4096x256 ~ U[-1,1] (encrypted as diagonals), weights
    W 256x128 ~ N(0, var 1/256) (forward A W); output gradient D^T 4096x128 ~ N(0, var 1/4096)
    (backward A^T D^T)."""
    rng = np.random.default_rng(seed)
    A = rng.uniform(-1.0, 1.0, (4096, 256))
    W = rng.normal(scale=1.0 / 16.0, size=(256, 128))
    Dt = rng.normal(scale=1.0 / 64.0, size=(4096, 128))
    return A, W, Dt


def batched_instances(count: int = 64, seed: int = 0):
    """Per-instance (batch b ~ U{128..4096}, features f ~ U{16..512}); X b x f ~ N(0,1), r ~ U[-1,1],
    gradient X^T [[r]] with m = f, n = b.  Data seed 1000 + i."""
    rng = np.random.default_rng(seed)
    shapes = [(int(rng.integers(128, 4097)), int(rng.integers(16, 513))) for _ in range(count)]
    out = []
    for i, (b, f) in enumerate(shapes):
        r2 = np.random.default_rng(1000 + i)
        X = r2.normal(size=(b, f))
        r = r2.uniform(-1.0, 1.0, b)
        out.append((X, r))
    return out


def random_matrix(m: int, n: int, seed: int):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(m, n)), rng.uniform(-1.0, 1.0, n)
