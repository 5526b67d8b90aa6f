"""Seeded synthetic inputs shared by the oracle tests, the CUDA tests and the
benchmark.

This module holds workload shapes and plaintext matrix generators only: no
step of the encrypted computation lives here, and it imports neither the
oracle nor the CUDA package.

The paper evaluates square matrices whose entries are drawn from N(0, 1)
with a fraction s of them set to zero (Sec. 4.1); under an exact integer
scheme the entries are small integers instead.  Zeros are placed by an
independent Bernoulli(s) draw per element, and nonzero entries exclude 0, so
the realised zero pattern is exactly the drawn one.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

T_PLAIN = 65537
SIGMA = 3.2


@dataclass(frozen=True)
class Ring:
    N: int           # ring degree
    L: int           # number of 54-bit ciphertext primes


@dataclass(frozen=True)
class MatmulShape:
    M: int
    K: int
    Nc: int
    sparsity: float
    lo: int
    hi: int
    seed: int


def sparse_int_matrix(rows: int, cols: int, sparsity: float, lo: int, hi: int, seed: int) -> np.ndarray:
    """Bernoulli(sparsity) zeros; other entries uniform in [lo, hi] without 0."""
    rng = np.random.default_rng(seed)
    zero = rng.random((rows, cols)) < sparsity
    nz_vals = np.array([v for v in range(lo, hi + 1) if v != 0], dtype=np.int64)
    vals = nz_vals[rng.integers(0, len(nz_vals), size=(rows, cols))]
    vals[zero] = 0
    return vals


def dense_int_matrix(rows: int, cols: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Entries uniform in [lo, hi], zero included."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=(rows, cols), dtype=np.int64)


def sparsify(M: np.ndarray, sparsity: float, seed: int) -> np.ndarray:
    """A copy of M with an independent Bernoulli(sparsity) draw of elements set to zero."""
    rng = np.random.default_rng(seed)
    out = np.array(M, dtype=np.int64, copy=True)
    out[rng.random(out.shape) < sparsity] = 0
    return out


def operands(shape: MatmulShape, b_sparse: bool = False) -> tuple[np.ndarray, np.ndarray]:
    """A with the shape's sparsity; B dense (uniform with 0), or with
    b_sparse both operands at the shape's sparsity (the paper draws both
    operands of its sweeps with the same fraction of zeros, Sec. 4.1)."""
    A = sparse_int_matrix(shape.M, shape.K, shape.sparsity, shape.lo, shape.hi, shape.seed)
    if b_sparse:
        B = sparse_int_matrix(shape.K, shape.Nc, shape.sparsity, shape.lo, shape.hi, shape.seed + 1_000_003)
    else:
        B = dense_int_matrix(shape.K, shape.Nc, shape.lo, shape.hi, shape.seed + 1_000_003)
    return A, B


# --- the five workloads ----------------------------------------------------

# tiny: 8x8 times 8x8, 50% zeros, seed 0; N=4096 with two primes
TINY_RING = Ring(4096, 2)
TINY = MatmulShape(8, 8, 8, 0.5, -16, 16, 0)

# sparsity sweep: 64x64 times 64x64; N=8192 with four primes
SWEEP_RING = Ring(8192, 4)
SWEEP_SPARSITIES = (0.0, 0.1, 0.3, 0.5, 0.7, 0.9, 0.99)


def sweep(sparsity: float, seed: int = 1) -> MatmulShape:
    return MatmulShape(64, 64, 64, sparsity, -16, 16, seed)


# DNN-layer shape: encrypted weights 128x256 times activations 256x16, [-8, 8]
LAYER_RING = Ring(8192, 4)
LAYER_SPARSITIES = (0.5, 0.7, 0.9)


def layer(sparsity: float, seed: int = 2) -> MatmulShape:
    return MatmulShape(128, 256, 16, sparsity, -8, 8, seed)


# mixed workload: 64 independent matmuls, M, K, Nc from {16..256},
# sparsity uniform in [0.30, 0.95]; N=16384 with eight primes
MIXED_RING = Ring(16384, 8)
MIXED_DIMS = (16, 32, 64, 128, 256)


def mixed(count: int = 64, seed: int = 3) -> list[MatmulShape]:
    rng = np.random.default_rng(seed)
    out = []
    for r in range(count):
        M, K, Nc = (int(x) for x in rng.choice(MIXED_DIMS, size=3))
        s = float(rng.uniform(0.30, 0.95))
        out.append(MatmulShape(M, K, Nc, s, -8, 8, seed * 1000 + r))
    return out


def poisson_arrivals(rate_per_s: float, count: int, seed: int = 4) -> np.ndarray:
    """Arrival times (s) of a Poisson process with the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))
