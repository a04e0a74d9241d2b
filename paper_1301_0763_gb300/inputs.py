"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds no arithmetic of the transform: it only draws random numbers.
Values are drawn in float64 with numpy's PCG64 and then cast to the storage
dtype; the *cast* values are what both the GPU path and the CPU oracle read.

The paper measures on random signals only (Sec. 6.3: random complex signals with
real and imaginary parts uniform in (-0.5, 0.5)); the workloads below follow the
shapes and distributions of the benchmark configurations:

* uniform complex in [-1, 1] (single-size N=1024 case, FP16/BF16 case),
* standard-normal complex / real (batched 2^28-element cases, ragged batch),
* Student-t with 3 degrees of freedom, each row scaled to max |re|,|im| = 1
  (heavy-tailed FP16/BF16 case),
* spectral-filter weights, re and im ~ N(0, 0.02^2).
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 13010763


def rng(seed_offset: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(BASE_SEED + int(seed_offset)))


def uniform_complex(rows: int, n: int, seed: int = 0, lo: float = -1.0, hi: float = 1.0,
                    dtype=np.complex64) -> np.ndarray:
    g = rng(seed)
    re = g.uniform(lo, hi, size=(rows, n))
    im = g.uniform(lo, hi, size=(rows, n))
    return (re + 1j * im).astype(dtype)


def normal_complex(rows: int, n: int, seed: int = 1, dtype=np.complex64) -> np.ndarray:
    g = rng(seed)
    re = g.standard_normal(size=(rows, n))
    im = g.standard_normal(size=(rows, n))
    return (re + 1j * im).astype(dtype)


def normal_real(rows: int, n: int, seed: int = 1, dtype=np.float32) -> np.ndarray:
    return rng(seed).standard_normal(size=(rows, n)).astype(dtype)


def q15_complex(rows: int, n: int, seed: int = 5) -> np.ndarray:
    """Complex Q15 samples for the fixed-point variant: int16 [rows, n, 2]
    (re, im), each round(32767 u) with u ~ U[-1, 1] drawn in float64."""
    u = rng(seed).uniform(-1.0, 1.0, size=(rows, n, 2))
    return np.round(u * 32767.0).astype(np.int16)


def student_t_complex(rows: int, n: int, seed: int = 3, dof: float = 3.0) -> np.ndarray:
    """Student-t(3) re and im, each row scaled so that max(|re|, |im|) = 1 (float64)."""
    g = rng(seed)
    re = g.standard_t(dof, size=(rows, n))
    im = g.standard_t(dof, size=(rows, n))
    m = np.maximum(np.abs(re).max(axis=1), np.abs(im).max(axis=1))[:, None]
    return (re / m) + 1j * (im / m)


def ragged_log2n(count: int = 4096, seed: int = 2, lo: int = 4, hi: int = 20) -> np.ndarray:
    """log2 N_i drawn uniformly from lo..hi (inclusive)."""
    return rng(seed).integers(lo, hi + 1, size=count).astype(np.int32)


def ragged_offsets(log2n: np.ndarray) -> np.ndarray:
    """Exclusive prefix sum of the row lengths (count+1 entries, int64)."""
    n = np.left_shift(np.int64(1), log2n.astype(np.int64))
    off = np.zeros(len(log2n) + 1, dtype=np.int64)
    np.cumsum(n, out=off[1:])
    return off


def ragged_values(total: int, seed: int = 2, dtype=np.complex64) -> np.ndarray:
    g = rng(seed + 1000)
    re = g.standard_normal(size=total)
    im = g.standard_normal(size=total)
    return (re + 1j * im).astype(dtype)


def filter_weights(channels: int, n: int, seed: int = 4, std: float = 0.02) -> np.ndarray:
    """Complex spectral-filter weights [channels, n/2+1], re and im ~ N(0, std^2)."""
    g = rng(seed)
    h = n // 2 + 1
    return (std * g.standard_normal(size=(channels, h))
            + 1j * std * g.standard_normal(size=(channels, h))).astype(np.complex64)
