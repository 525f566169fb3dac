"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module only draws random numbers (numpy ``default_rng``, identical
streams on x86 and Arm); it contains none of the transform's arithmetic.  The
paper has no dataset: every workload is Gaussian noise of the shapes below.

Workloads (the shapes the MrDFT is exercised on):
  * ``single_1k``:   one complex64 signal, N = 2^10, seed 0.
  * ``single_16m``:  one complex64 signal, N = 2^24, seed 1.
  * ``batch_256x64k``: 256 complex64 signals of N = 2^16, seed 2.
  * ``ragged_1024``: 1024 real FP32 signals, lengths 2^k with k uniform on
    8..18 (seed 3 for the lengths, then the samples from the same stream).
  * ``grad_64x256k``: 64 complex64 signals of N = 2^18 (seed 4) and
    complex64 targets T^(i) for every level (seed 5).
"""
from __future__ import annotations

import numpy as np


def complex_signals(batch: int, n: int, seed: int) -> np.ndarray:
    """[batch, n] complex64, real and imaginary parts i.i.d. N(0, 1)."""
    rng = np.random.default_rng(seed)
    f = rng.standard_normal((batch, n, 2), dtype=np.float32)
    return f.view(np.complex64).reshape(batch, n)


def real_signals(batch: int, n: int, seed: int) -> np.ndarray:
    """[batch, n] float32 i.i.d. N(0, 1)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((batch, n), dtype=np.float32)


def ragged_lengths(count: int, kmin: int, kmax: int, seed: int) -> np.ndarray:
    """``count`` power-of-two lengths 2^k, k uniform on [kmin, kmax]."""
    rng = np.random.default_rng(seed)
    k = rng.integers(kmin, kmax + 1, size=count)
    return (np.int64(1) << k.astype(np.int64))


def ragged_real(count: int = 1024, kmin: int = 8, kmax: int = 18, seed: int = 3):
    """Ragged batch: (lengths int64[count], concatenated float32 samples)."""
    rng = np.random.default_rng(seed)
    k = rng.integers(kmin, kmax + 1, size=count)
    lengths = (np.int64(1) << k.astype(np.int64))
    samples = rng.standard_normal(int(lengths.sum()), dtype=np.float32)
    return lengths, samples


def targets(batch: int, n: int, seed: int) -> np.ndarray:
    """Per-level complex64 targets [batch, m, n] with m = log2(n)."""
    m = int(n).bit_length() - 1
    rng = np.random.default_rng(seed)
    f = rng.standard_normal((batch, m, n, 2), dtype=np.float32)
    return f.view(np.complex64).reshape(batch, m, n)


WORKLOADS = {
    "single_1k": dict(kind="complex", batch=1, n=1 << 10, seed=0),
    "single_16m": dict(kind="complex", batch=1, n=1 << 24, seed=1),
    "batch_256x64k": dict(kind="complex", batch=256, n=1 << 16, seed=2),
    "ragged_1024": dict(kind="ragged_real", count=1024, kmin=8, kmax=18, seed=3),
    "grad_64x256k": dict(kind="complex", batch=64, n=1 << 18, seed=4, target_seed=5),
}
