"""Seeded synthetic inputs shared by the tests, the bench and the CPU baseline.

This module holds none of the transform's or the checksum scheme's arithmetic:
it only draws random numbers.  Every generator takes an explicit seed and
uses numpy's PCG64 ``default_rng``, so the CUDA path and the oracle see the
same bits.

Recipes (the paper's own workloads are synthetic: normally distributed test
signals for the fault-coverage study of Section V-C, and 2^28-element batches
for the throughput comparison of Section V-B):

* ``uniform_batch``  -- real and imaginary parts i.i.d. uniform on [-1, 1).
* ``normal_batch``   -- real and imaginary parts i.i.d. standard normal.
* ``tones_batch``    -- each signal is a sum of 8 complex exponentials with
  bins uniform on [0, N), amplitudes log-uniform on [1e-3, 1], phases uniform
  on [0, 2 pi), plus complex Gaussian noise of standard deviation 1e-4 per
  real/imaginary component.
* ``ragged_lengths`` -- log2 lengths uniform on {lo..hi} for a ragged batch.
"""
from __future__ import annotations

import numpy as np


def uniform_batch(n: int, batch: int, seed: int, dtype=np.complex64) -> np.ndarray:
    rng = np.random.default_rng(seed)
    real_dt = np.float32 if np.dtype(dtype) == np.complex64 else np.float64
    out = np.empty((batch, n), dtype=dtype)
    out.real = rng.uniform(-1.0, 1.0, size=(batch, n)).astype(real_dt)
    out.imag = rng.uniform(-1.0, 1.0, size=(batch, n)).astype(real_dt)
    return out


def normal_batch(n: int, batch: int, seed: int, dtype=np.complex128) -> np.ndarray:
    rng = np.random.default_rng(seed)
    real_dt = np.float32 if np.dtype(dtype) == np.complex64 else np.float64
    out = np.empty((batch, n), dtype=dtype)
    out.real = rng.standard_normal(size=(batch, n)).astype(real_dt)
    out.imag = rng.standard_normal(size=(batch, n)).astype(real_dt)
    return out


def tones_batch(n: int, batch: int, seed: int, ntones: int = 8, noise_std: float = 1e-4,
                dtype=np.complex64) -> np.ndarray:
    rng = np.random.default_rng(seed)
    bins = rng.integers(0, n, size=(batch, ntones))
    amps = 10.0 ** rng.uniform(-3.0, 0.0, size=(batch, ntones))
    phases = rng.uniform(0.0, 2.0 * np.pi, size=(batch, ntones))
    t = np.arange(n)
    out = np.zeros((batch, n), dtype=np.complex128)
    for k in range(ntones):
        ang = 2.0 * np.pi * ((bins[:, k:k + 1] * t[None, :]) % n) / n + phases[:, k:k + 1]
        out += amps[:, k:k + 1] * np.exp(1j * ang)
    out.real += rng.normal(0.0, noise_std, size=(batch, n))
    out.imag += rng.normal(0.0, noise_std, size=(batch, n))
    return out.astype(dtype)


def ragged_lengths(count: int, lo_log2: int, hi_log2: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return (1 << rng.integers(lo_log2, hi_log2 + 1, size=count)).astype(np.int64)


def uniform_batch_device(n: int, batch: int, seed: int, device="cuda", dtype=None):
    """Same distribution as ``uniform_batch`` drawn on the device with torch's
    seeded generator (for campaigns that only count detections and never
    compare against the oracle)."""
    import torch
    dtype = dtype or torch.complex64
    real = torch.float32 if dtype == torch.complex64 else torch.float64
    g = torch.Generator(device=device).manual_seed(seed)
    re = torch.rand(batch, n, generator=g, device=device, dtype=real) * 2 - 1
    im = torch.rand(batch, n, generator=g, device=device, dtype=real) * 2 - 1
    return torch.complex(re, im)
