"""Seeded synthetic inputs shaped like the paper's radar workloads.

This module only draws inputs: it holds none of the transform's arithmetic, so
both the CUDA path and the FP64 oracle may consume what it produces.  The
paper uses no dataset; its workloads are batched 1-D FFTs of radar lines,
N = 2^10..2^14, batch 256..16384 (Sec. II-D), timed on batches of N(0,1)-like
data (Sec. VI-A).  Every generator is deterministic in its ``seed`` and uses
NumPy's PCG64 stream.

Recipes
  gaussian     re and im i.i.d. N(0, 1) (float32), i.e. E|x|^2 = 2.
  uniform      re and im i.i.d. U[lo, hi).
  lfm_chirp    unit-amplitude linear-FM chirp per row, instantaneous frequency
               swept from -B/2 to +B/2 cycles/sample over Np samples
               (B = 0.8 by default), start phase U[0, 2 pi) per row, plus
               complex white Gaussian noise at the requested SNR.
  sar_echoes   range lines made of 8 delayed, complex-scaled copies of one
               reference chirp (Np samples, zero-padded to N) plus noise at
               the requested SNR relative to each line's signal power; also
               returns the zero-padded reference pulse.
  real_mask    real weights U[0, 1).
  ragged_draw  a mixed-size batch: log2 N ~ U{lo..hi}, direction ~
               Bernoulli(1/2) in {-1, +1}, packed contiguously in draw order.
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def gaussian(shape, seed: int = 0) -> np.ndarray:
    shape = tuple(int(s) for s in np.atleast_1d(shape))
    a = _rng(seed).standard_normal(shape + (2,), dtype=np.float32)
    return a.view(np.complex64).reshape(shape)


def uniform(shape, seed: int = 0, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    shape = tuple(int(s) for s in np.atleast_1d(shape))
    a = _rng(seed).uniform(lo, hi, size=shape + (2,)).astype(np.float32)
    return a.view(np.complex64).reshape(shape)


def _chirp_phase_cycles(n: np.ndarray, Np: int, bandwidth: float) -> np.ndarray:
    """Phase in cycles of an LFM sweeping -B/2..+B/2 cycles/sample over Np samples."""
    n = n.astype(np.float64)
    cyc = -0.5 * bandwidth * n + 0.5 * bandwidth * (n * n) / float(Np)
    return cyc - np.floor(cyc)


def _awgn(rng: np.random.Generator, shape, power: np.ndarray, snr_db: float) -> np.ndarray:
    """Complex white Gaussian noise with total variance power * 10^(-snr/10)."""
    sigma = np.sqrt(np.asarray(power, dtype=np.float64) * 10.0 ** (-snr_db / 10.0) / 2.0)
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return (re + 1j * im) * sigma


def lfm_chirp(batch: int, N: int, seed: int = 1, snr_db: float = 10.0,
              bandwidth: float = 0.8, Np: int | None = None) -> np.ndarray:
    """Rows of unit-amplitude LFM chirps (filling Np = N samples) plus AWGN."""
    rng = _rng(seed)
    Np = N if Np is None else int(Np)
    n = np.arange(N)
    base = _chirp_phase_cycles(np.minimum(n, Np - 1), Np, bandwidth)
    active = (n < Np).astype(np.float64)
    phi0 = rng.uniform(0.0, 1.0, size=(batch, 1))           # start phase, cycles
    out = np.empty((batch, N), dtype=np.complex64)
    step = max(1, (1 << 22) // max(N, 1))
    for r0 in range(0, batch, step):
        r1 = min(batch, r0 + step)
        ph = 2.0 * np.pi * (base[None, :] + phi0[r0:r1])
        sig = active[None, :] * np.exp(1j * ph)
        noise = _awgn(rng, (r1 - r0, N), 1.0, snr_db)
        out[r0:r1] = (sig + noise).astype(np.complex64)
    return out


def reference_pulse(N: int, Np: int, bandwidth: float = 0.8) -> np.ndarray:
    """The zero-padded reference chirp (start phase 0) used by sar_echoes."""
    n = np.arange(Np)
    p = np.zeros(N, dtype=np.complex128)
    p[:Np] = np.exp(2j * np.pi * _chirp_phase_cycles(n, Np, bandwidth))
    return p.astype(np.complex64)


def sar_echoes(lines: int, N: int, Np: int = 2048, seed: int = 0,
               n_targets: int = 8, snr_db: float = 10.0, bandwidth: float = 0.8):
    """Chirp-echo range lines: sum of delayed, scaled pulses plus noise.

    Returns (x [lines, N] complex64, pulse [N] complex64 zero-padded).
    """
    rng = _rng(seed)
    pulse = reference_pulse(N, Np, bandwidth).astype(np.complex128)[:Np]
    x = np.zeros((lines, N), dtype=np.complex128)
    rows = np.arange(lines)
    cols = np.arange(Np)
    for _ in range(n_targets):
        delay = rng.integers(0, max(1, N - Np), size=lines)
        amp = rng.standard_normal(lines) + 1j * rng.standard_normal(lines)
        x[rows[:, None], delay[:, None] + cols[None, :]] += amp[:, None] * pulse[None, :]
    power = np.mean(np.abs(x) ** 2, axis=1, keepdims=True)
    x += _awgn(rng, (lines, N), power, snr_db)
    return x.astype(np.complex64), reference_pulse(N, Np, bandwidth)


def real_mask(shape, seed: int = 2) -> np.ndarray:
    shape = tuple(int(s) for s in np.atleast_1d(shape))
    return _rng(seed).uniform(0.0, 1.0, size=shape).astype(np.float32)


def ragged_draw(count: int, seed: int = 0, log2_lo: int = 8, log2_hi: int = 14):
    """Sizes, directions and packed offsets (in complex elements) of a ragged batch.

    Returns a dict with int32 ``N``, int32 ``direction`` (-1 forward, +1
    inverse), int64 ``offset`` and the int64 ``total`` element count.
    """
    rng = _rng(seed)
    log2n = rng.integers(log2_lo, log2_hi + 1, size=count)
    direction = np.where(rng.integers(0, 2, size=count) == 1, 1, -1).astype(np.int32)
    N = (1 << log2n).astype(np.int32)
    offset = np.zeros(count, dtype=np.int64)
    if count:
        offset[1:] = np.cumsum(N[:-1].astype(np.int64))
    total = int(N.astype(np.int64).sum())
    return {"N": N, "direction": direction, "offset": offset, "total": total}
