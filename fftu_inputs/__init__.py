"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module holds no FFT arithmetic.  It only turns (seed, element index) into
numbers, so that the FP64 oracle and the CUDA path can be fed the exact same
array without either one importing the other.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), used in its counter form: the 64-bit word for
counter value c is mix64(seed + (c + 1) * GOLDEN), where mix64 is the
SplitMix64 output function (xor-shift 30, multiply, xor-shift 27, multiply,
xor-shift 31) and GOLDEN = 0x9E3779B97F4A7C15.  The top 53 bits give
u in [0, 1); the value is 2u - 1 in [-1, 1).  Element j of a complex array takes
counter 2j for its real part and 2j + 1 for its imaginary part, so any
sub-range can be regenerated on its own (the oracle's sampled checks use this).

The paper's workloads are arrays of N = 2^30 complex numbers in shapes 1024^3,
64^5 and 2^24 x 64 with no dataset behind them; these uniform[-1, 1) arrays
stand in for them.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22

__all__ = ["splitmix64", "uniform_pm1", "complex_uniform", "complex_uniform_range", "complex_loguniform"]


def splitmix64(seed: int, counters: np.ndarray) -> np.ndarray:
    """SplitMix64 output words for the given counter values (uint64 array)."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (c + np.uint64(1)) * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_pm1(seed: int, counters: np.ndarray) -> np.ndarray:
    """Doubles in [-1, 1) from the top 53 bits of each SplitMix64 word."""
    z = splitmix64(seed, counters)
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return 2.0 * u - 1.0


def complex_uniform_range(seed: int, start: int, count: int, dtype=np.complex128) -> np.ndarray:
    """Elements [start, start + count) of the seeded complex array, flat."""
    out = np.empty(count, dtype=dtype)
    real_dtype = np.float32 if np.dtype(dtype) == np.complex64 else np.float64
    view = out.view(real_dtype)
    pos = 0
    while pos < count:
        m = min(_CHUNK, count - pos)
        ctr = np.arange(2 * (start + pos), 2 * (start + pos + m), dtype=np.uint64)
        view[2 * pos: 2 * (pos + m)] = uniform_pm1(seed, ctr)
        pos += m
    return out


def complex_uniform(seed: int, shape, dtype=np.complex128) -> np.ndarray:
    """Row-major array of the given shape, Re and Im i.i.d. uniform[-1, 1).

    complex64 values are the FP64 draws rounded once to FP32; the oracle is then
    fed those exact FP32 values promoted to FP64.
    """
    shape = tuple(int(s) for s in shape)
    n = int(np.prod(shape)) if shape else 1
    return complex_uniform_range(seed, 0, n, dtype).reshape(shape)


def complex_loguniform(seed: int, shape, lo: float = 1e-3, hi: float = 1e3, dtype=np.complex128) -> np.ndarray:
    """Row-major array whose magnitudes are log-uniform in [lo, hi) and phases uniform.

    Element j: u = the (counter 2j, 2j + 1) pair mapped to [0, 1) as in complex_uniform;
    magnitude 10^(log10 lo + u_0 (log10 hi - log10 lo)), phase 2 pi u_1.  The wide dynamic
    range tests arithmetic whose 16-bit operands need scaling.
    """
    shape = tuple(int(s) for s in shape)
    n = int(np.prod(shape)) if shape else 1
    out = np.empty(n, dtype=dtype)
    a, b = np.log10(lo), np.log10(hi)
    pos = 0
    while pos < n:
        m = min(_CHUNK, n - pos)
        ctr = np.arange(2 * pos, 2 * (pos + m), dtype=np.uint64)
        u = 0.5 * (uniform_pm1(seed, ctr) + 1.0)
        mag = 10.0 ** (a + (b - a) * u[0::2])
        ph = 2.0 * np.pi * u[1::2]
        out[pos: pos + m] = mag * np.cos(ph) + 1j * (mag * np.sin(ph))
        pos += m
    return out.reshape(shape)
