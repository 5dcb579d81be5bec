"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module only draws random numbers and describes workload shapes; it holds
none of the transform's arithmetic, so both the CUDA path and the oracle may be
fed from it without sharing any code with each other.

Recipe (host numpy PCG64 generator, FP32 draws):
  * uniform:  re, im = 2 * U[0,1) - 1, i.e. i.i.d. uniform on [-1, 1)
  * gaussian: re, im i.i.d. standard normal (sigma = 1)
  * seed = 20260 + workload index, plus 1000 * size index inside a sweep.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 20260


def seed_for(workload: int, size_index: int = 0) -> int:
    return SEED_BASE + int(workload) + 1000 * int(size_index)


def uniform_c64(count: int, seed: int) -> np.ndarray:
    """``count`` complex64 values with real and imaginary parts i.i.d. uniform[-1, 1)."""
    rng = np.random.default_rng(seed)
    out = np.empty(int(count), dtype=np.complex64)
    v = out.view(np.float32)
    v[:] = rng.random(2 * int(count), dtype=np.float32)
    v *= 2.0
    v -= 1.0
    return out


def gaussian_c64(count: int, seed: int) -> np.ndarray:
    """``count`` complex64 values with real and imaginary parts i.i.d. N(0, 1)."""
    rng = np.random.default_rng(seed)
    out = np.empty(int(count), dtype=np.complex64)
    out.view(np.float32)[:] = rng.standard_normal(2 * int(count), dtype=np.float32)
    return out


# ---------------------------------------------------------------------------
# Workload shapes.  I/O dimensions are (n, input stride, output stride) in
# complex elements, as in dft(N, V, I, O).

def batched_1d(n: int, batch: int):
    """Contiguous batch of 1-D transforms: N = {(n,1,1)}, V = {(batch, n, n)}."""
    return [(n, 1, 1)], [(batch, n, n)]


def transposed_1d(n: int, batch: int):
    """Batch-fastest layout: N = {(n, batch, 1)}, V = {(batch, 1, n)}
    (input columns of a row-major n x batch matrix, output rows)."""
    return [(n, batch, 1)], [(batch, 1, n)]


POW2_SWEEP = [2 ** e for e in range(4, 25)]           # n = 2^4 .. 2^24
SWEEP_POINTS = 2 ** 26                                 # batch = 2^26 / n
UNEVEN_SIZES = [1000, 2187, 3125, 7168, 10007, 65536]  # batch 512 each
UNEVEN_BATCH = 512
UNEVEN_TRANSPOSED = {2187, 7168, 65536}                # the rest contiguous


# ---------------------------------------------------------------------------
# Serving workload: requests with Poisson arrivals.

SERVING_BUDGET = 40 * 10 ** 9


def _split_pow2(e, r):
    """2^e split into r near-equal power-of-two factors (exponents differ by <= 1)."""
    base, extra = divmod(e, r)
    return tuple(2 ** (base + (1 if i < extra else 0)) for i in range(r))


def serving_requests(count, seed):
    """Request shapes of the serving workload: with probability 0.8 a total size
    n = 2^e, e uniform in [6, 20], else n uniform in [100, 10^5] and not a power
    of two; rank 1 / 2 / 3 with probabilities 0.7 / 0.2 / 0.1 (a power of two is
    split into near-equal power-of-two factors, a non-power-of-two rank-r shape
    draws each dimension uniformly, not a power of two, in
    [ceil(100^(1/r)), floor(10^5^(1/r))]); batch uniform in [1, 256]; sign +-1.
    Returns a list of (shape tuple, batch, sign)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(int(count)):
        r = int(rng.choice([1, 2, 3], p=[0.7, 0.2, 0.1]))
        if rng.random() < 0.8:
            shape = _split_pow2(int(rng.integers(6, 21)), r)
        else:
            lo = int(np.ceil(100 ** (1.0 / r)))
            hi = int(np.floor((10 ** 5) ** (1.0 / r)))
            dims = []
            for _d in range(r):
                while True:
                    v = int(rng.integers(lo, hi + 1))
                    if v & (v - 1):
                        break
                dims.append(v)
            shape = tuple(dims)
        out.append((shape, int(rng.integers(1, 257)), int(rng.choice([-1, 1]))))
    return out


def poisson_arrivals(count, rate, seed):
    """Arrival times (seconds) of a Poisson process of the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=int(count)))
