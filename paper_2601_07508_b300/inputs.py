"""Seeded synthetic inputs: primes, matrices, shapes and arrival times.

This module holds no arithmetic of the multiword method. It produces the
inputs that the GPU path, the CPU oracle and the benchmark all consume, so
that every side sees bit-identical data from the same seed.

Generator. Every draw is a pure function of (seed, stream, counter): the
splitmix64 output function (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014; constants as published by
Vigna) applied to ``base + (counter + 1) * golden_gamma`` with
``base = mix(seed ^ mix(stream))``.  Being counter based it vectorises in
numpy, so 8192 x 8192 matrices are generated in seconds.

Entries uniform in [0, p): the top ``bitlen(p)`` bits of a draw are kept
and values >= p are rejected; a rejected element ``idx`` retries with
counter ``idx + attempt * 2^40`` until it lands in range, so the first r rows
of a matrix do not depend on how many rows are drawn.

Primes. ``is_prime`` is the deterministic Miller-Rabin test with the first
twelve prime bases, which is exact for every n < 3.3e24 (Sorenson and
Webster, Math. Comp. 2017), hence for all 64-bit n.
"""

from __future__ import annotations

import math
from typing import Iterable, List, Sequence, Tuple

import numpy as np

_MASK64 = (1 << 64) - 1
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Streams used by the workloads; A and B of one problem never share a stream.
STREAM_A = 1
STREAM_B = 2
STREAM_SHAPES = 3
STREAM_PRIMES = 4
STREAM_ARRIVALS = 5


def _mix_scalar(z: int) -> int:
    z &= _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def stream_base(seed: int, stream: int) -> int:
    return _mix_scalar((seed & _MASK64) ^ _mix_scalar(stream))


def draws(seed: int, stream: int, counters: np.ndarray) -> np.ndarray:
    """64-bit draws number ``counters`` of stream (seed, stream)."""
    base = np.uint64(stream_base(seed, stream))
    c = counters.astype(np.uint64, copy=False)
    with np.errstate(over="ignore"):
        z = base + (c + np.uint64(1)) * _GOLDEN
    return _mix(z)


def uniform_mod(seed: int, stream: int, count: int, p: int) -> np.ndarray:
    """``count`` integers uniform in [0, p) as uint64 (p < 2^63)."""
    if p < 1 or p >= (1 << 63):
        raise ValueError("p must be in [1, 2^63)")
    if count >= (1 << 40):
        raise ValueError("at most 2^40 draws per stream")
    bits = max(1, (p - 1).bit_length())
    shift = np.uint64(64 - bits)
    out = np.empty(count, dtype=np.uint64)
    idx = np.arange(count, dtype=np.uint64)
    todo = idx
    attempt = 0
    while todo.size:
        vals = draws(seed, stream, todo + np.uint64(attempt << 40)) >> shift
        ok = vals < np.uint64(p)
        out[todo[ok]] = vals[ok]
        todo = todo[~ok]
        attempt += 1
        if attempt > 10_000:
            raise RuntimeError("rejection sampling did not terminate")
    return out


def matrix(seed: int, stream: int, rows: int, cols: int, p: int) -> np.ndarray:
    """Row-major rows x cols uint64 matrix with entries uniform in [0, p)."""
    return uniform_mod(seed, stream, rows * cols, p).reshape(rows, cols)


def problem(seed: int, m: int, n: int, k: int, p: int) -> Tuple[np.ndarray, np.ndarray]:
    """A (m x k) and B (k x n) of one product, from streams STREAM_A / STREAM_B."""
    return matrix(seed, STREAM_A, m, k, p), matrix(seed, STREAM_B, k, n, p)


def uniform01(seed: int, stream: int, count: int) -> np.ndarray:
    """Doubles uniform in [0, 1) (53 top bits of each draw)."""
    d = draws(seed, stream, np.arange(count, dtype=np.uint64)) >> np.uint64(11)
    return d.astype(np.float64) * (1.0 / (1 << 53))


def loguniform_dims(seed: int, stream: int, count: int, lo: int, hi: int) -> np.ndarray:
    """Integers floor(exp(U[ln lo, ln(hi + 1)))) clamped to [lo, hi]."""
    u = uniform01(seed, stream, count)
    x = np.floor(np.exp(math.log(lo) + u * (math.log(hi + 1) - math.log(lo))))
    return np.clip(x, lo, hi).astype(np.int64)


# --------------------------------------------------------------------------
# Primes
# --------------------------------------------------------------------------
_MR_BASES = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)


def is_prime(n: int) -> bool:
    """Deterministic Miller-Rabin; exact for n < 3.3e24."""
    if n < 2:
        return False
    for b in _MR_BASES:
        if n % b == 0:
            return n == b
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in _MR_BASES:
        x = pow(a, d, n)
        if x == 1 or x == n - 1:
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def prev_prime(n: int) -> int:
    """Largest prime strictly below n (downward search)."""
    c = n - 1
    while c >= 2:
        if is_prime(c):
            return c
        c -= 1
    raise ValueError("no prime below %d" % n)


def largest_prime_below_pow2(b: int) -> int:
    return prev_prime(1 << b)


def primes_below(n: int, count: int) -> List[int]:
    """The ``count`` largest primes below n, in decreasing order."""
    out: List[int] = []
    c = n
    while len(out) < count:
        c = prev_prime(c)
        out.append(c)
    return out


def random_prime_of_bitsize(seed: int, stream: int, index: int, b: int) -> int:
    """A prime of bitsize b: the first prime at or below a uniform draw in
    [2^(b-1), 2^b), searching downward and wrapping upward if none is found."""
    lo, hi = 1 << (b - 1), 1 << b
    z = int(draws(seed, stream, np.array([index], dtype=np.uint64))[0])
    start = lo + z % (hi - lo)
    c = start
    while c >= lo:
        if is_prime(c):
            return c
        c -= 1
    c = start + 1
    while c < hi:
        if is_prime(c):
            return c
        c += 1
    raise ValueError("no prime of bitsize %d" % b)


def poisson_arrivals(seed: int, count: int, rate_per_s: float) -> np.ndarray:
    """Arrival times (seconds, increasing) of a Poisson process of the given rate."""
    u = uniform01(seed, STREAM_ARRIVALS, count)
    gaps = -np.log1p(-u) / rate_per_s
    return np.cumsum(gaps)


# --------------------------------------------------------------------------
# Workload recipes (shapes and primes of the configured workloads)
# --------------------------------------------------------------------------
SWEEP_BITS = (20, 23, 26, 32, 40, 48, 52)


def batch_instances(seed: int = 4, count: int = 512, nprimes: int = 64,
                    lo: int = 128, hi: int = 2048, top_bits: int = 50):
    """(m, n, k, p) of the batched multi-prime workload: instance i uses prime
    number i mod nprimes among the nprimes largest primes below 2^top_bits."""
    primes = primes_below(1 << top_bits, nprimes)
    dims = loguniform_dims(seed, STREAM_SHAPES, 3 * count, lo, hi).reshape(count, 3)
    return [(int(d[0]), int(d[1]), int(d[2]), primes[i % nprimes]) for i, d in enumerate(dims)]


def serve_requests(seed: int = 5, count: int = 20000, lo: int = 64, hi: int = 4096,
                   bmin: int = 20, bmax: int = 52):
    """(m, n, k, p) of the serving workload; bitsize uniform in [bmin, bmax]."""
    dims = loguniform_dims(seed, STREAM_SHAPES, 3 * count, lo, hi).reshape(count, 3)
    bz = draws(seed, STREAM_PRIMES, np.arange(count, dtype=np.uint64))
    bits = (bz % np.uint64(bmax - bmin + 1)).astype(np.int64) + bmin
    out = []
    for i in range(count):
        p = random_prime_of_bitsize(seed, STREAM_PRIMES + 100, i, int(bits[i]))
        out.append((int(dims[i, 0]), int(dims[i, 1]), int(dims[i, 2]), p))
    return out
