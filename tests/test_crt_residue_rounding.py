"""The rounding argument behind the CRT split's FP32 residues, checked
exhaustively on the host.

The split reduces an entry x < 2^52 modulo each odd prime m < 256 on the FP32
pipe: a congruent integer 0 <= z < 2^21 is formed from 11-bit limbs, then
q = rint(z * fl(1/m)) (one rounding, inside an FMA against 1.5 * 2^23) and
r = z - q m.  The claim is that r is always the balanced residue of z, i.e.
that the single rounding of z * fl(1/m) never lands on the wrong integer.
Here every z below 2^21 is run through that step for every modulus, with the
FMA's rounding emulated in exact integer arithmetic, and the result is
compared with the residue computed by integer division.  The device code
itself is compared with the oracle's residue words in the GPU tests."""
import numpy as np


def _odd_primes_below_256():
    return [q for q in range(3, 256) if all(q % d for d in range(2, int(q ** 0.5) + 1))]


def _rint_times_float32(z: np.ndarray, inv: np.float32) -> np.ndarray:
    """rint(z * inv) with ties to even, in exact integer arithmetic (inv a float32)."""
    mant, ex = np.frexp(np.float64(inv))      # a float32 value is exact in float64
    M = int(mant * (1 << 24))                 # inv = M * 2^(ex - 24), M < 2^24
    s = 24 - int(ex)
    assert M * 2.0 ** -s == float(inv)
    num = z * M                               # < 2^21 * 2^24: exact in int64
    q = num >> s
    rem = num - (q << s)
    half = 1 << (s - 1)
    up = (rem > half) | ((rem == half) & ((q & 1) == 1))
    return q + up.astype(np.int64)


def test_fp32_residue_step_is_the_balanced_residue_for_every_z():
    z = np.arange(0, 1 << 21, dtype=np.int64)
    for m in _odd_primes_below_256():
        inv = np.float32(1.0) / np.float32(m)  # what the host passes: IEEE single division
        r = z - _rint_times_float32(z, inv) * m
        h = (m - 1) // 2
        assert np.array_equal(r, (z + h) % m - h), m


def test_limb_sum_stays_below_2_21_and_is_congruent():
    rng = np.random.default_rng(7)
    x = np.concatenate([rng.integers(0, 1 << 52, 4096, dtype=np.int64),
                        np.array([0, 1, (1 << 52) - 1, (1 << 44) - 1, 1 << 44], dtype=np.int64)])
    limbs = [(x >> (11 * j)) & 0x7FF for j in range(4)] + [x >> 44]
    for m in _odd_primes_below_256():
        c = [1] + [(1 << (11 * j)) % m for j in range(1, 5)]
        z = sum(l * cj for l, cj in zip(limbs, c))
        assert int(z.max()) < (1 << 21)
        assert np.array_equal(z % m, x % m), m
