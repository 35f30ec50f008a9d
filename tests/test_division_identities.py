"""The two division shortcuts the sector kernels use, checked on the CPU
against exact integer division (the GPU parity tests exercise the kernels
that use them).

- Sector bounds of a run of equal clouds, floor(x / M) for x < 2^32: the
  high 64 bits of x * m with m = floor((2^64 - 1) / M) + 1.
- Stride-phase and cluster-record indices, floor(x / d) for x < 2^24: the
  float32 product of x and the rounded reciprocal of d, truncated, is at
  most one off, and one check each way corrects it.
"""
import numpy as np


def magic(d: int) -> int:
    return (2**64 - 1) // d + 1


def test_multiply_high_division():
    g = np.random.default_rng(5)
    ds = list(range(2, 300)) + [2**k for k in range(1, 31)] + \
        [2**k + 1 for k in range(1, 31)] + [2**k - 1 for k in range(2, 32)] + \
        [int(v) for v in g.integers(2, 2**31, 200)]
    for d in ds:
        m = magic(d)
        xs = [0, 1, d - 1, d, d + 1, 2**32 - 1, 2**32 - 2, (2**32 - 1) // d * d,
              (2**32 - 1) // d * d - 1] + [int(v) for v in g.integers(0, 2**32, 64)]
        for x in xs:
            if 0 <= x < 2**32:
                assert (x * m) >> 64 == x // d, (x, d)


def float_quotient(x: np.ndarray, d: int) -> np.ndarray:
    r = np.float32(1.0) / np.float32(d)                  # rounded reciprocal
    prod = x.astype(np.float32) * r                        # exact conversion (x < 2^24), rounded product
    return np.trunc(prod).astype(np.int64)


def test_float_reciprocal_division_is_within_one():
    x = np.arange(0, 2**17 + 64, dtype=np.int64)           # every index of the largest sector
    for d in list(range(1, 1100)) + [2**k + o for k in range(11, 18) for o in (-1, 0, 1)]:
        t = float_quotient(x, d)
        exact = x // d
        assert np.abs(t - exact).max() <= 1, d
        t = t - (t * d > x)
        t = t + ((t + 1) * d <= x)
        assert np.array_equal(t, exact), d


def test_float_reciprocal_division_large_numerators():
    g = np.random.default_rng(6)
    x = np.concatenate([g.integers(0, 2**24, 200000), np.arange(2**24 - 4096, 2**24)])
    for d in [2, 3, 5, 7, 9, 17, 33, 1000, 4095, 65537, 2**20 + 3, 2**23 - 1]:
        t = float_quotient(x, d)
        assert np.abs(t - x // d).max() <= 1, d
