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


def test_host_magic_numbers_from_the_runtime_header(tmp_path):
    """The runtime's own div_magic (afps_internal.h), compiled on the host:
    the high 64 bits of x * div_magic(d) equal x / d for 32-bit x."""
    import os
    import shutil
    import subprocess
    import pytest
    gxx = shutil.which("g++")
    cuda_inc = "/usr/local/cuda/include"
    if gxx is None or not os.path.isdir(cuda_inc):
        pytest.skip("needs g++ and the CUDA headers")
    here = os.path.dirname(os.path.abspath(__file__))
    csrc = os.path.join(here, "..", "paper_2208_08795_gb300", "csrc")
    src = tmp_path / "magic.cpp"
    src.write_text(r'''
#include "afps_internal.h"
#include <cstdio>
int main() {
    const uint32_t ds[] = {2, 3, 5, 7, 9, 16, 17, 31, 32, 33, 100, 255, 256, 1000, 4095, 65535,
                           65536, 65537, 1u << 20, (1u << 20) + 1, 123456789u, 2147483647u};
    uint64_t s = 88172645463325252ull, bad = 0, n = 0;
    for (uint32_t d : ds) {
        const uint64_t m = afps::div_magic((int32_t)d);
        for (int i = 0; i < 200000; ++i) {
            s ^= s << 13; s ^= s >> 7; s ^= s << 17;  // xorshift64
            uint32_t x = (uint32_t)s;
            if (i < 8) x = (uint32_t)(0xffffffffu - i);
            if (i >= 8 && i < 16) x = (uint32_t)((0xffffffffu / d) * d - (i - 8));
            const uint32_t hi = (uint32_t)(((unsigned __int128)x * m) >> 64);
            bad += hi != x / d;
            ++n;
        }
    }
    if (afps::div_magic(1) != 0 || afps::div_magic(0) != 0) ++bad;
    std::printf("%llu %llu\n", (unsigned long long)bad, (unsigned long long)n);
    return bad != 0;
}
''')
    exe = tmp_path / "magic"
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", csrc, "-I", cuda_inc, str(src), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
