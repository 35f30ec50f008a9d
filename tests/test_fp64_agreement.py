"""FP32 vs FP64 oracle on the benchmark workloads: index agreement rate and
relative coverage-radius difference (target at most 1e-5)."""
import numpy as np
import pytest

import oracle
from paper_2208_08795_gb300 import synth


def agreement(P, C, M, k):
    a = oracle.afps(P, C, M, k)
    b = oracle.afps(P, C, M, k, precision="f64")
    r32, r64 = oracle.coverage_radius(P, a), oracle.coverage_radius(P, b)
    return float(np.mean(a == b)), abs(r32 - r64) / r64


@pytest.mark.parametrize("M,k", [(1, 0), (4, 0), (32, 16)])
def test_sphere_torus(M, k):
    rate, drel = agreement(synth.sphere_torus_cloud(0), 512, M, k)
    print(f"M={M} k={k}: agreement {rate:.4f}, relative coverage-radius difference {drel:.2e}")
    assert drel <= 1e-5


def test_object_batch_sample():
    for P in synth.object_batch(1, 32, 2048)[:8]:
        for (M, k) in ((1, 0), (32, 16)):
            rate, drel = agreement(P, 512, M, k)
            assert drel <= 1e-5, (M, k, rate, drel)
