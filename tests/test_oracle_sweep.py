"""A seeded random sweep of the oracle against the from-scratch brute-force
restatement (tests/oracle_pins.py) on tiny clouds: every combination of
sorted / unsorted / duplicated points, sector count, window, reading and
start that fits, beyond the hand-picked cases of the pins."""
import numpy as np

import oracle
from oracle_pins import brute_force
from paper_2208_08795_gb300 import synth


def test_random_small_configurations():
    g = np.random.Generator(np.random.PCG64(2024))
    checked = 0
    for case in range(800):
        N = int(g.integers(1, 97))
        M = int(g.integers(1, min(N, 8) + 1))
        C = int(g.integers(M, N + 1))
        # every sector must be able to give its samples: c_s <= n_s
        lo = [(s * N) // M for s in range(M + 1)]
        off = [(s * C) // M for s in range(M + 1)]
        if any(off[s + 1] - off[s] > lo[s + 1] - lo[s] for s in range(M)):
            continue
        k = int(g.choice([0, 0, 1, 2, 3, 4, 5, 8, 16, 100]))
        method = int(g.integers(0, 4)) if k > 0 else 0
        start = int(g.integers(0, N))
        kind = case % 3
        if kind == 0:
            P = synth.uniform_cloud(1000 + case, N)
        elif kind == 1:
            P = synth.uniform_cloud(1000 + case, N, axis=None)
        else:  # repeated points: ties everywhere
            base = synth.uniform_cloud(1000 + case, max(1, N // 3))
            P = np.ascontiguousarray(np.resize(base, (N, 3)).astype(np.float32))
        got = oracle.afps(P, C, M, k, start, method=method)
        ref = brute_force(P, C, M, k, start, method)
        assert np.array_equal(got, ref), (case, N, C, M, k, method, start, kind)
        checked += 1
    assert checked >= 600
