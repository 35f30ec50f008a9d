"""The benchmark's count of algorithmic work (the numerator of its ALU
roofline) equals a direct count on small batches: every update after a
sample except the last reaches the sector's points inside the window (or the
whole sector without NPDU), and every argmax after the first sample scans
the sector."""
import numpy as np

import bench
import oracle
from paper_2208_08795_gb300 import afps as B
from paper_2208_08795_gb300 import synth


def direct_count(clouds, idx, C, M, k):
    evals = compares = 0
    for P, sel in zip(clouds, idx):
        N = P.shape[0]
        for s in range(M):
            lo, hi = s * N // M, (s + 1) * N // M
            o0, o1 = s * C // M, (s + 1) * C // M
            n = hi - lo
            for p in sel[o0:o1 - 1]:  # the last sample's update is never used
                local = int(p) - lo
                for j in range(n):
                    if k == 0 or (local - k // 2 <= j <= local + k - k // 2):
                        evals += 1
            compares += (o1 - o0 - 1) * n
    return evals, compares


def test_npdu_work_matches_a_direct_count():
    for (N, C, M, k) in ((256, 64, 4, 8), (300, 90, 3, 0), (200, 100, 10, 16), (97, 31, 1, 5)):
        clouds = synth.object_batch(3, 3, N)
        idx = [oracle.afps(P, C, M, k, 0) for P in clouds]
        _, off = synth.pack(clouds)
        ba = B.BatchArgs(off, C, M, k, 0)
        out = np.concatenate(idx)
        assert bench.npdu_work(out, ba, k) == direct_count(clouds, idx, C, M, k), (N, C, M, k)


def test_window_rule():
    assert [bench.k_rule(M) for M in (1, 4, 8, 16, 32, 128)] == [8, 8, 8, 16, 16, 16]
