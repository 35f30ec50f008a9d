"""Device ball query vs the oracle: full scans, and range-limited scans on
sorted clouds (which must give the full scan's result exactly)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2208_08795_gb300 import afps as B
from paper_2208_08795_gb300 import build as build_mod
from paper_2208_08795_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    build_mod.build()
    s = B.Sampler(0)
    yield s
    s.close()


@pytest.mark.parametrize("axis", [-1, 0])
@pytest.mark.parametrize("radius,K", [(0.2, 32), (0.05, 16), (0.5, 64), (1e-6, 8), (3.0, 128)])
def test_ball_query_matches_oracle(S, axis, radius, K):
    clouds = synth.object_batch(2, 6, 2048) + [synth.slab_cloud(5, 9000), synth.uniform_cloud(3, 40)]
    if axis == -1:  # unsorted storage for the full scan
        g = np.random.Generator(np.random.PCG64(1))
        clouds = [c[g.permutation(c.shape[0])] for c in clouds]
    Cs = [512] * 6 + [2000, 40]
    sels = [oracle.afps(P, Cs[b], 8 if Cs[b] >= 8 else 1, 0) for b, P in enumerate(clouds)]
    xyz, off = synth.pack(clouds)
    sel_off = np.zeros(len(sels) + 1, dtype=np.int64)
    np.cumsum([len(s) for s in sels], out=sel_off[1:])
    sel = torch.from_numpy(np.concatenate(sels)).cuda()
    got = S.ball_query(torch.from_numpy(xyz).cuda(), off, sel, sel_off, radius, K, axis)
    S.sync()
    got = got.cpu().numpy()
    for b, P in enumerate(clouds):
        ref = oracle.ball_query(P, sels[b], radius, K)
        assert np.array_equal(got[sel_off[b]:sel_off[b + 1]], ref), (b, radius, K, axis)


def test_grid_on_sphere_and_sorted_scan(S):
    """Points exactly on the sphere are excluded, also by the range-limited scan."""
    P = np.zeros((300, 3), dtype=np.float32)
    P[:, 0] = np.arange(300)
    cen = torch.tensor([0, 31, 32, 33, 150, 299], dtype=torch.int32).cuda()
    for axis in (-1, 0):
        got = S.ball_query(torch.from_numpy(P).cuda(), [0, 300], cen, [0, 6], 2.0, 4, axis)
        S.sync()
        ref = oracle.ball_query(P, cen.cpu().numpy(), 2.0, 4)
        assert np.array_equal(got.cpu().numpy(), ref), axis
