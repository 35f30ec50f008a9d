"""Device k nearest neighbours vs the oracle: indices and squared distances,
full scans of unsorted clouds and outward scans of sorted ones (which must
give the full scan's result exactly), with ties resolved by index."""
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


def run_knn(S, clouds, sels, K, axis):
    xyz, off = synth.pack(clouds)
    sel_off = np.zeros(len(sels) + 1, dtype=np.int64)
    np.cumsum([len(s) for s in sels], out=sel_off[1:])
    sel = torch.from_numpy(np.concatenate(sels).astype(np.int32)).cuda()
    d2 = torch.empty((int(sel_off[-1]), K), dtype=torch.float32, device="cuda")
    got = S.knn(torch.from_numpy(xyz).cuda(), off, sel, sel_off, K, axis, dist2=d2)
    S.sync()
    return got.cpu().numpy(), d2.cpu().numpy(), sel_off


@pytest.mark.parametrize("axis", [-1, 0])
@pytest.mark.parametrize("K", [1, 16, 32, 33, 64])
def test_knn_matches_oracle(S, axis, K):
    clouds = synth.object_batch(4, 5, 2048) + [synth.slab_cloud(6, 4000), synth.uniform_cloud(8, 70)]
    if axis == -1:  # unsorted storage for the full scan
        g = np.random.Generator(np.random.PCG64(2))
        clouds = [c[g.permutation(c.shape[0])] for c in clouds]
    Cs = [512] * 5 + [500, 70]
    sels = [oracle.afps(P, Cs[b], 4, 0) for b, P in enumerate(clouds)]
    got, d2, sel_off = run_knn(S, clouds, sels, K, axis)
    for b, P in enumerate(clouds):
        ref, rd2 = oracle.knn(P, sels[b], K, with_d2=True)
        assert np.array_equal(got[sel_off[b]:sel_off[b + 1]], ref), (b, K, axis)
        assert np.array_equal(d2[sel_off[b]:sel_off[b + 1]], rd2), (b, K, axis)


@pytest.mark.parametrize("K", [9, 40, 64])
def test_knn_grid_ties(S, K):
    """Integer grid: every distance but the centroid's own comes in equal
    pairs, resolved to the lower index, across 32-point chunk boundaries."""
    P = np.zeros((300, 3), dtype=np.float32)
    P[:, 0] = np.arange(300)
    cen = np.array([0, 31, 32, 33, 150, 298, 299])
    for axis in (-1, 0):
        got, _, _ = run_knn(S, [P], [cen], K, axis)
        assert np.array_equal(got, oracle.knn(P, cen, K)), axis


def test_knn_duplicates_and_coarse_coordinates(S):
    """Coordinates rounded to a coarse grid and repeated points: many equal
    distances; the sorted scan must still agree with the full one."""
    g = np.random.Generator(np.random.PCG64(3))
    P = np.round(g.uniform(0, 1, (3000, 3)) * 6).astype(np.float32)
    P[::5] = P[7]
    P = P[np.lexsort((P[:, 2], P[:, 1], P[:, 0]))]
    cen = np.arange(0, 3000, 11)
    for axis in (-1, 0):
        got, d2, _ = run_knn(S, [P], [cen], 64, axis)
        ref, rd2 = oracle.knn(P, cen, 64, with_d2=True)
        assert np.array_equal(got, ref), axis
        assert np.array_equal(d2, rd2), axis


def test_knn_rejects_bad_arguments(S):
    P = torch.from_numpy(synth.uniform_cloud(1, 50)).cuda()
    sel = torch.zeros(4, dtype=torch.int32, device="cuda")
    for K, axis in ((0, -1), (65, -1), (51, 0), (8, 3)):
        with pytest.raises(B.AfpsError) as ei:
            S.knn(P, [0, 50], sel, [0, 4], K, axis)
        assert ei.value.code == B.AFPS_ERR_INVALID_ARG
    S.sync()
