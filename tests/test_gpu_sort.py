"""Device sort by key vs the oracle (bit-exact permutation), and unsorted
input through sort -> NPDU-AFPS -> index composition."""
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


def shuffled(P, seed):
    g = np.random.Generator(np.random.PCG64(seed))
    return np.ascontiguousarray(P[g.permutation(P.shape[0])])


@pytest.mark.parametrize("key", [0, 1, 2, 3])
def test_sort_matches_oracle(S, key):
    clouds = [shuffled(synth.uniform_cloud(s, n, None), s) for s, n in
              enumerate([1, 2, 31, 32, 33, 1000, 2048, 4097, 32768, 70000])]
    clouds.append(shuffled(synth.lidar_frame(3), 1))
    for n in (3000, 50000):  # heavy ties on x; the second is sorted by a thread-block cluster
        q = synth.uniform_cloud(77 + n, n, None)
        q[:, 0] = np.round(q[:, 0] * 16) / 16
        q[:300, 1] = -0.0
        q[300:600, 1] = 0.0
        clouds.append(q)
    xyz, off = synth.pack(clouds)
    x = torch.from_numpy(xyz).cuda()
    out, perm = S.sort_by_key(x, off, key)
    S.sync()
    out, perm = out.cpu().numpy(), perm.cpu().numpy()
    for b, P in enumerate(clouds):
        ref_pts, ref_perm = oracle.sort_by_key(P, key)
        assert np.array_equal(perm[off[b]:off[b + 1]], ref_perm), (key, b)
        assert np.array_equal(out[off[b]:off[b + 1]], ref_pts), (key, b)


def test_unsorted_input_pipeline(S):
    """Unsorted cloud: sort by x on the device, sample, map the indices back."""
    P = shuffled(synth.slab_cloud(6, 16384), 3)
    x = torch.from_numpy(P).cuda()
    srt, perm = S.sort_by_key(x, [0, P.shape[0]], B.AFPS_KEY_X)
    idx = S.sample(srt, 4096, 32, 16, 0)
    frame_idx = perm[idx.long()]
    S.sync()
    ref_sorted, ref_perm = oracle.sort_by_key(P, oracle.KEY_X)
    ref = ref_perm[oracle.afps(ref_sorted, 4096, 32, 16)]
    assert np.array_equal(frame_idx.cpu().numpy(), ref)


def test_sort_cluster_capacity_boundary(S):
    """Clouds of 4096 points and below are sorted one CTA each, larger ones up
    to 16 x 12,288 points by a thread-block cluster in distributed shared
    memory, larger ones again one CTA each: every size around both limits
    gives the oracle's permutation."""
    clouds = [shuffled(synth.uniform_cloud(900 + i, n, None), i)
              for i, n in enumerate((4096, 4097, 16 * 12288, 16 * 12288 + 1))]
    xyz, off = synth.pack(clouds)
    x = torch.from_numpy(xyz).cuda()
    out, perm = S.sort_by_key(x, off, B.AFPS_KEY_Y)
    S.sync()
    out, perm = out.cpu().numpy(), perm.cpu().numpy()
    for b, P in enumerate(clouds):
        ref_pts, ref_perm = oracle.sort_by_key(P, B.AFPS_KEY_Y)
        assert np.array_equal(perm[off[b]:off[b + 1]], ref_perm), b
        assert np.array_equal(out[off[b]:off[b + 1]], ref_pts), b
