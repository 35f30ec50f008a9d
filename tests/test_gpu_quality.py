"""Device coverage radius vs the oracle's (fp64, bit-identical), and the
quality study's tables on a few clouds."""
import numpy as np
import pytest
import torch

import oracle
from paper_2208_08795_gb300 import afps as B
from paper_2208_08795_gb300 import build as build_mod
from paper_2208_08795_gb300 import quality, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    build_mod.build()
    s = B.Sampler(0)
    yield s
    s.close()


def test_coverage_radius_matches_oracle(S):
    clouds = [synth.uniform_cloud(1, 1), synth.uniform_cloud(2, 700), synth.slab_cloud(3, 9000),
              synth.sphere_torus_cloud(0)] + synth.object_batch(4, 4, 2048)
    sels = [np.array([0]), np.arange(0, 700, 7), oracle.afps(clouds[2], 2000, 8, 8),
            oracle.fps(clouds[3], 512)] + [oracle.afps(P, 512, 32, 16) for P in clouds[4:]]
    xyz, off = synth.pack(clouds)
    sel_off = np.zeros(len(sels) + 1, dtype=np.int64)
    np.cumsum([len(s) for s in sels], out=sel_off[1:])
    sel = torch.from_numpy(np.concatenate(sels).astype(np.int32)).cuda()
    r = S.coverage_radius(torch.from_numpy(xyz).cuda(), off, sel, sel_off)
    S.sync()
    got = r.cpu().numpy()
    for b, P in enumerate(clouds):
        assert got[b] == oracle.coverage_radius(P, sels[b]), b  # exact


def test_quality_tables(S):
    clouds = synth.object_batch(1, 4, 2048)
    t2 = quality.table_ii(S, clouds)
    assert set(t2) == set(quality.ORDERS)
    for vals in t2.values():
        assert all(v > 0.5 for v in vals.values())
    f6 = quality.fig6(S, clouds, ks=(8, 64))
    assert set(f6) == {"default", "full_first_pass", "window_has_sample"}
    f7 = quality.fig7(S, clouds, Ms=(4, 32), ks=(16,))
    assert f7["M=4"]["k=0"] > 0
