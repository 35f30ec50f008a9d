"""The oracle's sort by key against closed forms and the properties that
define a stable ascending sort."""
import numpy as np

import oracle
from paper_2208_08795_gb300 import synth


def test_diamond_angle_closed_form():
    x = np.array([1, 0, -1, 0, 1, -1, -1, 1, 0, 3, -2], np.float32)
    y = np.array([0, 1, 0, -1, 1, 1, -1, -1, 0, 1, -6], np.float32)
    want = [0, 1, 2, 3, 0.5, 1.5, 2.5, 3.5, 0, 0.25, 2.75]
    assert np.array_equal(oracle.diamond_angle(x, y), np.array(want, np.float32))


def test_diamond_angle_is_monotone_in_the_angle():
    g = np.random.Generator(np.random.PCG64(4))
    p = g.uniform(-2, 2, (30000, 2)).astype(np.float32)
    d = oracle.diamond_angle(p[:, 0], p[:, 1])
    a = np.mod(np.arctan2(p[:, 1].astype(np.float64), p[:, 0].astype(np.float64)), 2 * np.pi)
    o = np.argsort(d, kind="stable")
    strictly = d[o][1:] > d[o][:-1]
    assert not np.any(strictly & (a[o][1:] < a[o][:-1]))
    assert d.min() >= 0 and d.max() < 4


def test_sort_is_stable_ascending_permutation():
    g = np.random.Generator(np.random.PCG64(5))
    P = synth.uniform_cloud(9, 5000, axis=None)
    P[:, 0] = np.round(P[:, 0] * 20) / 20  # many equal keys
    P[:50, 1] = -0.0
    P[50:100, 1] = 0.0
    P = P[g.permutation(P.shape[0])]
    for key in (oracle.KEY_X, oracle.KEY_Y, oracle.KEY_Z, oracle.KEY_AZIMUTH):
        S, perm = oracle.sort_by_key(P, key)
        assert np.array_equal(np.sort(perm), np.arange(P.shape[0]))
        assert np.array_equal(S, P[perm])
        k = oracle.sort_key(P, key)[perm]
        assert np.all(k[1:] >= k[:-1])
        same = k[1:] == k[:-1]
        assert np.all(perm[1:][same] > perm[:-1][same])  # ties keep storage order
