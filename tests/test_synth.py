"""The seeded synthetic inputs match their stated recipes: sizes, storage
order (sorted by x, approximately sorted in bins, or column by column by
azimuth), value ranges, pairwise-distinct points, and determinism per seed.
Every parity test and the benchmark draw their inputs from these."""
import numpy as np

from paper_2208_08795_gb300 import synth


def distinct(p):
    return np.unique(p, axis=0).shape[0] == p.shape[0]


def sorted_by(p, axis=0):
    return bool(np.all(np.diff(p[:, axis]) >= 0))


def test_sphere_torus_cloud():
    p = synth.sphere_torus_cloud(0)
    assert p.shape == (2048, 3) and p.dtype == np.float32 and p.flags.c_contiguous
    assert sorted_by(p) and distinct(p)
    r = np.linalg.norm(p.astype(np.float64), axis=1)
    on_sphere = np.abs(r - 1.0) < 1e-5
    assert on_sphere.sum() >= 1024  # the sphere half (torus points can not reach r = 1)
    torus = p[~on_sphere].astype(np.float64)
    rho = np.hypot(torus[:, 0], torus[:, 1])
    tube = np.hypot(rho - 0.5, torus[:, 2])  # distance from the torus' core circle
    assert np.allclose(tube, 0.1, atol=1e-5)
    assert np.array_equal(p, synth.sphere_torus_cloud(0))
    assert not np.array_equal(p, synth.sphere_torus_cloud(1))


def test_object_batch():
    clouds = synth.object_batch(1, 32, 2048)
    assert len(clouds) == 32
    for c in clouds:
        assert c.shape == (2048, 3) and c.dtype == np.float32
        assert sorted_by(c) and distinct(c)
        r = np.linalg.norm(c.astype(np.float64), axis=1)
        assert r.max() <= 1.0 + 1e-6 and r.max() > 0.999  # normalised to the unit ball
        assert np.abs(c.astype(np.float64).mean(axis=0)).max() < 1e-3  # centred
    again = synth.object_batch(1, 32, 2048)
    assert all(np.array_equal(a, b) for a, b in zip(clouds, again))
    assert not np.array_equal(clouds[0], synth.object_batch(2, 1, 2048)[0])


def test_slab_cloud():
    for N in (8192, 32768):
        p = synth.slab_cloud(2, N)
        assert p.shape == (N, 3) and sorted_by(p) and distinct(p)
        inside = ((p >= 0) & (p <= np.array([1.0, 1.0, 0.2], dtype=np.float32))).all(axis=1)
        assert inside.mean() >= 0.95  # the uniform part; 5% are Gaussian bumps around centres in the slab
        assert np.array_equal(p, synth.slab_cloud(2, N))


def test_ragged_batch():
    clouds, Cs, Ms = synth.ragged_batch(3, 16)
    assert len(clouds) == len(Cs) == len(Ms) == 16
    for c, C, M in zip(clouds, Cs, Ms):
        N = c.shape[0]
        assert 2048 <= N <= 32768 and sorted_by(c) and distinct(c)
        assert C == N // 4 and M == max(1, int(round(N / 256)))
        assert C >= M  # every sector gets a sample
    assert len({c.shape[0] for c in clouds}) > 1  # ragged


def test_lidar_frame():
    f = synth.lidar_frame(7)
    N = f.shape[0]
    assert 0.97 * 32 * 530 <= N <= 32 * 1024 and distinct(f)
    p = f.astype(np.float64)
    rng_ = np.linalg.norm(p, axis=1)
    assert rng_.min() >= 2.0 - 1e-3 and rng_.max() <= 60.0 + 1e-3
    # emitted column by column: the azimuth never steps back by more than a
    # column, except once where it wraps from +pi to -pi
    az = np.arctan2(p[:, 1], p[:, 0])
    back = np.diff(az) < -2 * np.pi / 530 - 1e-6
    assert back.sum() <= 1 and np.all(np.diff(az)[back] < -np.pi)
    assert np.array_equal(f, synth.lidar_frame(7))


def test_orders_and_pack():
    g = synth.rng(4)
    base = synth.uniform_cloud(5, 1000)
    a = synth.approx_sort_by_axis(base, g, 0, 128)
    # bins of 128 are ordered by x; inside a bin the order is shuffled
    bins = [a[i:i + 128, 0] for i in range(0, 1000, 128)]
    assert all(bins[i].max() <= bins[i + 1].min() for i in range(len(bins) - 1))
    assert not sorted_by(a)
    s = synth.shuffled(base, synth.rng(6))
    assert sorted(map(tuple, s)) == sorted(map(tuple, base)) and not sorted_by(s)
    xyz, off = synth.pack([base, a[:300], s[:7]])
    assert off.tolist() == [0, 1000, 1300, 1307] and xyz.shape == (1307, 3)
    assert np.array_equal(xyz[1000:1300], a[:300])
    grid = synth.grid_1d(4)
    assert grid.shape == (17, 3) and grid[:, 0].tolist() == list(range(17))
