"""Seeded synthetic point clouds shaped like the paper's workloads.

This module holds no sampling arithmetic: it only draws points (numpy PCG64)
and puts them in storage order.  It is the one module that both the oracle
tests and the CUDA tests / benchmark use for inputs.

The paper evaluates on ShapeNet / ModelNet40 / S3DIS inputs of shape
(24, 1024..4096, 3) (Table I) and on single clouds of 1K-32K points
(Sec. IV-C, Table IV).  Those datasets are not available; the generators below
stand in for them with the same sizes and with the storage orders the method
relies on (Sec. III-A): exactly sorted along x, approximately sorted in bins
of 128 points (the footnote of Sec. IV-B), or emitted column by column like a
spinning LiDAR (approximately sorted by azimuth).

Every generator returns float32 arrays of shape (N, 3) whose rows are
pairwise distinct, so that the sample indices of FPS are distinct too.
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


# --------------------------------------------------------------------------
# storage order
# --------------------------------------------------------------------------
def sort_by_axis(pts: np.ndarray, axis: int = 0) -> np.ndarray:
    """Exact ascending sort along one coordinate (stable: ties keep order)."""
    order = np.argsort(pts[:, axis], kind="stable")
    return np.ascontiguousarray(pts[order])


def approx_sort_by_axis(pts: np.ndarray, g: np.random.Generator, axis: int = 0,
                        bin_size: int = 128) -> np.ndarray:
    """Approximate sort: bins of ``bin_size`` consecutive points are ordered
    by the key, points inside a bin are shuffled (footnote of Sec. IV-B)."""
    s = sort_by_axis(pts, axis)
    out = s.copy()
    for b0 in range(0, s.shape[0], bin_size):
        seg = s[b0:b0 + bin_size]
        out[b0:b0 + bin_size] = seg[g.permutation(seg.shape[0])]
    return out


def shuffled(pts: np.ndarray, g: np.random.Generator) -> np.ndarray:
    """Unsorted storage order (a random permutation)."""
    return np.ascontiguousarray(pts[g.permutation(pts.shape[0])])


def _distinct(pts: np.ndarray) -> bool:
    return np.unique(pts, axis=0).shape[0] == pts.shape[0]


def _finish(pts: np.ndarray, axis: int | None = 0) -> np.ndarray:
    p = np.ascontiguousarray(pts, dtype=np.float32)
    if axis is not None:
        p = sort_by_axis(p, axis)
    if not _distinct(p):
        raise RuntimeError("generator produced duplicate points; change the seed")
    return p


# --------------------------------------------------------------------------
# surfaces
# --------------------------------------------------------------------------
def sphere_surface(g: np.random.Generator, n: int) -> np.ndarray:
    """Uniform on the unit sphere: normalised Gaussian vectors."""
    v = g.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def torus_surface(g: np.random.Generator, n: int, R: float = 0.5,
                  r: float = 0.1) -> np.ndarray:
    """Uniform on a torus surface (axis z): area-weighted rejection in the
    tube angle."""
    out = np.empty((0, 3))
    while out.shape[0] < n:
        m = 2 * (n - out.shape[0]) + 16
        u = g.uniform(0.0, 2 * np.pi, m)
        v = g.uniform(0.0, 2 * np.pi, m)
        keep = g.uniform(0.0, 1.0, m) < (R + r * np.cos(v)) / (R + r)
        u, v = u[keep], v[keep]
        pts = np.stack([(R + r * np.cos(v)) * np.cos(u),
                        (R + r * np.cos(v)) * np.sin(u),
                        r * np.sin(v)], axis=1)
        out = np.concatenate([out, pts])
    return out[:n]


def box_surface(g: np.random.Generator, n: int, ext) -> np.ndarray:
    """Uniform on the surface of an axis-aligned box with half-extents ext."""
    a, b, c = ext
    areas = np.array([b * c, b * c, a * c, a * c, a * b, a * b])
    face = g.choice(6, size=n, p=areas / areas.sum())
    uv = g.uniform(-1.0, 1.0, (n, 2))
    p = np.empty((n, 3))
    for f in range(6):
        m = face == f
        ax = f // 2
        sgn = 1.0 if f % 2 == 0 else -1.0
        others = [i for i in range(3) if i != ax]
        p[m, ax] = sgn * ext[ax]
        p[m, others[0]] = uv[m, 0] * ext[others[0]]
        p[m, others[1]] = uv[m, 1] * ext[others[1]]
    return p


def cylinder_surface(g: np.random.Generator, n: int, radius: float,
                     half_h: float) -> np.ndarray:
    """Uniform on a closed cylinder (side + caps), axis z."""
    side = 2 * np.pi * radius * 2 * half_h
    cap = np.pi * radius * radius
    part = g.choice(3, size=n, p=np.array([side, cap, cap]) / (side + 2 * cap))
    th = g.uniform(0.0, 2 * np.pi, n)
    p = np.empty((n, 3))
    s = part == 0
    p[s, 0] = radius * np.cos(th[s])
    p[s, 1] = radius * np.sin(th[s])
    p[s, 2] = g.uniform(-half_h, half_h, s.sum())
    for code, z in ((1, half_h), (2, -half_h)):
        m = part == code
        rr = radius * np.sqrt(g.uniform(0.0, 1.0, m.sum()))
        p[m, 0] = rr * np.cos(th[m])
        p[m, 1] = rr * np.sin(th[m])
        p[m, 2] = z
    return p


def _rotation(g: np.random.Generator) -> np.ndarray:
    q, r = np.linalg.qr(g.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


# --------------------------------------------------------------------------
# the workloads
# --------------------------------------------------------------------------
def sphere_torus_cloud(seed: int = 0, n_sphere: int = 1024, n_torus: int = 1024) -> np.ndarray:
    """Single object-scale cloud: uniform on the unit sphere plus uniform on a
    torus of tube radius 0.1 (major radius 0.5), sorted ascending by x."""
    g = rng(seed)
    pts = np.concatenate([sphere_surface(g, n_sphere), torus_surface(g, n_torus)])
    return _finish(pts, 0)


def primitives_cloud(g: np.random.Generator, n: int, axis: int | None = 0) -> np.ndarray:
    """Object-scale cloud: 2-5 primitive surfaces (box / cylinder / sphere),
    each scaled U[0.2, 1] and placed with a random pose; Gaussian jitter
    sigma = 0.005; normalised to the unit ball; sorted along ``axis``."""
    k = int(g.integers(2, 6))
    kinds = g.integers(0, 3, k)
    scales = g.uniform(0.2, 1.0, k)
    weights = g.uniform(0.5, 1.5, k) * scales ** 2
    counts = np.floor(n * weights / weights.sum()).astype(int)
    counts[0] += n - counts.sum()
    parts = []
    for kind, s, c in zip(kinds, scales, counts):
        if kind == 0:
            p = box_surface(g, c, s * g.uniform(0.3, 1.0, 3))
        elif kind == 1:
            p = cylinder_surface(g, c, s * g.uniform(0.2, 0.6), s * g.uniform(0.3, 1.0))
        else:
            p = s * sphere_surface(g, c)
        p = p @ _rotation(g).T + g.uniform(-0.6, 0.6, 3)
        parts.append(p)
    pts = np.concatenate(parts)
    pts = pts + g.normal(0.0, 0.005, pts.shape)
    pts = pts - pts.mean(axis=0)
    pts = pts / np.linalg.norm(pts, axis=1).max()
    return _finish(pts, axis)


def object_batch(seed: int = 1, B: int = 32, N: int = 2048):
    """B object-scale clouds of N points each (the part-segmentation input
    shape of Table I, batch raised from 24 to 32)."""
    g = rng(seed)
    return [primitives_cloud(g, N) for _ in range(B)]


def slab_cloud(seed: int, N: int, bump_frac: float = 0.05, n_bumps: int = 12) -> np.ndarray:
    """Large scene-like cloud: uniform in a 1 x 1 x 0.2 slab, with a fraction
    of the points drawn from Gaussian density bumps; sorted by x."""
    g = rng(seed)
    nb = int(round(N * bump_frac))
    nu = N - nb
    lo = np.array([0.0, 0.0, 0.0])
    hi = np.array([1.0, 1.0, 0.2])
    uni = g.uniform(lo, hi, (nu, 3))
    centres = g.uniform(lo, hi, (n_bumps, 3))
    which = g.integers(0, n_bumps, nb)
    bumps = centres[which] + g.normal(0.0, 0.02, (nb, 3))
    return _finish(np.concatenate([uni, bumps]), 0)


def ragged_batch(seed: int = 3, B: int = 256, n_lo: int = 2048, n_hi: int = 32768,
                 sector_points: int = 256):
    """Ragged batch of object-scale clouds, N ~ U[n_lo, n_hi]; per cloud
    C = floor(N/4) and M = max(1, round(N / sector_points)).
    Returns (clouds, C list, M list)."""
    g = rng(seed)
    Ns = g.integers(n_lo, n_hi + 1, B)
    clouds = [primitives_cloud(g, int(n)) for n in Ns]
    Cs = [int(n) // 4 for n in Ns]
    Ms = [max(1, int(round(int(n) / sector_points))) for n in Ns]
    return clouds, Cs, Ms


def lidar_frame(seed: int, rings: int = 32, cols_lo: int = 530, cols_hi: int = 1024,
                r_lo: float = 2.0, r_hi: float = 60.0, dropout: float = 0.02) -> np.ndarray:
    """Spinning-LiDAR-like frame: ``rings`` beams swept in azimuth, a random
    range per return in [r_lo, r_hi] m, ``dropout`` of the returns missing.
    Points are emitted column by column, so the frame is approximately sorted
    by azimuth (one bin per column), as in Fig. 2(a) of the paper."""
    g = rng(seed)
    cols = int(g.integers(cols_lo, cols_hi + 1))
    elev = np.deg2rad(np.linspace(-25.0, 15.0, rings))
    az = np.linspace(-np.pi, np.pi, cols, endpoint=False)
    az = az + g.uniform(0.0, 2 * np.pi / cols, cols)  # jittered firing times
    A = np.repeat(az, rings)
    E = np.tile(elev, cols)
    Rg = g.uniform(r_lo, r_hi, A.size)
    keep = g.uniform(0.0, 1.0, A.size) >= dropout
    pts = np.stack([Rg * np.cos(E) * np.cos(A), Rg * np.cos(E) * np.sin(A),
                    Rg * np.sin(E)], axis=1)[keep]
    return _finish(pts, None)


# --------------------------------------------------------------------------
# small clouds for tests
# --------------------------------------------------------------------------
def uniform_cloud(seed: int, N: int, axis: int | None = 0) -> np.ndarray:
    """N points uniform in the unit cube, sorted along ``axis`` (None: as drawn)."""
    g = rng(seed)
    return _finish(g.uniform(0.0, 1.0, (N, 3)), axis)


def grid_1d(m: int) -> np.ndarray:
    """2**m + 1 points at x = 0, 1, ..., 2**m on the x axis."""
    n = (1 << m) + 1
    p = np.zeros((n, 3), dtype=np.float32)
    p[:, 0] = np.arange(n, dtype=np.float32)
    return p


# --------------------------------------------------------------------------
# batching helper
# --------------------------------------------------------------------------
def pack(clouds):
    """Concatenate clouds; returns (xyz (sum N, 3) float32, pt_off int64 (B+1))."""
    sizes = np.array([c.shape[0] for c in clouds], dtype=np.int64)
    off = np.zeros(len(clouds) + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    xyz = np.ascontiguousarray(np.concatenate(clouds).astype(np.float32, copy=False))
    return xyz, off
