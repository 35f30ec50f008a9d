"""Pins for the CPU oracle: checks against what the paper and the mathematics
fix, independent of the oracle's own code.

Every pin is a function ``pin(L)`` taking a loaded oracle library and raising
AssertionError when the library disagrees.  ``test_oracle_pins.py`` runs them
on the real oracle; ``test_oracle_mutants.py`` runs them on copies of the
oracle with one plausible mistake planted each, and requires every mistake to
be caught by at least one pin.
"""
from __future__ import annotations

import os

import numpy as np

import oracle
from paper_2208_08795_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
INIT = np.float32(1e10)  # Algorithm 1's initial distance


# --------------------------------------------------------------------------
# independent helpers (no code shared with the oracle)
# --------------------------------------------------------------------------
def sectors(N, C, M):
    """Reading of Sec. III-B: storage-order sectors, floor boundaries."""
    lo = [(s * N) // M for s in range(M + 1)]
    off = [(s * C) // M for s in range(M + 1)]
    return lo, off


def sqdist32(P, j, q):
    """fp32 squared distances from points j (array) to point q, each product
    and sum rounded on its own: (dx*dx + dy*dy) + dz*dz."""
    d = P[j] - P[q]
    dx, dy, dz = d[..., 0], d[..., 1], d[..., 2]
    return (dx * dx + dy * dy) + dz * dz


def brute_force(P, C, M, k, start, method=0):
    """From-scratch restatement: at every step, each point's distance is the
    minimum over the 1e10 of Algorithm 1 and its distances to the earlier
    samples of its sector whose update reached it (the whole sector without
    NPDU, the window [p - k//2, p + k - k//2] with it; with method bit 2 the
    window counts the sample, [p - (k-1)//2, p + (k-1) - (k-1)//2]; with
    method bit 1 the first sample's update reaches the whole sector).  No
    running array is kept; the next sample is the lowest-index maximum."""
    kl, kr = (k // 2, k - k // 2) if not method & 2 else ((k - 1) // 2, (k - 1) - (k - 1) // 2)
    P = np.asarray(P, dtype=np.float32)
    N = P.shape[0]
    lo, off = sectors(N, C, M)
    s0 = max(s for s in range(M) if lo[s] <= start)
    r = start - lo[s0]
    out = []
    for s in range(M):
        n, c = lo[s + 1] - lo[s], off[s + 1] - off[s]
        Q = P[lo[s]:lo[s + 1]]
        sel = [min(r, n - 1)]
        while len(sel) < c:
            D = np.full(n, INIT, dtype=np.float32)
            for t, p in enumerate(sel):
                js = np.arange(n)
                if k > 0 and not (method & 1 and t == 0):
                    js = js[(js >= p - kl) & (js <= p + kr)]
                D[js] = np.minimum(D[js], sqdist32(Q, js, p))
            sel.append(int(np.argmax(D)))  # first maximum = lowest index
        out += [lo[s] + p for p in sel]
    return np.array(out, dtype=np.int32)


def grid_closed_form(m):
    """FPS order on x = 0..2^m from 0: 0, 2^m, then for each level l the odd
    multiples of 2^(m-l) in ascending order (all tie at that level)."""
    seq = [0, 1 << m]
    for l in range(1, m + 1):
        step = 1 << (m - l)
        seq += list(range(step, 1 << m, 2 * step))
    return seq


def read_golden(name):
    fields = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, _, rest = line.partition(" ")
            fields[key] = rest.split()
    N = int(fields["N"][0])
    if fields["points"] == ["grid1d"]:
        P = np.zeros((N, 3), dtype=np.float32)
        P[:, 0] = np.arange(N)
    else:
        P = np.array([float(v) for v in fields["points"]], dtype=np.float32).reshape(N, 3)
    args = {key: int(fields[key][0]) for key in ("C", "M", "k", "start")}
    args["method"] = int(fields.get("method", ["0"])[0])
    expect = np.array([int(v) for v in fields["expect"]], dtype=np.int32)
    return P, args, expect


GOLDEN_FILES = sorted(f for f in os.listdir(GOLDEN) if f.endswith(".txt"))


# --------------------------------------------------------------------------
# pins
# --------------------------------------------------------------------------
def pin_golden(L):
    """Hand-worked examples of Algorithm 1 / Sec. III-B / III-C."""
    for name in GOLDEN_FILES:
        P, a, expect = read_golden(name)
        for prec in ("f32", "f64"):
            got = oracle.afps(P, a["C"], a["M"], a["k"], a["start"], precision=prec,
                              method=a["method"], library=L)
            assert np.array_equal(got, expect), (name, prec, got, expect)


def pin_grid_closed_form(L):
    """Closed form of FPS on a 1-D integer grid, along each axis in turn;
    squared distances are exact integers, so fp32 and fp64 agree exactly."""
    for m in range(1, 9):
        expect = np.array(grid_closed_form(m), dtype=np.int32)
        for axis in range(3):
            P = np.zeros(((1 << m) + 1, 3), dtype=np.float32)
            P[:, axis] = np.arange(P.shape[0])
            for prec in ("f32", "f64"):
                got = oracle.afps(P, P.shape[0], 1, 0, 0, precision=prec, library=L)
                assert np.array_equal(got, expect), (m, axis, prec)


def pin_npdu_stride_law(L):
    """Under NPDU read literally (no first full pass), untouched points keep
    1e10 and the lowest one wins, so from start 0 a sector's first
    ceil(n/(r+1)) samples are 0, r+1, 2(r+1), ... with r = k - k//2."""
    P = synth.uniform_cloud(11, 256)
    for k in (1, 2, 4, 8, 9, 16, 31):
        for M in (1, 4):
            n = 256 // M
            r = k - k // 2
            head = -(-n // (r + 1))
            C = M * n  # sample every point
            got = oracle.afps(P, C, M, k, 0, library=L)
            for s in range(M):
                seg = got[s * n: s * n + head] - s * n
                assert np.array_equal(seg, np.arange(head) * (r + 1)), (k, M, s)


def pin_brute_force(L):
    """The oracle equals the from-scratch restatement on tiny clouds."""
    cases = [(17, 17, 1, 0, 0), (40, 20, 1, 0, 5), (40, 20, 4, 0, 0), (48, 24, 3, 4, 7),
             (64, 32, 2, 8, 0), (64, 64, 4, 2, 63), (33, 11, 5, 1, 12), (50, 30, 1, 3, 49)]
    for i, (N, C, M, k, start) in enumerate(cases):
        for axis in (0, None):
            P = synth.uniform_cloud(100 + i, N, axis)
            got = oracle.afps(P, C, M, k, start, library=L)
            ref = brute_force(P, C, M, k, start)
            assert np.array_equal(got, ref), (N, C, M, k, start, axis)


def pin_brute_force_f64(L):
    """fp64 route: on coordinates that are multiples of 1/4 below 16 every
    squared distance is exact in both fp32 and fp64, so both routes must
    equal the brute force exactly (odd and even NPDU windows included)."""
    g = np.random.Generator(np.random.PCG64(7))
    for i in range(4):
        P = (g.integers(0, 64, (48, 3)) / 4.0).astype(np.float32)
        P = P[np.unique(P, axis=0, return_index=True)[1]]
        P = P[np.argsort(P[:, 0], kind="stable")]
        for (M, k) in ((1, 0), (3, 0), (2, 4), (2, 3), (1, 5)):
            C = 3 * (P.shape[0] // 4) // M * M
            a = oracle.afps(P, C, M, k, 0, precision="f32", library=L)
            b = oracle.afps(P, C, M, k, 0, precision="f64", library=L)
            ref = brute_force(P, C, M, k, 0)
            assert np.array_equal(a, ref) and np.array_equal(b, ref), (i, M, k)


def pin_reductions(L):
    """Special cases of Sec. III-B/C: a window of 2n covers the whole sector
    (NPDU = AFPS); M = C gives exactly the sector starts ("equivalent to
    RPS"); AFPS is FPS run on each sector's sub-cloud on its own."""
    P = synth.uniform_cloud(21, 300)
    for M in (1, 3, 7):
        lo, off = sectors(300, 90, M)
        full = oracle.afps(P, 90, M, 0, 0, library=L)
        n_max = max(lo[s + 1] - lo[s] for s in range(M))
        assert np.array_equal(oracle.afps(P, 90, M, 2 * n_max, 0, library=L), full)
        for s in range(M):
            sub = oracle.afps(P[lo[s]:lo[s + 1]], off[s + 1] - off[s], 1, 0, 0, library=L)
            assert np.array_equal(full[off[s]:off[s + 1]], sub + lo[s]), (M, s)
    for start in (0, 5, 299):
        got = oracle.afps(P, 60, 60, 0, start, library=L)
        lo, _ = sectors(300, 60, 60)
        r = start - lo[start * 60 // 300]
        starts = [lo[s] + min(r, lo[s + 1] - lo[s] - 1) for s in range(60)]
        assert np.array_equal(got, np.array(starts)), start
        lo_t, off_t, first_t = oracle.sector_table(300, 60, 60, start, library=L)
        assert list(lo_t) == lo and list(first_t) == starts
    # unequal sectors: N = 10, M = 3 gives sizes 3, 3, 4; start 9 is offset 3
    # of the last sector, which the smaller sectors clip to their last point
    Q = synth.uniform_cloud(22, 10)
    assert list(oracle.sector_table(10, 3, 3, 9, library=L)[2]) == [2, 5, 9]
    assert list(oracle.afps(Q, 3, 3, 0, 9, library=L)) == [2, 5, 9]


def pin_invariants(L):
    """Distinct samples inside their own sectors, c_s per sector, and every
    non-NPDU sample is the lowest-index argmax of the fp32 distance to the
    earlier samples of its sector; the selected distances never increase."""
    for seed, (N, C, M) in enumerate([(512, 128, 1), (1000, 250, 4), (777, 300, 13)]):
        P = synth.uniform_cloud(300 + seed, N)
        got = oracle.afps(P, C, M, 0, 0, library=L)
        lo, off = sectors(N, C, M)
        assert len(set(got.tolist())) == C
        for s in range(M):
            seg = got[off[s]:off[s + 1]]
            assert ((seg >= lo[s]) & (seg < lo[s + 1])).all()
            Q = P[lo[s]:lo[s + 1]]
            loc = seg - lo[s]
            D = np.full(Q.shape[0], INIT, dtype=np.float32)
            prev = np.inf
            for t in range(1, len(loc)):
                D = np.minimum(D, sqdist32(Q, np.arange(Q.shape[0]), loc[t - 1]))
                assert int(np.argmax(D)) == loc[t], (seed, s, t)
                assert D[loc[t]] <= prev
                prev = D[loc[t]]


def pin_every_point(L):
    """C = N samples every point exactly once, each sector exactly its own
    points, for any M (also when M does not divide N)."""
    for (N, M, k) in ((7, 3, 0), (100, 7, 0), (100, 7, 4), (64, 5, 3)):
        P = synth.uniform_cloud(60 + N + M, N)
        got = oracle.afps(P, N, M, k, 0, library=L)
        assert np.array_equal(np.sort(got), np.arange(N)), (N, M, k)
        lo, off = sectors(N, N, M)
        for s in range(M):
            assert np.array_equal(np.sort(got[off[s]:off[s + 1]]), np.arange(lo[s], lo[s + 1]))


def pin_metamorphic(L):
    """Exact symmetries of the fp32 arithmetic: scaling by a power of two,
    negating a coordinate, swapping x and y leave every index unchanged."""
    P = synth.uniform_cloud(41, 400)
    for (C, M, k) in ((100, 1, 0), (100, 4, 0), (120, 8, 8)):
        base = oracle.afps(P, C, M, k, 3, library=L)
        variants = [P * np.float32(8.0), P * np.float32(0.125)]
        for ax in range(3):
            Q = P.copy()
            Q[:, ax] = -Q[:, ax]
            variants.append(Q)
        variants.append(P[:, [1, 0, 2]])
        for V in variants:
            got = oracle.afps(np.ascontiguousarray(V), C, M, k, 3, library=L)
            assert np.array_equal(got, base), (C, M, k)


def pin_errors(L):
    """Argument checks: bad sizes, bad start, and a sector with more samples
    than points (N = 8, C = 7, M = 5 gives sector 2 one point, two samples)."""
    P = synth.uniform_cloud(1, 8)
    bad = [(0, 1, 0, 0), (9, 1, 0, 0), (4, 5, 0, 0), (4, 0, 0, 0), (4, 2, -1, 0),
           (4, 2, 0, 8), (4, 2, 0, -1)]
    for (C, M, k, start) in bad:
        try:
            oracle.afps(P, C, M, k, start, library=L)
        except oracle.OracleError as e:
            assert e.code == oracle.ERR_INVALID_ARG
        else:
            raise AssertionError(("accepted", C, M, k, start))
    try:
        oracle.afps(P, 7, 5, 0, 0, library=L)
    except oracle.OracleError as e:
        assert e.code == oracle.ERR_SECTOR_TOO_SMALL
    else:
        raise AssertionError("sector too small accepted")


def pin_coverage_radius(L):
    """Coverage radius: closed form on the grid (after a full FPS level l on
    x = 0..2^m the radius is 2^(m-l-1)) and numpy brute force on a cloud."""
    m = 6
    P = synth.grid_1d(m)
    seq = grid_closed_form(m)
    for l in range(0, m):
        C = (1 << l) + 1
        r = oracle.coverage_radius(P, np.array(seq[:C]), library=L)
        assert r == 2.0 ** (m - l - 1), (l, r)
    Q = synth.uniform_cloud(5, 300).astype(np.float64)
    idx = np.array([0, 17, 99, 150, 299])
    d = ((Q[:, None, :] - Q[None, idx, :]) ** 2).sum(-1)
    ref = float(np.sqrt(d.min(axis=1).max()))
    got = oracle.coverage_radius(Q.astype(np.float32), idx, library=L)
    assert abs(got - ref) <= 1e-12 * ref, (got, ref)


def pin_npdu_readings(L):
    """The other NPDU readings: a window that counts the sample with k + 1
    equals the default window with k; a full first pass with a window of 2n
    equals AFPS; both agree with the brute force restatement."""
    P = synth.uniform_cloud(31, 200)
    for k in (1, 2, 3, 8, 9, 16):
        for M in (1, 4):
            a = oracle.afps(P, 80, M, k, 0, library=L)
            b = oracle.afps(P, 80, M, k + 1, 0, method=oracle.NPDU_WINDOW_HAS_SAMPLE, library=L)
            assert np.array_equal(a, b), (k, M)
    full = oracle.afps(P, 80, 4, 0, 0, library=L)
    assert np.array_equal(oracle.afps(P, 80, 4, 400, 0, method=1, library=L), full)
    cases = [(40, 20, 1, 2, 0), (48, 24, 3, 4, 7), (64, 32, 2, 5, 3), (33, 11, 5, 1, 12)]
    for i, (N, C, M, k, start) in enumerate(cases):
        Q = synth.uniform_cloud(500 + i, N)
        for method in (1, 2, 3):
            got = oracle.afps(Q, C, M, k, start, method=method, library=L)
            assert np.array_equal(got, brute_force(Q, C, M, k, start, method)), (i, method)
            got64 = oracle.afps(Q, C, M, k, start, method=method, precision="f64", library=L)
            assert np.mean(got64 == got) > 0.5


def pin_chain_grid(L):
    """Chained levels on the grid 0..64: FPS with 2^l + 1 samples takes the
    multiples of 2^(6-l); sorted ascending they form the next, coarser grid,
    whose FPS order is the closed form scaled by the spacing."""
    P = synth.grid_1d(6)
    levels = [33, 17, 9, 5]
    got = oracle.chain(P, levels, 1, 0, library=L)
    for j, C in enumerate(levels):
        m = 5 - j  # the level-j cloud is a grid 0..2^(m+1) with spacing 2^j
        expect = [(1 << j) * v for v in grid_closed_form(m + 1)][:C]
        assert list(got[j]) == expect, (j, list(got[j]), expect)


def pin_ball_query(L):
    """Ball query: closed form on the integer grid (radius 2.5 holds the
    points i-2 .. i+2), and a vectorised numpy restatement on clouds."""
    P = np.zeros((50, 3), dtype=np.float32)
    P[:, 0] = np.arange(50)
    cen = np.array([0, 1, 10, 48, 49])
    got = oracle.ball_query(P, cen, 2.5, 6, library=L)
    for row, i in zip(got, cen):
        near = [j for j in range(i - 2, i + 3) if 0 <= j < 50]
        assert list(row) == near + [near[0]] * (6 - len(near)), (i, row)
    got = oracle.ball_query(P, cen, 2.5, 3, library=L)
    assert [list(r) for r in got] == [[0, 1, 2], [0, 1, 2], [8, 9, 10], [46, 47, 48], [47, 48, 49]]
    # radius exactly 2: the points at distance 2 lie on the sphere and are excluded
    got = oracle.ball_query(P, np.array([10]), 2.0, 4, library=L)
    assert list(got[0]) == [9, 10, 11, 9]
    for seed, (N, C, r, K) in enumerate([(500, 40, 0.15, 16), (300, 30, 0.3, 64), (200, 10, 0.02, 8)]):
        Q = synth.uniform_cloud(700 + seed, N, None)
        cen = np.arange(0, N, N // C)[:C]
        got = oracle.ball_query(Q, cen, r, K, library=L)
        r2 = np.float32(r) * np.float32(r)
        for row, c in zip(got, cen):
            d = Q - Q[c]
            d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
            hit = np.nonzero(d2 < r2)[0][:K]
            want = list(hit) + [hit[0]] * (K - len(hit)) if len(hit) else [-1] * K
            assert list(row) == want, (seed, c)


def knn_grid_closed_form(n, i, K):
    """Nearest-first order on the integer grid 0..n-1 from point i: i, then
    i-1, i+1, i-2, i+2, ... (the lower index first at equal distance),
    skipping points off the grid."""
    order = [i]
    for r in range(1, n):
        order += [j for j in (i - r, i + r) if 0 <= j < n]
    return order[:K]


def knn_brute_force(P, c, K):
    """Pure-Python loops with float32 scalars: the key (distance, index) of
    every point, sorted, the first K."""
    f = np.float32
    cx, cy, cz = (f(v) for v in P[c])
    keys = []
    for j in range(P.shape[0]):
        ex, ey, ez = f(P[j, 0]) - cx, f(P[j, 1]) - cy, f(P[j, 2]) - cz
        keys.append((f(f(ex * ex) + f(ey * ey)) + f(ez * ez), j))
    return [j for _, j in sorted(keys)[:K]]


def pin_knn(L):
    """k nearest neighbours: the closed form on an integer grid (ties to the
    lower index), brute force on small clouds, invariants (K = N is a
    permutation sorted by distance, the returned distances recompute), exact
    metamorphic scaling, and the argument checks."""
    P = np.zeros((40, 3), dtype=np.float32)
    P[:, 0] = np.arange(40)
    cen = np.array([0, 1, 17, 38, 39])
    for K in (1, 2, 5, 9, 40):
        got = oracle.knn(P, cen, K, library=L)
        for row, i in zip(got, cen):
            assert list(row) == knn_grid_closed_form(40, int(i), K), (K, i, list(row))
    for seed, (N, C, K) in enumerate([(60, 7, 5), (33, 33, 33), (90, 5, 17)]):
        Q = synth.uniform_cloud(900 + seed, N, None)
        if seed == 1:
            Q[5] = Q[20]  # a duplicate point: equal keys resolve by index
        cen = np.arange(0, N, max(1, N // C))[:C]
        got, d2 = oracle.knn(Q, cen, K, library=L, with_d2=True)
        for row, c in zip(got, cen):
            assert list(row) == knn_brute_force(Q, int(c), K), (seed, c)
        for row, dd, c in zip(got, d2, cen):
            e = Q[row] - Q[c]
            assert np.array_equal(dd, (e[:, 0] * e[:, 0] + e[:, 1] * e[:, 1]) + e[:, 2] * e[:, 2])
            key = list(zip(dd.tolist(), row.tolist()))
            assert key == sorted(key)
        if K == N:
            assert all(sorted(r) == list(range(N)) for r in got)
        assert np.array_equal(oracle.knn(Q * np.float32(8.0), cen, K, library=L), got)
    for bad in ((P, [0], 0), (P, [0], 41), (P, [40], 3), (P, [-1], 3)):
        try:
            oracle.knn(*bad, library=L)
        except oracle.OracleError:
            continue
        raise AssertionError(f"accepted {bad[1:]}")


PINS = [pin_golden, pin_grid_closed_form, pin_npdu_stride_law, pin_brute_force,
        pin_brute_force_f64, pin_reductions, pin_invariants, pin_every_point, pin_metamorphic,
        pin_errors, pin_coverage_radius, pin_chain_grid, pin_npdu_readings, pin_ball_query,
        pin_knn]
