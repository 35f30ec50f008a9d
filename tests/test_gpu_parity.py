"""CUDA path vs the FP32 oracle, element by element (int32 indices must be
bit-identical), on seeded synthetic clouds shaped like the paper's workloads
and on the method's edge cases.  Every call goes through the C ABI."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2208_08795_gb300 import afps as B
from paper_2208_08795_gb300 import build as build_mod
from paper_2208_08795_gb300 import synth

pytestmark = pytest.mark.gpu


def k_rule(M):
    """NPDU window per sector count (Sec. IV-D: k = 8 for M <= 8, 16 for M >= 16)."""
    return 8 if M <= 8 else 16


@pytest.fixture(scope="module")
def S():
    build_mod.build()
    s = B.Sampler(0)
    yield s
    s.close()


def gpu_one(S, pts, C, M, k, start=0):
    x = torch.from_numpy(np.ascontiguousarray(pts)).cuda()
    out = S.sample(x, C, M, k, start)
    S.sync()
    return out.cpu().numpy()


def gpu_batch(S, clouds, C, M, k, start=0):
    xyz, off = synth.pack(clouds)
    x = torch.from_numpy(xyz).cuda()
    ba = B.BatchArgs(off, C, M, k, start)
    out = S.sample_batched(x, ba)
    S.sync()
    o = out.cpu().numpy()
    return [o[ba.out_off[b]:ba.out_off[b + 1]] for b in range(ba.B)], ba


def assert_same(got, ref, what=""):
    got, ref = np.asarray(got), np.asarray(ref)
    assert got.shape == ref.shape, (what, got.shape, ref.shape)
    if not np.array_equal(got, ref):
        i = int(np.nonzero(got != ref)[0][0])
        raise AssertionError(f"{what}: first mismatch at {i}: gpu {got[i]} oracle {ref[i]}")


# --------------------------------------------------------------- workloads
@pytest.mark.parametrize("M,k", [(1, 0), (4, 0), (4, 8), (32, 16)])
def test_sphere_torus_2048(S, M, k):
    P = synth.sphere_torus_cloud(0)
    assert_same(gpu_one(S, P, 512, M, k), oracle.afps(P, 512, M, k), f"M={M} k={k}")


@pytest.fixture(scope="module")
def objects():
    return synth.object_batch(1, 32, 2048)


@pytest.mark.parametrize("M", [1, 4, 16, 32])
@pytest.mark.parametrize("npdu", [False, True])
def test_object_batch_32x2048(S, objects, M, npdu):
    k = k_rule(M) if npdu else 0
    got, _ = gpu_batch(S, objects, 512, M, k)
    for b, P in enumerate(objects):
        assert_same(got[b], oracle.afps(P, 512, M, k), f"cloud {b} M={M} k={k}")


@pytest.mark.parametrize("N", [8192, 16384, 32768])
@pytest.mark.parametrize("M,npdu", [(1, False), (1, True), (8, True), (32, True), (64, True),
                                    (128, True)])
def test_slab_large(S, N, M, npdu):
    P = synth.slab_cloud(2, N)
    k = k_rule(M) if npdu else 0
    assert_same(gpu_one(S, P, N // 4, M, k), oracle.afps(P, N // 4, M, k), f"N={N} M={M} k={k}")


@pytest.mark.parametrize("npdu", [False, True])
def test_ragged_batch_256(S, npdu):
    clouds, Cs, Ms = synth.ragged_batch(3, 256)
    ks = [k_rule(m) if npdu else 0 for m in Ms]
    got, ba = gpu_batch(S, clouds, Cs, Ms, ks)
    for b, P in enumerate(clouds):
        assert_same(got[b], oracle.afps(P, Cs[b], Ms[b], ks[b]), f"cloud {b}")
    if npdu:  # every sector of the batch in one launch of the window kernel
        plan = S.describe_batched(ba)
        assert plan.startswith("win ") and ";" not in plan and plan.endswith("items=17576"), plan


# --------------------------------------------------------------- edge cases
EDGE = [
    (1, 1, 1, 0, 0), (2, 2, 1, 0, 1), (2, 2, 2, 3, 1), (5, 3, 1, 1, 4), (31, 31, 1, 0, 30),
    (33, 10, 3, 0, 32), (100, 100, 7, 0, 0), (100, 100, 7, 4, 99), (64, 64, 64, 0, 0),
    (300, 40, 40, 2, 150), (513, 100, 1, 0, 0), (513, 100, 1, 5, 512), (1000, 250, 3, 1, 999),
    (4097, 600, 1, 0, 17), (8193, 300, 1, 0, 8192), (5000, 1000, 4, 7, 2500),
    (2048, 512, 16, 3000, 0), (777, 300, 13, 0, 5), (1030, 1030, 2, 0, 0),
]


@pytest.mark.parametrize("N,C,M,k,start", EDGE)
def test_edge_cases(S, N, C, M, k, start):
    P = synth.uniform_cloud(1000 + N + M + k, N)
    assert_same(gpu_one(S, P, C, M, k, start), oracle.afps(P, C, M, k, start), str((N, C, M, k, start)))


def test_max_sector(S):
    N = B.AFPS_MAX_SECTOR_POINTS
    P = synth.slab_cloud(9, N)
    assert_same(gpu_one(S, P, 48, 1, 0, 12345), oracle.afps(P, 48, 1, 0, 12345), "max sector")


def test_unsorted_and_duplicates(S):
    P = synth.uniform_cloud(5, 700, axis=None)
    assert_same(gpu_one(S, P, 200, 5, 6, 3), oracle.afps(P, 200, 5, 6, 3), "unsorted")
    Q = np.repeat(synth.uniform_cloud(6, 40), 3, axis=0)  # every point three times
    assert_same(gpu_one(S, Q, 120, 2, 0, 0), oracle.afps(Q, 120, 2, 0, 0), "duplicates")
    Z = np.zeros((96, 3), dtype=np.float32)  # all distances zero
    assert_same(gpu_one(S, Z, 96, 3, 0, 5), oracle.afps(Z, 96, 3, 0, 5), "all equal")


@pytest.mark.parametrize("shift", [1, 2, 3, 5])
def test_unaligned_base(S, shift):
    """Clouds starting at every 4-byte phase exercise the bulk copy's head and
    tail handling."""
    N = 3000
    P = synth.uniform_cloud(77, N)
    buf = torch.zeros(3 * N + 16, dtype=torch.float32, device="cuda")
    view = buf[shift:shift + 3 * N].view(N, 3)
    view.copy_(torch.from_numpy(P).cuda())
    for (C, M, k) in ((300, 1, 0), (300, 10, 0), (600, 30, 16)):
        out = S.sample(view, C, M, k, 7)
        S.sync()
        assert_same(out.cpu().numpy(), oracle.afps(P, C, M, k, 7), f"shift={shift} M={M}")


def test_errors(S):
    P = torch.from_numpy(synth.uniform_cloud(1, 64)).cuda()
    bad = [(0, 1, 0, 0, B.AFPS_ERR_INVALID_ARG), (65, 1, 0, 0, B.AFPS_ERR_INVALID_ARG),
           (8, 9, 0, 0, B.AFPS_ERR_INVALID_ARG), (8, 2, -1, 0, B.AFPS_ERR_INVALID_ARG),
           (8, 2, 0, 64, B.AFPS_ERR_INVALID_ARG)]
    for C, M, k, start, code in bad:
        with pytest.raises(B.AfpsError) as ei:
            S.sample(P, C, M, k, start, out=torch.empty(max(C, 1), dtype=torch.int32, device="cuda"))
        assert ei.value.code == code
    Q = torch.from_numpy(synth.uniform_cloud(2, 8)).cuda()
    with pytest.raises(B.AfpsError) as ei:
        S.sample(Q, 7, 5, 0, 0)
    assert ei.value.code == B.AFPS_ERR_SECTOR_TOO_SMALL
    big = torch.zeros((B.AFPS_MAX_SECTOR_POINTS + 1, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(B.AfpsError) as ei:
        S.sample(big, 4, 1, 0, 0)
    assert ei.value.code == B.AFPS_ERR_UNSUPPORTED
    S.sync()


# --------------------------------------------------------------- variants
def pow2(n):
    b = 1
    while b < n:
        b <<= 1
    return b


VARIANTS = [  # (N, C, M, k, kind, P, W, CS)
    (1024, 256, 4, 0, 1, 2, 4, 1), (1024, 256, 4, 0, 1, 4, 2, 1), (1024, 256, 4, 0, 1, 8, 1, 1),
    (1024, 256, 4, 0, 1, 2, 2, 2), (1024, 256, 4, 0, 1, 2, 1, 4), (1024, 256, 4, 8, 1, 2, 2, 2),
    (4096, 512, 1, 0, 1, 4, 2, 16), (4096, 512, 1, 0, 1, 8, 4, 4), (4096, 512, 1, 16, 1, 8, 2, 8),
    (10000, 700, 1, 0, 1, 8, 32, 2), (10000, 700, 1, 0, 1, 4, 8, 10), (10000, 700, 1, 5, 1, 8, 16, 3),
    (3000, 300, 10, 0, 0, 12, 1, 1), (3000, 300, 10, 0, 0, 16, 8, 1), (3000, 300, 10, 9, 0, 12, 2, 1),
    (640, 640, 20, 0, 0, 1, 8, 1), (640, 640, 20, 0, 0, 2, 4, 1), (640, 640, 20, 16, 0, 1, 8, 1),
    (2000, 400, 100, 4, 0, 1, 4, 1), (2000, 500, 8, 0, 0, 8, 8, 1), (2000, 500, 8, 12, 0, 8, 4, 1),
    (5000, 1000, 6, 0, 0, 32, 2, 1), (5000, 1000, 6, 16, 0, 32, 4, 1, 1),
    (4000, 800, 6, 16, 0, 24, 4, 1), (4000, 800, 6, 9, 0, 24, 2, 1, 1),
    (3000, 600, 4, 16, 1, 4, 8, 1, 1), (20000, 2000, 2, 8, 1, 8, 8, 5, 1),
    # window kernel (NPDU only): P = rows of 32 points per warp buffer; one,
    # two, four and eight row-maximum slots per lane; windows narrower and
    # wider than a row; every point sampled
    (3000, 300, 10, 9, 2, 10, 4, 1), (3000, 300, 10, 16, 2, 16, 2, 1),
    (2000, 1000, 2, 16, 2, 32, 1, 1), (2100, 500, 2, 16, 2, 33, 2, 1),
    (20000, 4000, 4, 8, 2, 157, 1, 1), (8192, 2048, 1, 8, 2, 256, 1, 1),
    (640, 640, 20, 16, 2, 1, 8, 1), (4000, 1500, 8, 70, 2, 16, 8, 1),
    (3000, 900, 3, 1, 2, 40, 2, 1),
    # the window kernel's lean round form (skip = 1): one and two row-maximum
    # slots, windows within and across rows, the widest sector
    (3000, 300, 10, 9, 2, 10, 4, 1, 1), (2100, 500, 2, 16, 2, 33, 2, 1, 1),
    (640, 640, 20, 16, 2, 1, 8, 1, 1), (8192, 2048, 1, 8, 2, 256, 1, 1, 1),
    (3000, 900, 3, 1, 2, 40, 2, 1, 1),
    # the pair kernel (two sectors per warp, 16-point rows; windows of at most
    # 17 points): one to eight row-maximum slots, an odd number of sectors
    # (the last pair's second half empty), every point sampled
    (3000, 300, 10, 9, 3, 19, 4, 1), (3000, 300, 10, 16, 3, 32, 2, 1),
    (2000, 1000, 2, 16, 3, 63, 1, 1), (640, 640, 20, 16, 3, 2, 8, 1),
    (8192, 1024, 4, 8, 3, 128, 1, 1), (2100, 500, 2, 1, 3, 66, 2, 1),
    (3000, 300, 3, 16, 3, 63, 2, 1),
]


@pytest.mark.parametrize("row", VARIANTS, ids=[str(r) for r in VARIANTS])
def test_forced_variant(tmp_path, row):
    """Pin one kernel variant through the tuning cache and compare."""
    N, C, M, k, kind, Pp, W, CS = row[:8]
    skip = row[8] if len(row) > 8 else 0
    build_mod.build()
    n_max = -(-N // M)
    c_max = -(-C // M)
    key = f"{'npdu' if k else 'full'}:n{n_max}:c{c_max}:i{pow2(M)}"
    path = tmp_path / "tune.txt"
    path.write_text(f"{key} {kind} {Pp} {W} {CS} 0 {skip}\n")
    s = B.Sampler(0, tune_cache=str(path))
    try:
        desc = s.describe_plan(n_max, c_max, k, M)
        if kind == 0:
            want = f"warp P={Pp} W={W}"
        elif kind == 2:
            want = f"win P={Pp} W={W}"
        elif kind == 3:
            want = f"pair P={Pp} W={W}"
        elif CS > 1:
            want = f"cluster P={Pp} W={W} CS={CS}"
        else:
            want = f"cta P={Pp} W={W}"
        if skip:
            want += " lean" if kind == 2 else " skip"
        P = synth.uniform_cloud(N + 31 * M + k, N)
        x = torch.from_numpy(P).cuda()
        out = s.sample(x, C, M, k, 1)
        s.sync()
        assert_same(out.cpu().numpy(), oracle.afps(P, C, M, k, 1), f"{key} -> {desc}")
        assert desc == want, (desc, want)
    finally:
        s.close()


@pytest.mark.parametrize("N", [2048, 8192, 32768])
@pytest.mark.parametrize("M,k", [(1, 0), (1, 8), (32, 0), (32, 16)])
def test_table_iv_sizes(S, N, M, k):
    """The benchmark's Table IV sweep: single slab clouds, C = 512."""
    P = synth.slab_cloud(2, N)
    assert_same(gpu_one(S, P, 512, M, k), oracle.afps(P, 512, M, k), f"N={N} M={M} k={k}")


# --------------------------------------------------------------- NPDU stride phase
# Under the literal NPDU reading (distances start at 1e10) the first samples of
# a sector started at offset r <= floor(k/2) are r, r + q, r + 2q, ... with
# q = k - floor(k/2) + 1, until a window reaches the sector's end; the kernels
# apply those windows at once and skip the argmax rounds whose outcome that
# fixes, unless a windowed distance reaches 1e10 (then they run the serial
# loop from the start).  The cases put the number of samples on either side
# of the stride's length, on a 32-sample row boundary, with starts inside and
# outside the half window, the other window reading, and coordinates far
# enough apart to reach 1e10.
STRIDE_KERNELS = [(0, 2, 4, 1), (0, 8, 2, 1), (1, 2, 8, 1), (1, 8, 4, 1), (1, 16, 8, 1),
                  (1, 4, 8, 4), (1, 16, 4, 2),  # these two: thread-block clusters
                  (2, 9, 4, 1), (2, 40, 2, 1),  # window kernel, one and two slots per lane
                  (2, 9, 4, 1, 1), (2, 40, 2, 1, 1),  # ... and its lean round form
                  (3, 19, 4, 1), (3, 63, 2, 1)]  # pair kernel, 16-point rows


def stride_len(n, k, r, method=0):
    kl, kr = ((k - 1) // 2, (k - 1) - (k - 1) // 2) if method == 2 else (k // 2, k - k // 2)
    x = n - 1 - kr - r
    return 1 if x <= 0 else (x + kr) // (kr + 1) + 1


def stride_cases(n):
    ts = stride_len(n, 16, 0)
    rows = [(16, 0, 0, max(1, ts - 1), 1.0), (16, 0, 0, ts, 1.0), (16, 0, 3, ts + 1, 1.0),
            (16, 0, 8, min(n, stride_len(n, 16, 8) + 40), 1.0),
            (16, 0, 9, min(n, ts + 5), 1.0), (8, 2, 1, min(n, 2 * stride_len(n, 8, 1, 2)), 1.0),
            (16, 0, 0, min(n, ts + 7), 3e5), (2, 0, 1, n, 1.0), (16, 0, 0, 1, 1.0)]
    # a stride of exactly 32 samples ends on a row boundary: n = 31 q + kr + 1
    if n >= 288:
        rows.append((16, 0, 0, 40, 1.0))
    return rows


@pytest.mark.parametrize("kern", STRIDE_KERNELS, ids=[str(k) for k in STRIDE_KERNELS])
def test_npdu_stride_phase(tmp_path, kern):
    kind, Pp, W, CS = kern[:4]
    lean = kern[4] if len(kern) > 4 else 0
    build_mod.build()
    cap = 32 * W * Pp * CS if kind == 1 else 16 * Pp if kind == 3 else 32 * Pp
    sizes = [cap - 3] + ([288] if cap >= 288 else [])
    for n in sizes:
        M = 3
        N = M * n
        for (k, method, r, c, scale) in stride_cases(n):
            if n == 288 and (k, c) != (16, 40):
                continue
            C = M * c
            key = f"npdu:n{n}:c{c}:i{pow2(M)}"
            path = tmp_path / "tune.txt"
            path.write_text(f"{key} {kind} {Pp} {W} {CS} 0 {lean}\n")
            s = B.Sampler(0, tune_cache=str(path))
            try:
                P = (synth.uniform_cloud(7 * n + k + r, N) * scale).astype(np.float32)
                out = s.sample(torch.from_numpy(P).cuda(), C, M, k, r, method=method)
                s.sync()
                ref = oracle.afps(P, C, M, k, r, method=method)
                assert_same(out.cpu().numpy(), ref,
                            f"{s.describe_plan(n, c, k, M)} n={n} c={c} k={k} r={r} m={method} x{scale}")
            finally:
                s.close()


# --------------------------------------------------------------- runs of equal clouds
# A class whose clouds share N, C, M, window, reading and start and sit back
# to back (points and outputs) has its items computed in the kernel instead
# of read from a table; anything else takes the table.  Both must agree with
# the oracle, and output slots outside [out_off[b], out_off[b] + C) stay
# untouched.
def _batched(S, clouds, C, M, k, start, out_off=None, method=None):
    xyz, off = synth.pack(clouds)
    ba = B.BatchArgs(off, C, M, k, start, out_off=out_off, method=method)
    out = torch.full((ba.total_out,), -1, dtype=torch.int32, device="cuda")
    S.sample_batched(torch.from_numpy(xyz).cuda(), ba, out=out)
    S.sync()
    return out.cpu().numpy(), ba


@pytest.mark.parametrize("method", [0, 2])
def test_equal_cloud_run(S, method):
    clouds = [synth.uniform_cloud(300 + i, 1500) for i in range(40)]
    o, ba = _batched(S, clouds, 300, 12, 16, 5, method=method)
    for b, P in enumerate(clouds):
        assert_same(o[ba.out_off[b]:ba.out_off[b + 1]],
                    oracle.afps(P, 300, 12, 16, 5, method=method), f"cloud {b}")


def test_equal_clouds_with_output_gaps(S):
    clouds = [synth.uniform_cloud(400 + i, 1000) for i in range(9)]
    out_off = np.arange(10, dtype=np.int64) * (200 + 7)
    o, ba = _batched(S, clouds, 200, 4, 8, 0, out_off=out_off)
    for b, P in enumerate(clouds):
        assert_same(o[out_off[b]:out_off[b] + 200], oracle.afps(P, 200, 4, 8, 0), f"cloud {b}")
        assert np.all(o[out_off[b] + 200:out_off[b + 1]] == -1)


def test_equal_run_broken_inside_a_class(S):
    """Same sector sizes (one class) but one cloud with another C, another
    start, and one of another size class: no run, every cloud still exact."""
    clouds = [synth.uniform_cloud(500 + i, 2048) for i in range(8)] + [synth.uniform_cloud(9, 4000)]
    Cs = [512] * 8 + [800]
    Cs[3] = 480
    starts = [0] * 9
    starts[5] = 3
    o, ba = _batched(S, clouds, Cs, [32] * 8 + [8], 16, starts)
    for b, P in enumerate(clouds):
        M = 32 if b < 8 else 8
        assert_same(o[ba.out_off[b]:ba.out_off[b + 1]], oracle.afps(P, Cs[b], M, 16, starts[b]),
                    f"cloud {b}")


def test_equal_run_persistent_queue(S):
    """1200 clouds x 32 sectors: more items than resident warps, so the
    dynamic queue hands out computed items."""
    clouds = synth.object_batch(3, 1200, 2048)
    o, ba = _batched(S, clouds, 512, 32, 16, 0)
    for b in range(0, 1200, 7):
        assert_same(o[ba.out_off[b]:ba.out_off[b + 1]], oracle.afps(clouds[b], 512, 32, 16, 0),
                    f"cloud {b}")


# --------------------------------------------------------------- NPDU readings
READINGS = [(2048, 512, 32, 16), (2048, 512, 4, 8), (16384, 4096, 1, 8), (5000, 1000, 6, 9),
            (1000, 250, 3, 1), (40000, 2000, 1, 5)]


@pytest.mark.parametrize("method", [1, 2, 3])
@pytest.mark.parametrize("N,C,M,k", READINGS)
def test_npdu_readings(S, N, C, M, k, method):
    """The other readings of the NPDU window, on warp, CTA and cluster paths."""
    P = synth.uniform_cloud(N + method, N)
    x = torch.from_numpy(P).cuda()
    out = S.sample(x, C, M, k, 3, method=method)
    S.sync()
    assert_same(out.cpu().numpy(), oracle.afps(P, C, M, k, 3, method=method), f"method={method}")


def test_npdu_readings_mixed_batch(S, objects):
    clouds = objects[:6]
    Ms, ks, methods = [32, 16, 4, 1, 32, 8], [16, 16, 8, 4, 1, 0], [1, 2, 3, 1, 2, 0]
    xyz, off = synth.pack(clouds)
    ba = B.BatchArgs(off, 512, Ms, ks, 0, method=methods)
    out = S.sample_batched(torch.from_numpy(xyz).cuda(), ba)
    S.sync()
    o = out.cpu().numpy()
    for b, P in enumerate(clouds):
        ref = oracle.afps(P, 512, Ms[b], ks[b], 0, method=methods[b])
        assert_same(o[ba.out_off[b]:ba.out_off[b + 1]], ref, f"cloud {b}")


# --------------------------------------------------------------- batching
def test_graph_replay_and_launch_count(objects):
    build_mod.build()
    s = B.Sampler(0, graph=True)
    try:
        xyz, off = synth.pack(objects)
        x = torch.from_numpy(xyz).cuda()
        Ms = [32] * 16 + [4] * 8 + [1] * 8  # three launch classes in one graph
        ks = [16] * 16 + [0] * 8 + [0] * 8
        ba = B.BatchArgs(off, 512, Ms, ks, 0)
        out = torch.full((ba.total_out,), -1, dtype=torch.int32, device="cuda")
        s.sample_batched(x, ba, out=out)
        n0 = s.launch_count
        for _ in range(3):
            out.fill_(-1)
            s.sample_batched(x, ba, out=out)
        s.sync()
        assert s.launch_count - n0 == 3 * 3  # three classes, three replays
        o = out.cpu().numpy()
        for b, P in enumerate(objects):
            assert_same(o[ba.out_off[b]:ba.out_off[b + 1]], oracle.afps(P, 512, Ms[b], ks[b]), f"cloud {b}")
    finally:
        s.close()


def test_host_buffers_match_device(S, objects):
    xyz, off = synth.pack(objects[:8])
    ba = B.BatchArgs(off, 512, 16, 16, 0)
    h_xyz = torch.from_numpy(xyz).pin_memory().numpy()
    h_out = torch.full((ba.total_out,), -1, dtype=torch.int32).pin_memory().numpy()
    S.sample_batched_host(h_xyz, ba, h_out)
    for b, P in enumerate(objects[:8]):
        assert_same(h_out[ba.out_off[b]:ba.out_off[b + 1]], oracle.afps(P, 512, 16, 16), f"cloud {b}")


@pytest.mark.parametrize("graph", [False, True])
def test_host_buffers_async_pipelined(objects, graph):
    """afps_sample_batched_host_async: several calls queued back to back on
    page-locked buffers (inputs rotating over three, one output each), one
    synchronisation at the end; every output must be its own batch's."""
    build_mod.build()
    s = B.Sampler(0, graph=graph)
    try:
        sets = [objects[:8], objects[8:16], objects[16:24]]
        packs = [synth.pack(c) for c in sets]
        ba = B.BatchArgs(packs[0][1], 512, 32, 16, 0)
        hx = [torch.from_numpy(p[0]).pin_memory().numpy() for p in packs]
        ho = [torch.full((ba.total_out,), -1, dtype=torch.int32).pin_memory().numpy()
              for _ in range(12)]
        for j, o in enumerate(ho):
            s.sample_batched_host_async(hx[j % 3], ba, o)
        s.sync()
        for j, o in enumerate(ho):
            for b in (0, 7):
                assert_same(o[ba.out_off[b]:ba.out_off[b + 1]],
                            oracle.afps(sets[j % 3][b], 512, 32, 16), f"call {j} cloud {b}")
        with pytest.raises(B.AfpsError) as ei:  # pageable buffers cannot be queued
            s.sample_batched_host_async(packs[0][0], ba, np.zeros(ba.total_out, dtype=np.int32))
        assert ei.value.code == B.AFPS_ERR_INVALID_ARG
    finally:
        s.close()


def test_host_buffers_graph_replay(objects):
    """Pinned host buffers with graphs: copies and launches replay as one graph."""
    build_mod.build()
    s = B.Sampler(0, graph=True)
    try:
        xyz, off = synth.pack(objects[8:16])
        ba = B.BatchArgs(off, 512, [32, 16, 4, 1, 32, 32, 8, 2], [16, 16, 8, 0, 0, 3, 0, 0], 0)
        h_xyz = torch.from_numpy(xyz).pin_memory().numpy()
        h_out = torch.full((ba.total_out,), -1, dtype=torch.int32).pin_memory().numpy()
        n0 = s.launch_count
        for rep in range(3):
            h_out[:] = -1
            s.sample_batched_host(h_xyz, ba, h_out)
            for b, P in enumerate(objects[8:16]):
                ref = oracle.afps(P, 512, int(ba.M[b]), int(ba.k[b]))
                assert_same(h_out[ba.out_off[b]:ba.out_off[b + 1]], ref, f"rep {rep} cloud {b}")
        assert s.launch_count > n0
    finally:
        s.close()


def test_same_alone_and_in_a_mix(S, objects):
    """Each cloud's result is the same alone and inside a mixed batch."""
    clouds = objects[:6] + [synth.slab_cloud(4, 9000), synth.uniform_cloud(8, 300)]
    Cs = [512] * 6 + [2000, 100]
    Ms = [1, 4, 16, 32, 2, 8, 1, 3]
    ks = [0, 8, 16, 16, 0, 0, 0, 5]
    mixed, _ = gpu_batch(S, clouds, Cs, Ms, ks, 0)
    for b, P in enumerate(clouds):
        alone = gpu_one(S, P, Cs[b], Ms[b], ks[b], 0)
        assert_same(mixed[b], alone, f"cloud {b}")
        assert_same(alone, oracle.afps(P, Cs[b], Ms[b], ks[b]), f"cloud {b}")


def test_autotune(objects, tmp_path):
    build_mod.build()
    s = B.Sampler(0, tune_cache=str(tmp_path / "t.txt"))
    try:
        xyz, off = synth.pack(objects)
        x = torch.from_numpy(xyz).cuda()
        ba = B.BatchArgs(off, 512, 32, 16, 0)
        out = torch.full((ba.total_out,), -1, dtype=torch.int32, device="cuda")
        assert s.autotune_batched(x, ba, out) >= 1
        s.sync()
        assert B.afps_save_tuning(s.ctx, None) == 0
        assert (tmp_path / "t.txt").read_text().strip()
        o = out.cpu().numpy()
        for b, P in enumerate(objects):
            assert_same(o[ba.out_off[b]:ba.out_off[b + 1]], oracle.afps(P, 512, 32, 16), f"cloud {b}")
    finally:
        s.close()


def test_autotune_on_first_use(objects, tmp_path):
    """AFPS_FLAG_AUTOTUNE: the first batched call of a new argument set tunes
    its classes (then samples); later calls reuse the choice."""
    build_mod.build()
    path = tmp_path / "t.txt"
    s = B.Sampler(0, flags=B.AFPS_FLAG_AUTOTUNE, tune_cache=str(path))
    try:
        xyz, off = synth.pack(objects)
        x = torch.from_numpy(xyz).cuda()
        ba = B.BatchArgs(off, 512, 32, 16, 0)
        for _ in range(2):
            o = s.sample_batched(x, ba).cpu().numpy()
            for b in (0, 5, len(objects) - 1):
                assert_same(o[ba.out_off[b]:ba.out_off[b + 1]], oracle.afps(objects[b], 512, 32, 16),
                            f"cloud {b}")
        assert B.afps_save_tuning(s.ctx, None) == 0
        assert "npdu:n64:c16:i1024" in path.read_text()
    finally:
        s.close()


def test_tuning_file_names_its_device(tmp_path):
    """A saved tuning file names the GPU; a file naming another GPU is ignored,
    one naming this GPU (or none) is used."""
    build_mod.build()
    key = "npdu:n64:c16:i1024"
    forced = f"{key} 0 2 8 1 0 1\n"
    path = tmp_path / "t.txt"
    s = B.Sampler(0, tune_cache=str(path))
    try:
        default = s.describe_plan(64, 16, 16, 1024)
        assert default != "warp P=2 W=8 skip"  # the untuned choice differs from the forced one
        assert B.afps_save_tuning(s.ctx, None) == 0
        header = path.read_text().splitlines()[0]
        assert header.startswith("# device ") and "sms=" in header
    finally:
        s.close()
    for text, expect_forced in ((header + "\n" + forced, True), (forced, True),
                                ("# device Other_GPU sms=1 cc=1.0\n" + forced, False)):
        path.write_text(text)
        s = B.Sampler(0, tune_cache=str(path))
        try:
            got = s.describe_plan(64, 16, 16, 1024)
            assert got == ("warp P=2 W=8 skip" if expect_forced else default), (text, got)
        finally:
            s.close()


def test_cached_plan_with_new_buffers(objects):
    """Without graphs a repeated argument set reuses its plan: other device
    buffers and other points must still give each set's own result, also
    after the autotuner has changed the variants."""
    build_mod.build()
    s = B.Sampler(0)
    try:
        sets = [objects[:8], [synth.object_batch(9, 8, 2048)[i] for i in range(8)]]
        bas = [B.BatchArgs(synth.pack(c)[1], 512, 16, 16, 0) for c in sets]
        xs = [torch.from_numpy(synth.pack(c)[0]).cuda() for c in sets]
        for rep in range(2):
            for c, ba, x in zip(sets, bas, xs):
                o = s.sample_batched(x, ba).cpu().numpy()
                for b in (0, 7):
                    assert_same(o[ba.out_off[b]:ba.out_off[b + 1]], oracle.afps(c[b], 512, 16, 16),
                                f"rep {rep} cloud {b}")
            if rep == 0:
                s.autotune_batched(xs[0], bas[0], torch.empty(bas[0].total_out, dtype=torch.int32,
                                                                device="cuda"))
    finally:
        s.close()


# --------------------------------------------------------------- stream ordering
# The sector kernels are launched with programmatic stream serialization:
# they may become resident while the previous kernel of the stream runs, and
# wait for it before touching global memory (an L2 prefetch hint is the only
# access issued earlier).  Points produced by the kernel right before, and
# outputs written by the call right before, must still be ordered.
def test_points_written_by_the_previous_kernel(objects):
    build_mod.build()
    for graph in (False, True):
        s = B.Sampler(0, graph=graph)
        try:
            xyz, off = synth.pack(objects[:8])
            base = torch.from_numpy(xyz).cuda()
            ba = B.BatchArgs(off, 512, 32, 16, 0)
            out = torch.empty(ba.total_out, dtype=torch.int32, device="cuda")
            x = torch.empty_like(base)
            for rep in range(3):
                # a long sampling call is still running when the points are rewritten
                s.sample_batched(base, B.BatchArgs(off, 512, 1, 0, 0))
                torch.mul(base, float(2 ** rep), out=x)  # exact scaling: same indices
                s.sample_batched(x, ba, out=out)
                o = out.cpu().numpy()
                for b in (0, 7):
                    assert_same(o[ba.out_off[b]:ba.out_off[b + 1]],
                                oracle.afps(objects[b], 512, 32, 16), f"graph={graph} rep {rep}")
        finally:
            s.close()


def test_back_to_back_calls_on_one_output(objects):
    """Calls on different clouds write the same output buffer one after the
    other; the last call's result must be what remains, for every pair."""
    build_mod.build()
    s = B.Sampler(0)
    try:
        sets = [objects[:8], objects[8:16], objects[16:24]]
        xs = [torch.from_numpy(synth.pack(c)[0]).cuda() for c in sets]
        ba = B.BatchArgs(synth.pack(sets[0])[1], 512, 32, 16, 0)
        out = torch.empty(ba.total_out, dtype=torch.int32, device="cuda")
        refs = [[oracle.afps(P, 512, 32, 16) for P in c] for c in sets]
        for order in ((0, 1, 2), (2, 0, 1), (1, 2, 0, 1)):
            for i in order:
                s.sample_batched(xs[i], ba, out=out)
            o = out.cpu().numpy()
            last = order[-1]
            for b in range(8):
                assert_same(o[ba.out_off[b]:ba.out_off[b + 1]], refs[last][b], f"order {order}")
        # a long chain of calls, each checked through its own output
        outs = [torch.empty(ba.total_out, dtype=torch.int32, device="cuda") for _ in range(60)]
        for j, o in enumerate(outs):
            s.sample_batched(xs[j % 3], ba, out=o)
        for j, o in enumerate(outs):
            oo = o.cpu().numpy()
            assert_same(oo[ba.out_off[5]:ba.out_off[6]], refs[j % 3][5], f"chain {j}")
    finally:
        s.close()


def test_calls_on_several_streams(objects):
    """One context, four streams.  Calls that share none of the context's
    workspace overlap on the device; calls that use it (the item table of a
    ragged batch, the work-queue counters of a batch wider than one wave of
    the grid) wait for its previous user on whatever stream.  Every output
    must equal the same call made alone, and those the oracle's."""
    build_mod.build()
    s = B.Sampler(0)
    try:
        wide = [objects[i % 32] for i in range(1024)]  # 32768 sectors: the work queue
        ragged = [objects[i][:2048 - 97 * i] for i in range(16)]  # an item table
        cases = [(wide, 32, 16), (ragged, 8, 8), (objects, 32, 16), (ragged, 32, 0),
                 (objects, 1, 0)]
        calls = []
        for clouds, M, k in cases:
            xyz, off = synth.pack(clouds)
            calls.append((torch.from_numpy(xyz).cuda(), B.BatchArgs(off, 256, M, k, 0)))
        alone = []
        for x, ba in calls:
            alone.append(s.sample_batched(x, ba).cpu())
            s.sync()
        for j, (clouds, M, k) in enumerate(cases):
            ba = calls[j][1]
            for b in (0, len(clouds) - 1):
                assert_same(alone[j][ba.out_off[b]:ba.out_off[b + 1]].numpy(),
                            oracle.afps(clouds[b], 256, M, k), f"case {j} cloud {b}")
        streams = [torch.cuda.Stream() for _ in range(4)]
        plan = [(rep, j) for rep in range(6) for j in range(len(calls))]
        outs = [torch.full((calls[j][1].total_out,), -1, dtype=torch.int32, device="cuda")
                for _, j in plan]
        torch.cuda.synchronize()
        for (rep, j), o in zip(plan, outs):
            x, ba = calls[j]
            s.sample_batched(x, ba, out=o, stream=streams[(rep + j) % 4])
        torch.cuda.synchronize()
        s.sync()
        for (rep, j), o in zip(plan, outs):
            assert torch.equal(o.cpu(), alone[j]), f"rep {rep} case {j}"
    finally:
        s.close()


# --------------------------------------------------------------- failure detection
def test_bounded_wait_reports_timeout_and_context_survives():
    """Fault injection on the host side of the barrier: the copy is never
    issued, every bounded wait runs out after 1 ms, the kernel returns, the
    status word says so, and the GPU and a fresh call still work."""
    build_mod.build()
    P = synth.uniform_cloud(3, 2048)
    x = torch.from_numpy(P).cuda()
    s = B.Sampler(0, timeout_ns=1_000_000, flags=B.AFPS_FLAG_TEST_STALL_COPY)
    try:
        for (M, k) in ((32, 16), (1, 0)):
            s.sample(x, 64, M, k, 0)
            with pytest.raises(B.AfpsError) as ei:
                s.sync()
            assert ei.value.code == B.AFPS_ERR_TIMEOUT
            s.sync()  # cleared
    finally:
        s.close()
    s2 = B.Sampler(0)
    try:
        assert_same(gpu_one(s2, P, 512, 4, 0), oracle.afps(P, 512, 4, 0), "after timeout")
    finally:
        s2.close()


def _timed_stall(s, fn):
    import time
    t0 = time.perf_counter()
    fn()
    with pytest.raises(B.AfpsError) as ei:
        s.sync()
    assert ei.value.code == B.AFPS_ERR_TIMEOUT
    s.sync()  # cleared
    return time.perf_counter() - t0


def test_timeout_halts_every_kernel_kind():
    """After a bounded wait runs out, the kernels compute nothing more: each
    warp, CTA or cluster leaves its remaining items undone, so a stalled call
    costs a few timeouts, not one per item or per iteration.  Injected on the
    host side: stage-in copies never issued (window kernel over the 17,576
    items of the ragged batch, through its work queue; the warp and CTA
    kernels; the 8-CTA cluster of plain FPS on a 32K-point cloud), and
    cluster records never sent (the same cluster, 8,192 exchanges, which
    without the halt would each wait out the timeout).  The GPU and a fresh
    context keep working."""
    build_mod.build()
    clouds, Cs, Ms = synth.ragged_batch(3, 256)
    ks = [k_rule(m) for m in Ms]
    xyz, off = synth.pack(clouds)
    xr = torch.from_numpy(xyz).cuda()
    ba = B.BatchArgs(off, Cs, Ms, ks, 0)
    P = synth.slab_cloud(2, 32768)
    xs = torch.from_numpy(P).cuda()
    tmo = 1_000_000  # 1 ms
    x4k = xs[:4096].contiguous()
    cases = [  # (flags, call, kernel kind the planner picks)
        (B.AFPS_FLAG_TEST_STALL_COPY, lambda s: s.sample_batched(xr, ba), (17576, "win")),
        (B.AFPS_FLAG_TEST_STALL_COPY, lambda s: s.sample(xs, 4096, 512, 0, 0), (512, "warp")),
        (B.AFPS_FLAG_TEST_STALL_COPY, lambda s: s.sample(x4k, 1024, 1, 0, 0), (1, "cta")),
        (B.AFPS_FLAG_TEST_STALL_COPY, lambda s: s.sample(xs, 1024, 1, 0, 0), (1, "cluster")),
        (B.AFPS_FLAG_TEST_STALL_EXCHANGE, lambda s: s.sample(xs, 8192, 1, 0, 0), (1, "cluster")),
    ]
    for flags, call, (items, kind) in cases:
        s = B.Sampler(0, timeout_ns=tmo, flags=flags)
        try:
            if items == 17576:
                assert s.describe_batched(ba).startswith(kind)
            else:
                n = {512: 64, 1: 32768 if kind == "cluster" else 4096}[items]
                assert s.describe_plan(n, 8, 0, items).startswith(kind)
            secs = _timed_stall(s, lambda: call(s))
            assert secs < 1.0, (flags, kind, secs)  # thousands of timeouts would take seconds
        finally:
            s.close()
    s2 = B.Sampler(0)
    try:
        assert_same(gpu_one(s2, P, 8192, 1, 0), oracle.afps(P, 8192, 1, 0), "fresh context")
        got, _ = gpu_batch(s2, clouds[:8], Cs[:8], Ms[:8], ks[:8])
        for b in range(8):
            assert_same(got[b], oracle.afps(clouds[b], Cs[b], Ms[b], ks[b]), f"cloud {b}")
    finally:
        s2.close()


def test_timeout_halts_later_launches_until_sync():
    """A recorded timeout makes later launches on the context skip their
    work (their outputs stay untouched) until afps_sync reports it; after
    that the same call computes normally."""
    build_mod.build()
    P = synth.uniform_cloud(4, 4096)
    x = torch.from_numpy(P).cuda()
    s = B.Sampler(0, timeout_ns=1_000_000, flags=B.AFPS_FLAG_TEST_STALL_EXCHANGE)
    try:
        s.sample(torch.from_numpy(synth.slab_cloud(2, 16384)).cuda(), 4096, 1, 0, 0)
        out = torch.full((512,), -1, dtype=torch.int32, device="cuda")
        s.sample(x, 512, 16, 16, 0, out=out)  # queued behind the stalled call
        torch.cuda.synchronize()
        assert bool((out == -1).all())
        with pytest.raises(B.AfpsError) as ei:
            s.sync()
        assert ei.value.code == B.AFPS_ERR_TIMEOUT
        s.sample(x, 512, 16, 16, 0, out=out)
        s.sync()
        assert_same(out.cpu().numpy(), oracle.afps(P, 512, 16, 16), "after sync")
    finally:
        s.close()


def test_allocation_failure_is_reported_and_context_survives(objects):
    """Fault injection on the host: every growth of the context's workspace
    fails as on an exhausted device.  Batched calls that need an item table
    return AFPS_ERR_NO_MEMORY before launching anything, their
    outputs untouched; a server cannot reserve its tables; the context, the
    GPU and a fresh context still work."""
    build_mod.build()
    # clouds of different sizes: the batch needs an item table
    xyz, off = synth.pack([objects[0][:1500], objects[1], objects[2][:1900], objects[3]])
    x = torch.from_numpy(xyz).cuda()
    s = B.Sampler(0, flags=B.AFPS_FLAG_TEST_FAIL_ALLOC)
    try:
        for (M, k) in ((1, 0), (32, 16)):
            ba = B.BatchArgs(off, 512, M, k, 0)
            out = torch.full((ba.total_out,), -1, dtype=torch.int32, device="cuda")
            with pytest.raises(B.AfpsError) as ei:
                s.sample_batched(x, ba, out=out)
            assert ei.value.code == B.AFPS_ERR_NO_MEMORY
            s.sync()  # nothing was launched: no device-side error either
            assert bool((out == -1).all())
        with pytest.raises(B.AfpsError) as ei:
            B.Server(s, [1024, 256], 32, 16, hbm_budget_bytes=1 << 20)
        assert ei.value.code == B.AFPS_ERR_NO_MEMORY
        # a single-cloud call needs no workspace and still runs on this context
        P = objects[0]
        assert_same(gpu_one(s, P, 512, 4, 0), oracle.afps(P, 512, 4, 0), "no-workspace call")
    finally:
        s.close()
    s2 = B.Sampler(0)
    try:
        got, _ = gpu_batch(s2, objects[:4], 512, 32, 16)
        for b in range(4):
            assert_same(got[b], oracle.afps(objects[b], 512, 32, 16), f"fresh context, cloud {b}")
    finally:
        s2.close()


# --------------------------------------------------------------- chained levels
def test_chained_levels_lidar(S):
    frame = synth.lidar_frame(5)
    levels = [16384, 4096, 1024, 256]
    ref = oracle.chain(frame, levels, 32, 16)
    cloud = torch.from_numpy(frame).cuda()
    fidx = None
    for L, C in enumerate(levels):
        n = cloud.shape[0]
        sel = S.sample(cloud, C, 32, 16, 0)
        nxt = torch.empty((C, 3), dtype=torch.float32, device="cuda")
        nfr = torch.empty(C, dtype=torch.int32, device="cuda")
        sfr = torch.empty(C, dtype=torch.int32, device="cuda")
        S.gather_levels([0, n], cloud, fidx, [0, C], sel, nxt, nfr, sfr)
        S.sync()
        assert_same(sfr.cpu().numpy(), ref[L], f"level {L}")
        assert np.all(np.diff(nfr.cpu().numpy()) > 0)
        cloud, fidx = nxt, nfr


# --------------------------------------------------------------- random sweep
def test_random_configurations_batched(S):
    """A seeded random sweep through the batched entry point: ragged clouds
    (sorted, unsorted, with repeated points) with their own C, M, window,
    reading and start in one call, each equal to the oracle."""
    g = np.random.Generator(np.random.PCG64(31))
    for rep in range(4):
        clouds, Cs, Ms, ks, starts, methods = [], [], [], [], [], []
        while len(clouds) < 24:
            N = int(g.integers(1, 3000))
            M = int(g.integers(1, min(N, 64) + 1))
            C = int(g.integers(M, min(N, 600) + 1))
            lo = [(s * N) // M for s in range(M + 1)]
            off = [(s * C) // M for s in range(M + 1)]
            if any(off[s + 1] - off[s] > lo[s + 1] - lo[s] for s in range(M)):
                continue
            k = int(g.choice([0, 0, 2, 3, 8, 16, 33]))
            kind = len(clouds) % 3
            seed = 5000 + 100 * rep + len(clouds)
            if kind == 0:
                P = synth.uniform_cloud(seed, N)
            elif kind == 1:
                P = synth.uniform_cloud(seed, N, axis=None)
            else:
                P = np.ascontiguousarray(np.resize(synth.uniform_cloud(seed, max(1, N // 3)),
                                                   (N, 3)).astype(np.float32))
            clouds.append(P)
            Cs.append(C)
            Ms.append(M)
            ks.append(k)
            starts.append(int(g.integers(0, N)))
            methods.append(int(g.integers(0, 4)) if k > 0 else 0)
        xyz, off = synth.pack(clouds)
        ba = B.BatchArgs(off, Cs, Ms, ks, starts, method=methods)
        out = S.sample_batched(torch.from_numpy(xyz).cuda(), ba)
        S.sync()
        o = out.cpu().numpy()
        for b, P in enumerate(clouds):
            ref = oracle.afps(P, Cs[b], Ms[b], ks[b], starts[b], method=methods[b])
            assert_same(o[ba.out_off[b]:ba.out_off[b + 1]], ref,
                        f"rep {rep} cloud {b}: N={P.shape[0]} C={Cs[b]} M={Ms[b]} k={ks[b]} "
                        f"start={starts[b]} method={methods[b]}")
