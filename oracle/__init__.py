"""CPU oracle for FPS / AFPS / NPDU-AFPS (arXiv 2208.08795) -- test infrastructure.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It never serves as a fallback for the
CUDA path and shares no code with it.

The arithmetic lives in ``afps_oracle.c`` (plain C, compiled with
``-ffp-contract=off`` so every product and sum is rounded on its own, as in
the CUDA path).  This module builds it with gcc and wraps it with ctypes;
numpy is used only to marshal arrays, and, for the chained-level gather, as a
library sort.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(_HERE, "afps_oracle.c")
LIBRARY = os.path.join(_HERE, "liboracle.so")

OK = 0
ERR_INVALID_ARG = -1
ERR_SECTOR_TOO_SMALL = -2
ERR_NO_MEMORY = -3

_lock = threading.Lock()
_lib = None


def compile_oracle(source: str = SOURCE, output: str = LIBRARY, werror: bool = True,
                   extra_flags=()) -> str:
    """Compile the oracle C source into a shared library; returns its path.
    ``extra_flags`` are added to the compiler line (sanitizer builds)."""
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-std=c11", "-Wall"] + (["-Werror"] if werror else []) + list(extra_flags) + \
          ["-o", output, source, "-lm"]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    return output


def _declare(lib: ctypes.CDLL) -> ctypes.CDLL:
    i64, i32 = ctypes.c_int64, ctypes.c_int32
    vp = ctypes.c_void_p
    for name in ("oracle_afps_f32", "oracle_afps_f64"):
        fn = getattr(lib, name)
        fn.argtypes = [vp, i64, i32, i32, i32, i64, vp]
        fn.restype = ctypes.c_int
    for name in ("oracle_afps_ex_f32", "oracle_afps_ex_f64"):
        fn = getattr(lib, name)
        fn.argtypes = [vp, i64, i32, i32, i32, i64, ctypes.c_uint32, vp]
        fn.restype = ctypes.c_int
    lib.oracle_sector_table.argtypes = [i64, i32, i32, i64, vp, vp, vp]
    lib.oracle_sector_table.restype = ctypes.c_int
    lib.oracle_coverage_radius.argtypes = [vp, i64, vp, i32]
    lib.oracle_coverage_radius.restype = ctypes.c_double
    return lib


def load_library(path: str) -> ctypes.CDLL:
    """Load an oracle library built by :func:`compile_oracle`."""
    return _declare(ctypes.CDLL(path))


def lib() -> ctypes.CDLL:
    """The oracle library, compiled on first use if it is missing or stale."""
    global _lib
    with _lock:
        if _lib is None:
            stale = (not os.path.exists(LIBRARY)
                     or os.path.getmtime(LIBRARY) < os.path.getmtime(SOURCE))
            if stale:
                compile_oracle()
            _lib = load_library(LIBRARY)
        return _lib


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle error {code}")
        self.code = code


def _points(xyz) -> np.ndarray:
    a = np.ascontiguousarray(xyz, dtype=np.float32)
    if a.ndim != 2 or a.shape[1] != 3:
        raise ValueError("xyz must have shape (N, 3)")
    return a


NPDU_FULL_FIRST_PASS = 1
NPDU_WINDOW_HAS_SAMPLE = 2


def afps(xyz, C: int, M: int = 1, k: int = 0, start: int = 0, *,
         precision: str = "f32", method: int = 0,
         library: ctypes.CDLL | None = None) -> np.ndarray:
    """NPDU-AFPS of one cloud: C int32 global indices, sector-major.

    M = 1 and k = 0 is plain FPS (Algorithm 1); k = 0 is AFPS (Sec. III-B);
    k > 0 adds the NPDU window of Sec. III-C.  ``precision`` is "f32" (the
    bit-exact reference for the GPU) or "f64".  ``method`` selects other
    readings of the NPDU window (NPDU_FULL_FIRST_PASS, NPDU_WINDOW_HAS_SAMPLE).
    """
    L = library or lib()
    pts = _points(xyz)
    out = np.full(max(int(C), 0), -1, dtype=np.int32)
    if method:
        fn = L.oracle_afps_ex_f32 if precision == "f32" else L.oracle_afps_ex_f64
        rc = fn(pts.ctypes.data, pts.shape[0], int(C), int(M), int(k), int(start), int(method),
                out.ctypes.data if out.size else None)
    else:
        fn = L.oracle_afps_f32 if precision == "f32" else L.oracle_afps_f64
        rc = fn(pts.ctypes.data, pts.shape[0], int(C), int(M), int(k), int(start),
                out.ctypes.data if out.size else None)
    if rc != OK:
        raise OracleError(rc)
    return out


def fps(xyz, C: int, start: int = 0, **kw) -> np.ndarray:
    """Plain FPS (Algorithm 1, fixed start)."""
    return afps(xyz, C, 1, 0, start, **kw)


def sector_table(N: int, C: int, M: int, start: int = 0, *, library=None):
    """(lo[M+1], off[M+1], first[M]) of the AFPS sector partition."""
    L = library or lib()
    lo = np.zeros(M + 1, dtype=np.int64)
    off = np.zeros(M + 1, dtype=np.int64)
    first = np.zeros(M, dtype=np.int64)
    rc = L.oracle_sector_table(int(N), int(C), int(M), int(start),
                               lo.ctypes.data, off.ctypes.data, first.ctypes.data)
    if rc != OK:
        raise OracleError(rc)
    return lo, off, first


def coverage_radius(xyz, idx, *, library=None) -> float:
    """max_j min_{s in idx} ||p_j - p_s|| in fp64."""
    L = library or lib()
    pts = _points(xyz)
    ix = np.ascontiguousarray(idx, dtype=np.int32)
    r = L.oracle_coverage_radius(pts.ctypes.data, pts.shape[0], ix.ctypes.data, ix.size)
    if r < 0:
        raise ValueError("bad arguments to coverage_radius")
    return float(r)


def afps_batched(xyz, pt_off, C, M, k, start, *, precision="f32", library=None):
    """Ragged batch: cloud b is xyz[pt_off[b]:pt_off[b+1]]; returns a list of
    per-cloud index arrays (relative to the cloud's first point)."""
    res = []
    for b in range(len(pt_off) - 1):
        pts = xyz[pt_off[b]:pt_off[b + 1]]
        res.append(afps(pts, C[b], M[b], k[b], start[b], precision=precision,
                        library=library))
    return res


def chain(xyz, levels, M: int, k: int, start: int = 0, *, library=None):
    """Chained multi-level sampling (PointNet++ hierarchy, Sec. I).

    Level 0 samples levels[0] points from the frame; level L+1 samples from
    level L's samples taken in ascending frame index (this keeps the storage
    order, and hence the dimensional locality of Sec. III-A).  Returns, per
    level, the sampled frame indices in emission order.
    """
    frame_idx = np.arange(np.asarray(xyz).shape[0], dtype=np.int64)
    cloud = _points(xyz)
    out = []
    for C in levels:
        Ml = min(M, C)
        sel = afps(cloud, C, Ml, k, start, library=library)
        out.append(frame_idx[sel].astype(np.int32))
        order = np.sort(sel)
        cloud = cloud[order]
        frame_idx = frame_idx[order]
    return out


# --------------------------------------------------------------------------
# sorting by key (for unsorted input; binning or sorting restores the
# dimensional locality of Sec. III-A)
# --------------------------------------------------------------------------
KEY_X, KEY_Y, KEY_Z, KEY_AZIMUTH = 0, 1, 2, 3


def diamond_angle(x, y):
    """A monotone stand-in for atan2(y, x) mapped to [0, 4): each quadrant's
    angle is replaced by a ratio of coordinates (every operation rounded on
    its own in fp32); the origin maps to 0."""
    x = np.asarray(x, dtype=np.float32)
    y = np.asarray(y, dtype=np.float32)
    one, two, three = np.float32(1), np.float32(2), np.float32(3)
    out = np.zeros(x.shape, dtype=np.float32)
    with np.errstate(invalid="ignore", divide="ignore"):
        q0 = (y >= 0) & (x >= 0)
        q1 = (y >= 0) & (x < 0)
        q2 = (y < 0) & (x < 0)
        q3 = (y < 0) & (x >= 0)
        out[q0] = y[q0] / (x[q0] + y[q0])
        out[q1] = one - x[q1] / (-x[q1] + y[q1])
        out[q2] = two - y[q2] / (-x[q2] - y[q2])
        out[q3] = three + x[q3] / (x[q3] - y[q3])
    out[(x == 0) & (y == 0)] = 0
    return out


def sort_key(xyz, key: int) -> np.ndarray:
    pts = _points(xyz)
    if key in (KEY_X, KEY_Y, KEY_Z):
        k = pts[:, key].copy()
    elif key == KEY_AZIMUTH:
        k = diamond_angle(pts[:, 0], pts[:, 1])
    else:
        raise ValueError("unknown key")
    return k + np.float32(0)  # -0 becomes +0


def sort_by_key(xyz, key: int):
    """Stable ascending sort of the points by key: (sorted points, permutation
    such that sorted[i] = xyz[perm[i]])."""
    pts = _points(xyz)
    perm = np.argsort(sort_key(pts, key), kind="stable").astype(np.int32)
    return pts[perm], perm


def knn(xyz, centroids, K: int, *, library=None, with_d2: bool = False):
    """The K nearest points of each centroid, nearest first, ties to the lower
    index: (C, K) int32 (and the (C, K) float32 squared distances)."""
    L = library or lib()
    if not hasattr(L, "_knn"):
        L.oracle_knn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                 ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                 ctypes.c_void_p]
        L.oracle_knn.restype = ctypes.c_int
        L._knn = True
    pts = _points(xyz)
    c = np.ascontiguousarray(centroids, dtype=np.int32)
    out = np.full((c.size, int(K)), -1, dtype=np.int32)
    d2 = np.zeros((c.size, int(K)), dtype=np.float32)
    rc = L.oracle_knn(pts.ctypes.data, pts.shape[0], c.ctypes.data, c.size, int(K),
                      out.ctypes.data, d2.ctypes.data)
    if rc != OK:
        raise OracleError(rc)
    return (out, d2) if with_d2 else out


def ball_query(xyz, centroids, radius: float, K: int, *, library=None) -> np.ndarray:
    """First K points (storage order) within `radius` of each centroid,
    padded with the first one found: (C, K) int32."""
    L = library or lib()
    if not hasattr(L, "_bq"):
        L.oracle_ball_query.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                        ctypes.c_int32, ctypes.c_float, ctypes.c_int32,
                                        ctypes.c_void_p]
        L.oracle_ball_query.restype = ctypes.c_int
        L._bq = True
    pts = _points(xyz)
    c = np.ascontiguousarray(centroids, dtype=np.int32)
    out = np.full((c.size, int(K)), -1, dtype=np.int32)
    rc = L.oracle_ball_query(pts.ctypes.data, pts.shape[0], c.ctypes.data, c.size,
                             float(radius), int(K), out.ctypes.data)
    if rc != OK:
        raise OracleError(rc)
    return out
