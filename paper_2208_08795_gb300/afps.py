"""Thin ctypes binding of libafps.so (include/afps.h).

The functions ``afps_*`` below have the C names and arguments (device and
host buffers as integer addresses, the stream as a ``cudaStream_t`` address);
they only marshal arguments.  :class:`Sampler` wraps them for torch tensors:
torch provides device memory and the current stream, every step of the
sampling runs in the library's CUDA kernels.  There is no CPU fallback: a
missing or unloadable library raises :class:`AfpsLibraryError`.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIBRARY = os.path.join(_PKG, "libafps.so")

AFPS_OK = 0
AFPS_ERR_INVALID_ARG = -1
AFPS_ERR_SECTOR_TOO_SMALL = -2
AFPS_ERR_NO_MEMORY = -3
AFPS_ERR_TIMEOUT = -4
AFPS_ERR_CUDA = -5
AFPS_ERR_UNSUPPORTED = -6
AFPS_ERR_SCRATCH_TOO_SMALL = -7
AFPS_NOALLOC_MAX_ITEMS = 8192
AFPS_MAX_SECTOR_POINTS = 131072
AFPS_FLAG_GRAPH = 1
AFPS_FLAG_AUTOTUNE = 2
AFPS_FLAG_TEST_STALL_COPY = 0x100
AFPS_FLAG_TEST_STALL_EXCHANGE = 0x400
AFPS_FLAG_TEST_FAIL_ALLOC = 0x200

# every symbol include/afps.h declares
EXPORTS = ("afps_create", "afps_destroy", "afps_sample", "afps_sample_batched",
           "afps_sample_batched_host", "afps_gather_levels", "afps_sync",
           "afps_last_error", "afps_autotune_batched", "afps_save_tuning",
           "afps_describe_plan", "afps_describe_batched", "afps_launch_count",
           "afps_sample_batched_noalloc",
           "afps_server_create", "afps_server_submit", "afps_server_step", "afps_server_poll",
           "afps_server_stats", "afps_server_clock_ms", "afps_server_destroy",
           "afps_sort_by_key", "afps_sample_ex", "afps_sample_batched_ex",
           "afps_coverage_radius", "afps_ball_query", "afps_knn",
           "afps_sample_batched_host_async", "afps_server_submit_pinned", "afps_server_cancel")


class AfpsLibraryError(RuntimeError):
    pass


class AfpsError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"afps error {code}: {message}")
        self.code = code
        self.message = message


AFPS_ERR_BUSY = -8
AFPS_ERR_DEVICE_CHECK = -9
AFPS_KEY_X, AFPS_KEY_Y, AFPS_KEY_Z, AFPS_KEY_AZIMUTH = 0, 1, 2, 3
AFPS_METHOD_FULL_FIRST_PASS = 1
AFPS_METHOD_WINDOW_HAS_SAMPLE = 2
AFPS_METHOD_ALL = 3
AFPS_SERVER_MAX_LEVELS = 8


class afps_server_config(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("max_queued", ctypes.c_int64),
                ("max_inflight", ctypes.c_int32), ("n_levels", ctypes.c_int32),
                ("levels", ctypes.c_int32 * AFPS_SERVER_MAX_LEVELS), ("M", ctypes.c_int32),
                ("npdu_window", ctypes.c_int32), ("max_steps_ahead", ctypes.c_int32),
                ("levels_per_step", ctypes.c_int32), ("host_pool_bytes", ctypes.c_int64)]


class afps_server_result(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("status", ctypes.c_int32), ("n_levels", ctypes.c_int32),
                ("count", ctypes.c_int32 * AFPS_SERVER_MAX_LEVELS),
                ("indices", ctypes.POINTER(ctypes.c_int32)), ("submit_ms", ctypes.c_double),
                ("admit_ms", ctypes.c_double), ("done_ms", ctypes.c_double)]


class afps_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("timeout_ns", ctypes.c_int64), ("tune_cache", ctypes.c_char_p)]


_lock = threading.Lock()
_lib = None


def _declare(L: ctypes.CDLL) -> ctypes.CDLL:
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    L.afps_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(afps_config)]
    L.afps_create.restype = ctypes.c_int
    L.afps_destroy.argtypes = [vp]
    L.afps_destroy.restype = None
    L.afps_sample.argtypes = [vp, vp, i64, i32, i32, i32, i64, vp, vp]
    L.afps_sample.restype = ctypes.c_int
    batched = [vp, vp, vp, i32, vp, vp, vp, vp, vp, vp, vp]
    for name in ("afps_sample_batched", "afps_sample_batched_host",
                 "afps_sample_batched_host_async", "afps_autotune_batched"):
        getattr(L, name).argtypes = batched
        getattr(L, name).restype = ctypes.c_int
    L.afps_gather_levels.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    L.afps_gather_levels.restype = ctypes.c_int
    L.afps_sync.argtypes = [vp, vp]
    L.afps_sync.restype = ctypes.c_int
    L.afps_last_error.argtypes = [vp]
    L.afps_last_error.restype = ctypes.c_char_p
    L.afps_save_tuning.argtypes = [vp, ctypes.c_char_p]
    L.afps_save_tuning.restype = ctypes.c_int
    L.afps_describe_plan.argtypes = [vp, i64, i32, i32, i32, ctypes.c_char_p, i32]
    L.afps_describe_plan.restype = ctypes.c_int
    L.afps_describe_batched.argtypes = [vp, vp, i32, vp, vp, vp, vp, vp, ctypes.c_char_p, i32]
    L.afps_describe_batched.restype = ctypes.c_int
    L.afps_launch_count.argtypes = [vp]
    L.afps_launch_count.restype = ctypes.c_int64
    L.afps_sample_batched_noalloc.argtypes = [vp, vp, i32, vp, vp, vp, vp, vp, vp, vp]
    L.afps_sample_batched_noalloc.restype = ctypes.c_int
    L.afps_sample_ex.argtypes = [vp, vp, i64, i32, i32, i32, i64, ctypes.c_uint32, vp, vp]
    L.afps_sample_ex.restype = ctypes.c_int
    L.afps_sample_batched_ex.argtypes = [vp, vp, vp, i32, vp, vp, vp, vp, vp, vp, vp, vp]
    L.afps_sample_batched_ex.restype = ctypes.c_int
    L.afps_sort_by_key.argtypes = [vp, i32, vp, vp, i32, vp, vp, vp]
    L.afps_coverage_radius.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp]
    L.afps_ball_query.argtypes = [vp, i32, vp, vp, vp, vp, ctypes.c_float, i32, i32, vp, vp]
    L.afps_ball_query.restype = ctypes.c_int
    L.afps_knn.argtypes = [vp, i32, vp, vp, vp, vp, i32, i32, vp, vp, vp]
    L.afps_knn.restype = ctypes.c_int
    L.afps_coverage_radius.restype = ctypes.c_int
    L.afps_sort_by_key.restype = ctypes.c_int
    L.afps_server_create.argtypes = [ctypes.POINTER(vp), vp, ctypes.POINTER(afps_server_config), vp]
    L.afps_server_create.restype = ctypes.c_int
    L.afps_server_submit.argtypes = [vp, vp, i64, ctypes.c_uint64]
    L.afps_server_submit.restype = ctypes.c_int
    L.afps_server_submit_pinned.argtypes = [vp, vp, i64, ctypes.c_uint64]
    L.afps_server_submit_pinned.restype = ctypes.c_int
    L.afps_server_cancel.argtypes = [vp, ctypes.c_uint64]
    L.afps_server_cancel.restype = ctypes.c_int
    L.afps_server_step.argtypes = [vp]
    L.afps_server_step.restype = ctypes.c_int
    L.afps_server_poll.argtypes = [vp, ctypes.POINTER(afps_server_result), i32]
    L.afps_server_poll.restype = ctypes.c_int
    L.afps_server_stats.argtypes = [vp, vp, vp, vp]
    L.afps_server_stats.restype = ctypes.c_int
    L.afps_server_clock_ms.argtypes = [vp]
    L.afps_server_clock_ms.restype = ctypes.c_double
    L.afps_server_destroy.argtypes = [vp]
    L.afps_server_destroy.restype = None
    return L


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libafps.so (built by ``paper_2208_08795_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIBRARY
            if not os.path.exists(p):
                raise AfpsLibraryError(
                    f"{p} is missing: build it with `python -m paper_2208_08795_gb300.build` "
                    "(there is no CPU fallback)")
            try:
                _lib = _declare(ctypes.CDLL(p))
            except OSError as e:
                raise AfpsLibraryError(f"cannot load {p}: {e}") from e
        return _lib


# ------------------------------------------------------------- raw C calls
def afps_create(device: int = 0, flags: int = 0, timeout_ns: int = 0,
                tune_cache: str | None = None) -> int:
    cfg = afps_config(device, flags, timeout_ns,
                      tune_cache.encode() if tune_cache else None)
    h = ctypes.c_void_p()
    rc = load().afps_create(ctypes.byref(h), ctypes.byref(cfg))
    if rc != AFPS_OK:
        raise AfpsError(rc, "afps_create failed")
    return h.value


def afps_destroy(ctx: int) -> None:
    load().afps_destroy(ctx)


def afps_sample(ctx, d_xyz, N, C, M, npdu_window, start_idx, d_out, stream) -> int:
    return load().afps_sample(ctx, d_xyz, N, C, M, npdu_window, start_idx, d_out, stream)


def afps_sample_ex(ctx, d_xyz, N, C, M, npdu_window, start_idx, method, d_out, stream) -> int:
    return load().afps_sample_ex(ctx, d_xyz, N, C, M, npdu_window, start_idx, method, d_out,
                                 stream)


def afps_sample_batched_ex(ctx, d_xyz, h_pt_off, B, h_C, h_M, h_win, h_start, h_method,
                           h_out_off, d_out, stream) -> int:
    return load().afps_sample_batched_ex(ctx, d_xyz, h_pt_off, B, h_C, h_M, h_win, h_start,
                                         h_method, h_out_off, d_out, stream)


def afps_sample_batched(ctx, d_xyz, h_pt_off, B, h_C, h_M, h_win, h_start, h_out_off,
                        d_out, stream) -> int:
    return load().afps_sample_batched(ctx, d_xyz, h_pt_off, B, h_C, h_M, h_win, h_start,
                                      h_out_off, d_out, stream)


def afps_sample_batched_host(ctx, h_xyz, h_pt_off, B, h_C, h_M, h_win, h_start, h_out_off,
                             h_out, stream) -> int:
    return load().afps_sample_batched_host(ctx, h_xyz, h_pt_off, B, h_C, h_M, h_win,
                                           h_start, h_out_off, h_out, stream)


def afps_sample_batched_host_async(ctx, h_xyz, h_pt_off, B, h_C, h_M, h_win, h_start,
                                   h_out_off, h_out, stream) -> int:
    return load().afps_sample_batched_host_async(ctx, h_xyz, h_pt_off, B, h_C, h_M, h_win,
                                                 h_start, h_out_off, h_out, stream)


def afps_autotune_batched(ctx, d_xyz, h_pt_off, B, h_C, h_M, h_win, h_start, h_out_off,
                          d_out, stream) -> int:
    return load().afps_autotune_batched(ctx, d_xyz, h_pt_off, B, h_C, h_M, h_win, h_start,
                                        h_out_off, d_out, stream)


def afps_gather_levels(ctx, B, h_in_pt_off, d_in_xyz, d_in_frame, h_sel_off, d_sel,
                       d_out_xyz, d_out_frame, d_sel_frame, stream) -> int:
    return load().afps_gather_levels(ctx, B, h_in_pt_off, d_in_xyz, d_in_frame, h_sel_off,
                                     d_sel, d_out_xyz, d_out_frame, d_sel_frame, stream)


def afps_sync(ctx, stream) -> int:
    return load().afps_sync(ctx, stream)


def afps_last_error(ctx) -> str:
    return load().afps_last_error(ctx).decode()


def afps_save_tuning(ctx, path: str | None) -> int:
    return load().afps_save_tuning(ctx, path.encode() if path else None)


def afps_describe_plan(ctx, n_sector: int, c_sector: int, npdu_window: int,
                       n_items: int = 1) -> str:
    buf = ctypes.create_string_buffer(128)
    rc = load().afps_describe_plan(ctx, n_sector, c_sector, npdu_window, n_items, buf, 128)
    if rc < 0:
        raise AfpsError(rc, "afps_describe_plan failed")
    return buf.value.decode()


def afps_describe_batched(ctx, h_pt_off, B, h_C, h_M, h_win, h_start, h_out_off) -> str:
    buf = ctypes.create_string_buffer(1024)
    rc = load().afps_describe_batched(ctx, h_pt_off, B, h_C, h_M, h_win, h_start, h_out_off,
                                      buf, 1024)
    if rc < 0:
        raise AfpsError(rc, afps_last_error(ctx))
    return buf.value.decode()


def afps_launch_count(ctx) -> int:
    return load().afps_launch_count(ctx)


def afps_sort_by_key(ctx, B, h_pt_off, d_xyz, key, d_xyz_sorted, d_perm, stream) -> int:
    return load().afps_sort_by_key(ctx, B, h_pt_off, d_xyz, key, d_xyz_sorted, d_perm, stream)


def afps_coverage_radius(ctx, B, h_pt_off, d_xyz, h_sel_off, d_sel, d_radius, stream) -> int:
    return load().afps_coverage_radius(ctx, B, h_pt_off, d_xyz, h_sel_off, d_sel, d_radius, stream)


def afps_ball_query(ctx, B, h_pt_off, d_xyz, h_sel_off, d_sel, radius, K, sorted_axis, d_group,
                    stream) -> int:
    return load().afps_ball_query(ctx, B, h_pt_off, d_xyz, h_sel_off, d_sel, radius, K,
                                  sorted_axis, d_group, stream)


def afps_knn(ctx, B, h_pt_off, d_xyz, h_sel_off, d_sel, K, sorted_axis, d_group, d_dist2,
             stream) -> int:
    return load().afps_knn(ctx, B, h_pt_off, d_xyz, h_sel_off, d_sel, K, sorted_axis, d_group,
                           d_dist2, stream)


def afps_sample_batched_noalloc(d_xyz, h_pt_off, B, h_C, h_M, h_win, h_start, h_out_off,
                                d_out, stream) -> int:
    """The batched call for callers that cannot allocate (no context)."""
    return load().afps_sample_batched_noalloc(d_xyz, h_pt_off, B, h_C, h_M, h_win, h_start,
                                              h_out_off, d_out, stream)


# ---------------------------------------------------------------- helpers
def _i64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64))


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


class BatchArgs:
    """Host arrays of a batched call, kept alive for the call's duration."""

    def __init__(self, pt_off, C, M, k, start, out_off=None, method=None):
        self.pt_off = _i64(pt_off)
        B = self.pt_off.size - 1
        self.B = B
        self.method = (None if method is None else
                       np.ascontiguousarray(np.broadcast_to(method, (B,)), dtype=np.uint32))
        self.C = _i32(np.broadcast_to(C, (B,)))
        self.M = _i32(np.broadcast_to(M, (B,)))
        self.k = _i32(np.broadcast_to(k, (B,)))
        self.start = _i64(np.broadcast_to(start, (B,)))
        if out_off is None:
            out_off = np.zeros(B + 1, dtype=np.int64)
            np.cumsum(self.C, out=out_off[1:])
        self.out_off = _i64(out_off)

    def args(self):
        return (_ptr(self.pt_off), self.B, _ptr(self.C), _ptr(self.M), _ptr(self.k),
                _ptr(self.start), _ptr(self.out_off))

    @property
    def total_out(self) -> int:
        return int(self.out_off[-1])


class Sampler:
    """A libafps context on one CUDA device, driven with torch tensors."""

    def __init__(self, device: int = 0, graph: bool = False, timeout_ns: int = 0,
                 tune_cache: str | None = None, flags: int = 0):
        flags |= AFPS_FLAG_GRAPH if graph else 0
        self.device = device
        self.ctx = afps_create(device, flags, timeout_ns, tune_cache)

    def close(self):
        if self.ctx:
            afps_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int):
        if rc != AFPS_OK:
            raise AfpsError(rc, afps_last_error(self.ctx))

    @staticmethod
    def _stream(stream):
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        return s.cuda_stream

    @staticmethod
    def _points(xyz):
        import torch
        if not (isinstance(xyz, torch.Tensor) and xyz.is_cuda and xyz.dtype == torch.float32
                and xyz.dim() == 2 and xyz.shape[1] == 3 and xyz.is_contiguous()):
            raise ValueError("xyz must be a contiguous float32 CUDA tensor of shape (N, 3)")
        return xyz

    def sample(self, xyz, C: int, M: int = 1, k: int = 0, start: int = 0, out=None,
               stream=None, method: int = 0):
        """NPDU-AFPS of one cloud; returns C int32 indices (sector-major).
        ``method``: AFPS_METHOD_* reading of the NPDU window (0 = default)."""
        import torch
        xyz = self._points(xyz)
        if out is None:
            out = torch.empty(C, dtype=torch.int32, device=xyz.device)
        if method:
            rc = afps_sample_ex(self.ctx, xyz.data_ptr(), xyz.shape[0], C, M, k, start, method,
                                out.data_ptr(), self._stream(stream))
        else:
            rc = afps_sample(self.ctx, xyz.data_ptr(), xyz.shape[0], C, M, k, start,
                             out.data_ptr(), self._stream(stream))
        self._check(rc)
        return out

    def sample_batched(self, xyz, pt_off, C=None, M=None, k=None, start=0, out_off=None,
                       out=None, stream=None):
        """Ragged batch: cloud b is xyz[pt_off[b]:pt_off[b+1]]; pt_off may be a
        prepared :class:`BatchArgs` (then C, M, k, start, out_off are unused)."""
        import torch
        xyz = self._points(xyz)
        ba = pt_off if isinstance(pt_off, BatchArgs) else BatchArgs(pt_off, C, M, k, start, out_off)
        if out is None:
            out = torch.empty(ba.total_out, dtype=torch.int32, device=xyz.device)
        if ba.method is not None:
            pt, B, c, m, k, st, oo = ba.args()
            rc = afps_sample_batched_ex(self.ctx, xyz.data_ptr(), pt, B, c, m, k, st,
                                        _ptr(ba.method), oo, out.data_ptr(), self._stream(stream))
        else:
            rc = afps_sample_batched(self.ctx, xyz.data_ptr(), *ba.args(), out.data_ptr(),
                                     self._stream(stream))
        self._check(rc)
        return out

    def sample_batched_host(self, h_xyz: np.ndarray, ba: "BatchArgs", h_out: np.ndarray,
                            stream=None):
        """Host buffers in and out; the copies run inside the call."""
        assert h_xyz.dtype == np.float32 and h_xyz.flags.c_contiguous
        assert h_out.dtype == np.int32 and h_out.flags.c_contiguous
        self._check(load().afps_sample_batched_host(
            self.ctx, h_xyz.ctypes.data, _ptr(ba.pt_off), ba.B, _ptr(ba.C), _ptr(ba.M),
            _ptr(ba.k), _ptr(ba.start), _ptr(ba.out_off), h_out.ctypes.data,
            self._stream(stream)))
        return h_out

    def sample_batched_host_async(self, h_xyz: np.ndarray, ba: "BatchArgs", h_out: np.ndarray,
                                  stream=None):
        """Page-locked host buffers in and out, returning once queued; h_out
        is valid after `sync` (keep both buffers alive and unchanged until then)."""
        assert h_xyz.dtype == np.float32 and h_xyz.flags.c_contiguous
        assert h_out.dtype == np.int32 and h_out.flags.c_contiguous
        self._check(load().afps_sample_batched_host_async(
            self.ctx, h_xyz.ctypes.data, _ptr(ba.pt_off), ba.B, _ptr(ba.C), _ptr(ba.M),
            _ptr(ba.k), _ptr(ba.start), _ptr(ba.out_off), h_out.ctypes.data,
            self._stream(stream)))
        return h_out

    def autotune_batched(self, xyz, ba: "BatchArgs", out, stream=None) -> int:
        rc = load().afps_autotune_batched(self.ctx, xyz.data_ptr(), _ptr(ba.pt_off), ba.B,
                                          _ptr(ba.C), _ptr(ba.M), _ptr(ba.k), _ptr(ba.start),
                                          _ptr(ba.out_off), out.data_ptr(), self._stream(stream))
        if rc < 0:
            raise AfpsError(rc, afps_last_error(self.ctx))
        return rc

    def gather_levels(self, in_pt_off, in_xyz, in_frame, sel_off, sel, out_xyz, out_frame,
                      sel_frame=None, stream=None):
        ipo, so = _i64(in_pt_off), _i64(sel_off)
        self._check(afps_gather_levels(
            self.ctx, ipo.size - 1, _ptr(ipo), in_xyz.data_ptr(),
            in_frame.data_ptr() if in_frame is not None else None, _ptr(so), sel.data_ptr(),
            out_xyz.data_ptr(), out_frame.data_ptr() if out_frame is not None else None,
            sel_frame.data_ptr() if sel_frame is not None else None, self._stream(stream)))

    def sort_by_key(self, xyz, pt_off, key: int = AFPS_KEY_X, out=None, perm=None,
                    stream=None):
        """Stable sort of each cloud by key; returns (sorted points, permutation)."""
        import torch
        xyz = self._points(xyz)
        po = _i64(pt_off)
        if out is None:
            out = torch.empty_like(xyz)
        if perm is None:
            perm = torch.empty(xyz.shape[0], dtype=torch.int32, device=xyz.device)
        self._check(afps_sort_by_key(self.ctx, po.size - 1, _ptr(po), xyz.data_ptr(), key,
                                     out.data_ptr(), perm.data_ptr(), self._stream(stream)))
        return out, perm

    def coverage_radius(self, xyz, pt_off, sel, sel_off, stream=None):
        """fp64 coverage radius of each cloud's samples (a float64 tensor of B)."""
        import torch
        xyz = self._points(xyz)
        po, so = _i64(pt_off), _i64(sel_off)
        out = torch.empty(po.size - 1, dtype=torch.float64, device=xyz.device)
        self._check(afps_coverage_radius(self.ctx, po.size - 1, _ptr(po), xyz.data_ptr(), _ptr(so),
                                         sel.data_ptr(), out.data_ptr(), self._stream(stream)))
        return out

    def ball_query(self, xyz, pt_off, sel, sel_off, radius: float, K: int,
                   sorted_axis: int = -1, out=None, stream=None):
        """First K points within `radius` of every centroid: (sum C, K) int32."""
        import torch
        xyz = self._points(xyz)
        po, so = _i64(pt_off), _i64(sel_off)
        if out is None:
            out = torch.empty((int(so[-1]), K), dtype=torch.int32, device=xyz.device)
        self._check(afps_ball_query(self.ctx, po.size - 1, _ptr(po), xyz.data_ptr(), _ptr(so),
                                    sel.data_ptr(), radius, K, sorted_axis, out.data_ptr(),
                                    self._stream(stream)))
        return out

    def knn(self, xyz, pt_off, sel, sel_off, K: int, sorted_axis: int = -1, out=None,
            dist2=None, stream=None):
        """The K nearest points of every centroid, nearest first: (sum C, K)
        int32; ``dist2`` (optional, (sum C, K) float32) gets the squared
        distances."""
        import torch
        xyz = self._points(xyz)
        po, so = _i64(pt_off), _i64(sel_off)
        if out is None:
            out = torch.empty((int(so[-1]), K), dtype=torch.int32, device=xyz.device)
        self._check(afps_knn(self.ctx, po.size - 1, _ptr(po), xyz.data_ptr(), _ptr(so),
                             sel.data_ptr(), K, sorted_axis, out.data_ptr(),
                             dist2.data_ptr() if dist2 is not None else None,
                             self._stream(stream)))
        return out

    def sync(self, stream=None):
        self._check(afps_sync(self.ctx, self._stream(stream)))

    def describe_plan(self, n_sector: int, c_sector: int, k: int, n_items: int = 1) -> str:
        return afps_describe_plan(self.ctx, n_sector, c_sector, k, n_items)

    def describe_batched(self, ba: "BatchArgs") -> str:
        """The kernel launches of a batched call: "<variant> items=<n>; ..."."""
        return afps_describe_batched(self.ctx, *ba.args())

    @property
    def launch_count(self) -> int:
        return afps_launch_count(self.ctx)


# ------------------------------------------------------------------ serving
def afps_server_create(ctx, cfg: afps_server_config, stream=None) -> int:
    h = ctypes.c_void_p()
    rc = load().afps_server_create(ctypes.byref(h), ctx, ctypes.byref(cfg), stream)
    if rc != AFPS_OK:
        raise AfpsError(rc, "afps_server_create failed")
    return h.value


def afps_server_submit(srv, h_xyz, N, tag) -> int:
    return load().afps_server_submit(srv, h_xyz, N, tag)


def afps_server_submit_pinned(srv, h_xyz, N, tag) -> int:
    return load().afps_server_submit_pinned(srv, h_xyz, N, tag)


def afps_server_cancel(srv, tag) -> int:
    return load().afps_server_cancel(srv, tag)


def afps_server_step(srv) -> int:
    return load().afps_server_step(srv)


def afps_server_poll(srv, out, max_results) -> int:
    return load().afps_server_poll(srv, out, max_results)


def afps_server_stats(srv, queued, inflight, arena_used) -> int:
    return load().afps_server_stats(srv, queued, inflight, arena_used)


def afps_server_clock_ms(srv) -> float:
    return load().afps_server_clock_ms(srv)


def afps_server_destroy(srv) -> None:
    load().afps_server_destroy(srv)


# afps_server_result as a NumPy record (the pointer as an address), so that a
# poll reads all its results' fields at once
_RESULT_DTYPE = np.dtype({
    "names": ["tag", "status", "n_levels", "count", "indices", "submit_ms", "admit_ms", "done_ms"],
    "formats": ["<u8", "<i4", "<i4", ("<i4", (AFPS_SERVER_MAX_LEVELS,)), "<u8", "<f8", "<f8",
                "<f8"],
    "offsets": [getattr(afps_server_result, f).offset for f in
                ("tag", "status", "n_levels", "count", "indices", "submit_ms", "admit_ms",
                 "done_ms")],
    "itemsize": ctypes.sizeof(afps_server_result)})


class ServerResult:
    """One finished request: per-level frame indices and times.  With
    copy=False the indices are a view of the runtime's page-locked result
    slot, valid until the next poll (made when first read)."""

    __slots__ = ("tag", "status", "_counts", "_addr", "_indices", "submit_ms", "admit_ms",
                 "done_ms")

    def __init__(self, tag, status, counts, addr, submit_ms, admit_ms, done_ms, copy=True):
        self.tag, self.status, self._counts, self._addr = tag, status, counts, addr
        self.submit_ms, self.admit_ms, self.done_ms = submit_ms, admit_ms, done_ms
        self._indices = self._view().copy() if copy else None

    def _view(self):
        total = sum(self._counts)
        return np.frombuffer((ctypes.c_int32 * total).from_address(self._addr), dtype=np.int32)

    @property
    def indices(self):
        if self._indices is None:
            self._indices = self._view()
        return self._indices

    @property
    def levels(self):
        """The frame indices of each level's samples, in emission order."""
        return np.split(self.indices, np.cumsum(self._counts)[:-1])


class Server:
    """Continuous-batching server for chained sampling requests (afps_server_*)."""

    def __init__(self, sampler: "Sampler", levels, M: int, k: int, hbm_budget_bytes: int,
                 max_inflight: int = 256, max_queued: int = 4096, max_steps_ahead: int = 2,
                 host_pool_bytes: int = 0, levels_per_step: int = 0, stream=None):
        cfg = afps_server_config()
        cfg.hbm_budget_bytes = int(hbm_budget_bytes)
        cfg.max_queued = int(max_queued)
        cfg.max_inflight = int(max_inflight)
        cfg.n_levels = len(levels)
        for i, c in enumerate(levels):
            cfg.levels[i] = int(c)
        cfg.M, cfg.npdu_window, cfg.max_steps_ahead = int(M), int(k), int(max_steps_ahead)
        cfg.host_pool_bytes = int(host_pool_bytes)
        cfg.levels_per_step = int(levels_per_step)
        self.sampler = sampler
        self.srv = afps_server_create(sampler.ctx, cfg, stream)
        self._buf = (afps_server_result * 256)()
        self._rows = np.frombuffer(self._buf, dtype=_RESULT_DTYPE)

    def close(self):
        if self.srv:
            afps_server_destroy(self.srv)
            self.srv = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, xyz: np.ndarray, tag: int) -> int:
        a = np.ascontiguousarray(xyz, dtype=np.float32)
        return afps_server_submit(self.srv, a.ctypes.data, a.shape[0], tag)

    def submit_pinned(self, xyz: np.ndarray, tag: int) -> int:
        """Queue a frame held in page-locked memory without copying it; the
        array must stay alive and unchanged until its result is polled."""
        assert xyz.dtype == np.float32 and xyz.flags.c_contiguous
        return afps_server_submit_pinned(self.srv, xyz.ctypes.data, xyz.shape[0], tag)

    def cancel(self, tag: int) -> int:
        """Withdraw a queued or admitted request (0, or AFPS_ERR_INVALID_ARG)."""
        return afps_server_cancel(self.srv, tag)

    def step(self) -> int:
        rc = afps_server_step(self.srv)
        if rc < 0:
            raise AfpsError(rc, afps_last_error(self.sampler.ctx))
        return rc

    def poll(self, copy: bool = True):
        """Finished requests.  copy=False: their indices are views of the
        runtime's result slots, valid until the next poll (no copy)."""
        n = afps_server_poll(self.srv, self._buf, len(self._buf))
        if n < 0:
            raise AfpsError(n, "afps_server_poll failed")
        if n == 0:
            return []
        rows = self._rows[:n]
        nl = rows["n_levels"].tolist()
        counts = [c[:k] for c, k in zip(rows["count"].tolist(), nl)]
        return [ServerResult(*f, copy=copy) for f in
                zip(rows["tag"].tolist(), rows["status"].tolist(), counts,
                    rows["indices"].tolist(), rows["submit_ms"].tolist(),
                    rows["admit_ms"].tolist(), rows["done_ms"].tolist())]

    def stats(self):
        q, f, u = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        afps_server_stats(self.srv, ctypes.byref(q), ctypes.byref(f), ctypes.byref(u))
        return q.value, f.value, u.value

    def clock_ms(self) -> float:
        return afps_server_clock_ms(self.srv)
