"""afps_sample_batched_noalloc: the batched sampler for callers that cannot
allocate device memory (a plugin whose host owns every allocation, a process
under a fixed memory pool or budget, a real-time loop that must not take the
allocator's locks).  It keeps its work-item table in a static device array.

Checked through the C ABI against the existing batched entry point, on two
calls in a row with different batches, so a stale table from the first call
would show in the second.  This file is collected last on purpose."""
import numpy as np
import pytest
import torch

from paper_2208_08795_gb300 import afps as B
from paper_2208_08795_gb300 import build as build_mod
from paper_2208_08795_gb300 import synth

pytestmark = pytest.mark.gpu


def _batches():
    objs = synth.object_batch(1, 12, 2048)
    first = (objs[:8] + [synth.slab_cloud(4, 9000), synth.uniform_cloud(8, 300)],
             [512] * 8 + [2000, 100], [1, 4, 16, 32, 32, 8, 2, 1, 2, 3],
             [0, 8, 16, 16, 0, 0, 4, 9, 0, 5])
    second = (objs[8:] + [synth.slab_cloud(5, 20000)], [512] * 4 + [3000],
              [32, 32, 4, 1, 1], [16, 0, 0, 0, 0])
    return first, second


def _existing(S, x, ba):
    out = S.sample_batched(x, ba)
    S.sync()
    return out.cpu().numpy()


def test_noalloc_matches_batched_on_two_calls():
    build_mod.build()
    L = B.load()
    S = B.Sampler(0)
    try:
        stream = torch.cuda.current_stream().cuda_stream
        for clouds, Cs, Ms, ks in _batches():
            xyz, off = synth.pack(clouds)
            x = torch.from_numpy(xyz).cuda()
            ba = B.BatchArgs(off, Cs, Ms, ks, 0)
            ref = _existing(S, x, ba)
            out = torch.full((ba.total_out,), -1, dtype=torch.int32, device="cuda")
            rc = L.afps_sample_batched_noalloc(x.data_ptr(), *ba.args(), out.data_ptr(), stream)
            torch.cuda.synchronize()
            assert rc == B.AFPS_OK
            assert np.array_equal(out.cpu().numpy(), ref)
    finally:
        S.close()


def test_noalloc_rejects_batches_beyond_its_scratch():
    build_mod.build()
    L = B.load()
    n = B.AFPS_NOALLOC_MAX_ITEMS + 1  # one sector too many
    x = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    ba = B.BatchArgs([0, n], n, n, 0, 0)
    rc = L.afps_sample_batched_noalloc(x.data_ptr(), *ba.args(), out.data_ptr(),
                                       torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert rc == B.AFPS_ERR_SCRATCH_TOO_SMALL
    assert int((out != -1).sum()) == 0  # nothing launched, nothing written


def test_noalloc_refuses_stream_capture():
    """On a stream that is capturing a CUDA graph the call does nothing and
    returns AFPS_ERR_INVALID_ARG (a captured upload would replay from the
    static host copy after later calls had overwritten it); the capture
    itself is unharmed and the next call outside it works."""
    build_mod.build()
    L = B.load()
    clouds = synth.object_batch(2, 4, 2048)
    xyz, off = synth.pack(clouds)
    x = torch.from_numpy(xyz).cuda()
    ba = B.BatchArgs(off, 512, 32, 16, 0)
    out = torch.full((ba.total_out,), -1, dtype=torch.int32, device="cuda")
    y = torch.zeros(16, device="cuda")
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        g.capture_begin()
        rc = L.afps_sample_batched_noalloc(x.data_ptr(), *ba.args(), out.data_ptr(),
                                           side.cuda_stream)
        y.add_(1.0)  # the capture records this
        g.capture_end()
    assert rc == B.AFPS_ERR_INVALID_ARG
    g.replay()
    torch.cuda.synchronize()
    assert float(y[0]) == 1.0 and int((out != -1).sum()) == 0
    rc = L.afps_sample_batched_noalloc(x.data_ptr(), *ba.args(), out.data_ptr(),
                                       torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert rc == B.AFPS_OK
    S = B.Sampler(0)
    try:
        assert np.array_equal(out.cpu().numpy(), _existing(S, x, ba))
    finally:
        S.close()
