"""Serving runtime: continuous batching of chained requests
16384 -> 4096 -> 1024 -> 256 (NPDU-AFPS, M = 32, k = 16) on LiDAR-like
frames.  Every result must equal the oracle's chained sampling and the same
frame served alone, whatever else shares the GPU steps."""
import numpy as np
import pytest

import oracle
from paper_2208_08795_gb300 import afps as B
from paper_2208_08795_gb300 import build as build_mod
from paper_2208_08795_gb300 import serving, synth

pytestmark = pytest.mark.gpu

LEVELS = [16384, 4096, 1024, 256]


@pytest.fixture(scope="module")
def sampler():
    build_mod.build()
    s = B.Sampler(0)
    yield s
    s.close()


def drain(server, n):
    done = {}
    while len(done) < n:
        server.step()
        for r in server.poll():
            done[r.tag] = r
    return done


@pytest.mark.parametrize("levels_per_step", [0, 1, 2])
def test_mixed_stream_matches_oracle_and_alone(sampler, levels_per_step):
    frames = [synth.lidar_frame(s) for s in range(10)]
    # a budget for about three requests at once: the rest waits for admission
    srv = B.Server(sampler, LEVELS, 32, 16, hbm_budget_bytes=3_000_000,
                   levels_per_step=levels_per_step)
    try:
        for t, f in enumerate(frames):
            assert srv.submit(f, t) == 0
        q, inflight, used = srv.stats()
        assert q == len(frames)
        srv.step()
        q, inflight, used = srv.stats()
        assert 1 <= inflight < len(frames) and q == len(frames) - inflight and used <= 3_000_000
        mixed = drain(srv, len(frames))
    finally:
        srv.close()
    for t, f in enumerate(frames):
        ref = oracle.chain(f, LEVELS, 32, 16)
        for l in range(len(LEVELS)):
            assert np.array_equal(mixed[t].levels[l], ref[l]), (t, l)
        assert mixed[t].submit_ms <= mixed[t].admit_ms <= mixed[t].done_ms
    alone = B.Server(sampler, LEVELS, 32, 16, hbm_budget_bytes=3_000_000)
    try:
        for t in (0, 7):
            assert alone.submit(frames[t], 100 + t) == 0
            r = drain(alone, 1)[100 + t]
            for l in range(len(LEVELS)):
                assert np.array_equal(r.levels[l], mixed[t].levels[l]), (t, l)
    finally:
        alone.close()


def test_poisson_stream_completes(sampler):
    frames = [synth.lidar_frame(s) for s in range(4)]
    srv = B.Server(sampler, LEVELS, 32, 16, hbm_budget_bytes=64 << 20)
    try:
        res = serving.poisson_run(srv, frames, rate_hz=2000.0, n_requests=60, seed=1,
                                  keep_results=True)
    finally:
        srv.close()
    assert res["requests"] == 60 and res["p99_ms"] >= res["p50_ms"] > 0
    ref0 = oracle.chain(frames[0], LEVELS, 32, 16)
    for t in (0, 4, 8):
        for l in range(len(LEVELS)):
            assert np.array_equal(res["results"][t].levels[l], ref0[l])


def test_submit_rejects_bad_frames(sampler):
    srv = B.Server(sampler, LEVELS, 32, 16, hbm_budget_bytes=3_000_000, max_queued=1)
    try:
        small = synth.uniform_cloud(1, 1000)
        assert srv.submit(small, 0) == B.AFPS_ERR_INVALID_ARG  # fewer points than level 0
        f = synth.lidar_frame(3)
        assert srv.submit(f, 1) == 0
        assert srv.submit(f, 2) == B.AFPS_ERR_BUSY  # queue of one is full
        drain(srv, 1)
    finally:
        srv.close()


def test_host_pool_recycles_blocks(sampler):
    """Queued frames wait in a page-locked pool of two frames' size: a third
    submit is refused until admission has copied a frame out, and the blocks
    are reused for a stream of frames without changing any result."""
    frames = [synth.lidar_frame(s) for s in range(6)]
    n_max = max(f.shape[0] for f in frames)
    pool = 2 * ((12 * n_max + 47) // 48 * 48)
    srv = B.Server(sampler, LEVELS, 32, 16, hbm_budget_bytes=64 << 20, host_pool_bytes=pool)
    try:
        assert srv.submit(frames[0], 0) == 0
        assert srv.submit(frames[1], 1) == 0
        assert srv.submit(frames[2], 2) == B.AFPS_ERR_BUSY  # pool holds two frames
        done = {}
        t = 2
        for _ in range(10_000):
            if t < len(frames) and srv.submit(frames[t], t) == 0:
                t += 1
            srv.step()
            for r in srv.poll():
                done[r.tag] = r
            if len(done) == len(frames):
                break
    finally:
        srv.close()
    assert sorted(done) == list(range(len(frames)))
    for t in (0, 3, 5):
        ref = oracle.chain(frames[t], LEVELS, 32, 16)
        for l in range(len(LEVELS)):
            assert np.array_equal(done[t].levels[l], ref[l]), (t, l)


def test_pinned_frames_without_copy(sampler):
    """submit_pinned: page-locked frames are read in place at admission; a
    Poisson stream over them matches the oracle, and pageable memory is
    refused."""
    torch = pytest.importorskip("torch")
    frames = [synth.lidar_frame(s) for s in range(4)]
    pinned = [torch.from_numpy(f).pin_memory().numpy() for f in frames]
    srv = B.Server(sampler, LEVELS, 32, 16, hbm_budget_bytes=64 << 20)
    try:
        assert srv.submit_pinned(frames[0], 0) == B.AFPS_ERR_INVALID_ARG  # pageable
        res = serving.poisson_run(srv, pinned, rate_hz=4000.0, n_requests=40, seed=2,
                                  keep_results=True, pinned=True)
    finally:
        srv.close()
    for t in (0, 1, 2, 3, 17):
        ref = oracle.chain(frames[t % 4], LEVELS, 32, 16)
        for l in range(len(LEVELS)):
            assert np.array_equal(res["results"][t].levels[l], ref[l]), (t, l)


def test_device_timeouts_of_both_streams_reach_the_callers_context():
    """By default the server alternates its steps between the caller's stream
    (and context) and a second stream with a second context of its own; a
    device error on either must reach the caller's context, whose afps_sync
    reports it.  The copy-stall fault flag (host-side injection: each stage-in
    waits 1 ms for a copy that is never issued, then the kernels stop) makes
    every step's sampling time out; the first step runs on the caller's
    stream, the second on the server's own.  A fresh context serves the same
    frame exactly afterwards."""
    build_mod.build()
    frames = [synth.lidar_frame(s) for s in range(2)]
    s = B.Sampler(0, timeout_ns=1_000_000, flags=B.AFPS_FLAG_TEST_STALL_COPY)
    srv = B.Server(s, LEVELS, 32, 16, hbm_budget_bytes=64 << 20)
    try:
        for t, f in enumerate(frames):
            assert srv.submit(f, t) == 0
            drain(srv, 1)  # one step (admission and every level), this frame only
            with pytest.raises(B.AfpsError) as ei:
                s.sync()
            assert ei.value.code == B.AFPS_ERR_TIMEOUT, t
        s.sync()  # reported once, then cleared
    finally:
        srv.close()
        s.close()
    fresh = B.Sampler(0)
    srv = B.Server(fresh, LEVELS, 32, 16, hbm_budget_bytes=64 << 20)
    try:
        assert srv.submit(frames[1], 7) == 0
        r = drain(srv, 1)[7]
        ref = oracle.chain(frames[1], LEVELS, 32, 16)
        for l in range(len(LEVELS)):
            assert np.array_equal(r.levels[l], ref[l]), l
    finally:
        srv.close()
        fresh.close()


def test_cancel_queued_and_admitted(sampler):
    """Withdrawing a queued and an admitted request: the others still match
    the oracle, the withdrawn ones never come back, and all device memory
    and result slots are returned."""
    frames = [synth.lidar_frame(s) for s in range(8)]
    srv = B.Server(sampler, LEVELS, 32, 16, hbm_budget_bytes=3_000_000,  # about three at once
                   levels_per_step=1)
    try:
        for t, f in enumerate(frames):
            assert srv.submit(f, t) == 0
        srv.step()  # admits the first few and advances them one level
        assert srv.cancel(1) == 0  # admitted
        assert srv.cancel(6) == 0  # still queued
        assert srv.cancel(6) == B.AFPS_ERR_INVALID_ARG  # already withdrawn
        assert srv.cancel(99) == B.AFPS_ERR_INVALID_ARG
        done = drain(srv, len(frames) - 2)
        for _ in range(4):
            srv.step()
            assert not srv.poll()
        q, inflight, used = srv.stats()
        assert (q, inflight, used) == (0, 0, 0)
    finally:
        srv.close()
    assert sorted(done) == [t for t in range(8) if t not in (1, 6)]
    for t in (0, 2, 7):
        ref = oracle.chain(frames[t], LEVELS, 32, 16)
        for l in range(len(LEVELS)):
            assert np.array_equal(done[t].levels[l], ref[l]), (t, l)


def test_router_over_two_replicas(sampler):
    """Two serving runtimes behind the least-outstanding router (one per GPU
    in a deployment; both on the one GPU here, each with its own context and
    stream): every result equals the oracle's chained sampling, both
    replicas serve, and all times are on the first replica's clock."""
    from paper_2208_08795_gb300 import routing
    s2 = B.Sampler(0)
    reps = [B.Server(sampler, LEVELS, 32, 16, hbm_budget_bytes=64 << 20),
            B.Server(s2, LEVELS, 32, 16, hbm_budget_bytes=64 << 20)]
    try:
        router = routing.ReplicaRouter(reps)
        frames = [synth.lidar_frame(100 + s) for s in range(6)]
        refs = [oracle.chain(f, LEVELS, 32, 16) for f in frames]
        # a burst: the frames are outstanding together, so both replicas get some
        for t, f in enumerate(frames):
            assert router.submit(f, 100 + t) == 0
        burst = {}
        while len(burst) < len(frames):
            router.step()
            burst.update({r.tag: r for r in router.poll()})
        assert {r.replica for r in burst.values()} == {0, 1}
        for t, r in burst.items():
            for l in range(len(LEVELS)):
                assert np.array_equal(r.levels[l], refs[t - 100][l]), (t, l)
        # a Poisson stream through the router
        out = serving.poisson_run(router, frames, rate_hz=4000.0, n_requests=24, seed=3,
                                  keep_results=True)
        res = out["results"]
        assert sorted(res) == list(range(24))
        for t, r in res.items():
            assert r.status == 0
            for l in range(len(LEVELS)):
                assert np.array_equal(r.levels[l], refs[t % len(frames)][l]), (t, l)
            assert r.submit_ms <= r.admit_ms <= r.done_ms <= router.clock_ms() + 1.0
        assert sum(router.routed) == 30
        assert router.points == [0, 0] and not router.owner
    finally:
        for r in reps:
            r.close()
        s2.close()
