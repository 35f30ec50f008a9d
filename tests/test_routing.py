"""Routing serving requests over replicas (one serving runtime per GPU), on
CPU: the replicas here are stand-ins with the serving runtime's interface
whose results come from the oracle's chained sampling, so what is checked is
the front-end -- where frames go, that every result comes back once with its
own tag, cancellation, a full queue, one clock for all replicas, and the
same over gloo with replicas in other processes."""
import os
import socket
import time

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_2208_08795_gb300 import routing, serving, synth

LEVELS = [128, 32]
M, K = 4, 8


class FakeServer:
    """Queue, admit `per_step` requests a step, finish them one step later."""

    def __init__(self, per_step=2, max_queued=64, clock_offset_ms=0.0):
        self.per_step, self.max_queued = per_step, max_queued
        self.queue, self.running, self.done = [], [], []
        self.t0 = time.perf_counter() - clock_offset_ms / 1e3
        self.steps = 0

    def clock_ms(self):
        return (time.perf_counter() - self.t0) * 1e3

    def submit(self, xyz, tag):
        if len(self.queue) >= self.max_queued:
            return routing.ERR_BUSY
        self.queue.append((tag, np.array(xyz, dtype=np.float32), self.clock_ms()))
        return 0

    submit_pinned = submit

    def cancel(self, tag):
        for lst in (self.queue, self.running):
            for j, item in enumerate(lst):
                if item[0] == tag:
                    del lst[j]
                    return 0
        return routing.ERR_INVALID_ARG

    def step(self):
        now = self.clock_ms()
        finished = 0
        for tag, xyz, sub, adm in self.running:
            self.done.append(serving_result(tag, oracle.chain(xyz, LEVELS, M, K), sub, adm, now))
            finished += 1
        self.running = [(t, x, s, now) for (t, x, s) in self.queue[:self.per_step]]
        self.queue = self.queue[self.per_step:]
        self.steps += 1
        return finished * len(LEVELS) + len(self.running)

    def poll(self, copy=True):
        out, self.done = self.done, []
        return out

    def stats(self):
        return len(self.queue), len(self.running), 0


class serving_result:
    def __init__(self, tag, levels, sub, adm, done):
        self.tag, self.status, self.levels = tag, 0, levels
        self.submit_ms, self.admit_ms, self.done_ms = sub, adm, done


def frames(n, seed=0):
    g = np.random.default_rng(seed)
    return [synth.object_batch(seed + i, 1, int(g.integers(300, 700)))[0] for i in range(n)]


def drain(router, n, max_steps=10000):
    got = {}
    for _ in range(max_steps):
        router.step()
        for r in router.poll():
            assert r.tag not in got, "a result came back twice"
            got[r.tag] = r
        if len(got) >= n:
            break
    return got


def check(got, fr):
    for t, f in enumerate(fr):
        ref = oracle.chain(f, LEVELS, M, K)
        for l in range(len(LEVELS)):
            assert np.array_equal(got[t].levels[l], ref[l]), (t, l)


def test_least_outstanding_points_routing():
    reps = [FakeServer(), FakeServer(), FakeServer()]
    router = routing.ReplicaRouter(reps)
    fr = frames(12)
    for t, f in enumerate(fr):
        assert router.submit(f, t) == 0
        # the frame went to a replica that had no more outstanding points than any other
    owners = [router.owner[t][0] for t in range(3)]
    assert owners == [0, 1, 2]  # idle replicas: ties to the lowest index
    assert sum(router.points) == sum(f.shape[0] for f in fr)
    assert max(router.points) - min(router.points) <= max(f.shape[0] for f in fr)
    got = drain(router, len(fr))
    check(got, fr)
    assert all(n > 0 for n in router.routed)
    assert router.points == [0, 0, 0] and router.requests == [0, 0, 0] and not router.owner
    assert {r.replica for r in got.values()} == {0, 1, 2}


def test_full_queue_goes_to_the_next_replica_and_busy_when_all_full():
    a, b = FakeServer(max_queued=0), FakeServer(max_queued=2)
    router = routing.ReplicaRouter([a, b])
    fr = frames(3, seed=5)
    assert router.submit(fr[0], 0) == 0 and router.owner[0][0] == 1  # a is full
    assert router.submit(fr[1], 1) == 0
    assert router.submit(fr[2], 2) == routing.ERR_BUSY  # both full: retry later
    assert 2 not in router.owner and router.routed == [0, 2]
    got = drain(router, 2)
    assert sorted(got) == [0, 1]
    assert router.submit(fr[2], 2) == 0  # room again
    check({**got, **drain(router, 1)}, fr)


def test_cancel_duplicate_tags_and_one_clock():
    reps = [FakeServer(), FakeServer(clock_offset_ms=5000.0)]
    router = routing.ReplicaRouter(reps)
    assert abs(router.offset[1] - 5000.0) < 50.0
    fr = frames(6, seed=9)
    for t, f in enumerate(fr):
        assert router.submit(f, t) == 0
    with pytest.raises(ValueError):
        router.submit(fr[0], 0)
    assert router.cancel(3) == 0 and 3 not in router.owner
    assert router.cancel(3) == routing.ERR_INVALID_ARG
    assert router.cancel(99) == routing.ERR_INVALID_ARG
    got = drain(router, 5)
    assert sorted(got) == [0, 1, 2, 4, 5]  # the cancelled request never comes back
    now = router.clock_ms()
    for r in got.values():  # every replica's times on the first replica's clock
        assert 0.0 <= r.submit_ms <= r.admit_ms <= r.done_ms <= now + 1.0
    assert sum(router.points) == 0


def test_poisson_run_drives_the_router():
    reps = [FakeServer(per_step=1), FakeServer(per_step=3)]
    router = routing.ReplicaRouter(reps)
    fr = frames(4, seed=2)
    out = serving.poisson_run(router, fr, rate_hz=2000.0, n_requests=20, seed=1,
                              keep_results=True, max_wall_s=60.0)
    assert out["requests"] == 20 and len(out["results"]) == 20
    for t, r in out["results"].items():
        ref = oracle.chain(fr[t % len(fr)], LEVELS, M, K)
        assert all(np.array_equal(r.levels[l], ref[l]) for l in range(len(LEVELS)))
    assert out["p99_ms"] >= out["p50_ms"] >= 0.0
    # (which replicas serve depends on how the arrivals overlap: an idle
    # router sends every frame to replica 0; the order is checked above)
    assert sum(router.routed) == 20 and not router.owner


# ------------------------------------------------- replicas in other processes
def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _node(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        if rank != 0:
            q.put(("served", rank, routing.replica_loop(FakeServer(per_step=rank))))
            return
        remotes = [routing.RemoteReplica(r) for r in range(1, world)]
        router = routing.ReplicaRouter([FakeServer(per_step=2)] + remotes)
        fr = frames(16, seed=11)
        for t, f in enumerate(fr):
            assert router.submit(f, t) == 0
        assert router.cancel(15) == 0  # still buffered at the front-end
        got = drain(router, 15)
        for rr in remotes:
            rr.close()
        res = {t: [np.asarray(v) for v in r.levels] for t, r in got.items()}
        q.put(("front", sorted(got), res, router.routed))
    finally:
        dist.destroy_process_group()


def test_replicas_in_other_processes_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 3
    procs = [ctx.Process(target=_node, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    msgs = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    front = next(m for m in msgs if m[0] == "front")
    _, tags, res, routed = front
    assert tags == list(range(15))  # the cancelled frame 15 never comes back
    fr = frames(16, seed=11)
    for t in tags:
        ref = oracle.chain(fr[t], LEVELS, M, K)
        assert all(np.array_equal(res[t][l], ref[l]) for l in range(len(LEVELS))), t
    served = {m[1]: m[2] for m in msgs if m[0] == "served"}
    assert set(served) == {1, 2} and all(v > 0 for v in served.values())
    assert routed[1] > 0 and routed[2] > 0
