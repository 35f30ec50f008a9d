"""Routing a stream of serving requests over independent replicas.

Clouds are independent (Sec. III-B), so the serving runtime scales out by
replicas: one serving runtime (afps_server_*) per GPU, and a front-end that
only decides where each frame goes and collects the results; replicas never
exchange data.

- `ReplicaRouter` is the front-end policy over any objects with the `Server`
  interface (submit / submit_pinned / step / poll / stats / cancel /
  clock_ms): a frame goes to the replica with the fewest points outstanding
  (submitted and not yet returned), ties to the lowest index; a replica whose
  queue is full is skipped.  `poisson_run` (serving.py) drives it like one
  server.
- `RemoteReplica` / `replica_loop` put a replica in another process (one
  process per GPU) behind torch.distributed point-to-point messages on the
  host (gloo): each front-end step sends a replica its new frames and
  cancellations, the replica submits them, runs one step of its own server
  and answers with the finished results and its counts.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

ERR_INVALID_ARG = -1  # AFPS_ERR_INVALID_ARG
ERR_BUSY = -8         # AFPS_ERR_BUSY


@dataclass
class RoutedResult:
    """A finished request as the front-end returns it: per-level frame
    indices, the replica that served it, and times on the front-end's clock
    (the first replica's)."""
    tag: int
    status: int
    levels: list
    replica: int
    submit_ms: float
    admit_ms: float
    done_ms: float


class ReplicaRouter:
    """Least-outstanding-points routing over replicas (see module doc)."""

    def __init__(self, replicas):
        self.replicas = list(replicas)
        if not self.replicas:
            raise ValueError("ReplicaRouter needs at least one replica")
        n = len(self.replicas)
        self.owner = {}             # tag -> (replica, points) while outstanding
        self.points = [0] * n       # points outstanding per replica
        self.requests = [0] * n     # requests outstanding per replica
        self.routed = [0] * n       # frames ever sent to each replica
        # each replica's clock against the first one's, so that results
        # from every replica are reported on one clock
        base = self.replicas[0].clock_ms()
        self.offset = [r.clock_ms() - base for r in self.replicas]

    def _order(self):
        return sorted(range(len(self.replicas)), key=lambda i: (self.points[i], i))

    def _submit(self, xyz, tag: int, pinned: bool) -> int:
        if tag in self.owner:
            raise ValueError(f"tag {tag} is already outstanding")
        n = int(np.shape(xyz)[0])
        rc = ERR_BUSY
        for i in self._order():
            r = self.replicas[i]
            rc = (r.submit_pinned if pinned else r.submit)(xyz, tag)
            if rc == 0:
                self.owner[tag] = (i, n)
                self.points[i] += n
                self.requests[i] += 1
                self.routed[i] += 1
                return 0
            if rc != ERR_BUSY:
                return rc  # an error that another replica would repeat
        return rc  # every queue is full: the caller retries later

    def submit(self, xyz: np.ndarray, tag: int) -> int:
        return self._submit(xyz, tag, False)

    def submit_pinned(self, xyz: np.ndarray, tag: int) -> int:
        return self._submit(xyz, tag, True)

    def _release(self, tag: int):
        i, n = self.owner.pop(tag)
        self.points[i] -= n
        self.requests[i] -= 1

    def cancel(self, tag: int) -> int:
        if tag not in self.owner:
            return ERR_INVALID_ARG
        i, _ = self.owner[tag]
        rc = self.replicas[i].cancel(tag)
        if rc == 0:  # a cancelled request is never returned by poll
            self._release(tag)
        return rc

    def step(self) -> int:
        return sum(r.step() for r in self.replicas)

    def poll(self, copy: bool = True):
        """Finished requests of every replica (always copied: a replica's
        result slots are reused at its next poll)."""
        out = []
        for i, r in enumerate(self.replicas):
            off = self.offset[i]
            for res in r.poll():
                if res.tag in self.owner:
                    self._release(res.tag)
                out.append(RoutedResult(res.tag, res.status, list(res.levels), i,
                                        res.submit_ms - off, res.admit_ms - off,
                                        res.done_ms - off))
        return out

    def stats(self):
        q = f = u = 0
        for r in self.replicas:
            a, b, c = r.stats()
            q, f, u = q + a, f + b, u + c
        return q, f, u

    def clock_ms(self) -> float:
        return self.replicas[0].clock_ms()


# ------------------------------------------------------------ other processes
@dataclass
class _Result:
    tag: int
    status: int
    levels: list
    submit_ms: float
    admit_ms: float
    done_ms: float


@dataclass
class RemoteReplica:
    """The front-end's handle on a replica running `replica_loop` in process
    `rank`.  Frames are buffered until the next `step`, which exchanges one
    message each way; result times are taken on this process's clock (submit
    when queued here, done when received).  A cancelled request's result is
    dropped if the replica had already finished it."""
    rank: int
    group: object = None
    _frames: list = field(default_factory=list)
    _cancels: list = field(default_factory=list)
    _results: list = field(default_factory=list)
    _submit_ms: dict = field(default_factory=dict)
    _cancelled: set = field(default_factory=set)
    _stats: tuple = (0, 0, 0)
    _t0: float = field(default_factory=time.perf_counter)
    max_queued: int = 4096

    def clock_ms(self) -> float:
        return (time.perf_counter() - self._t0) * 1e3

    def submit(self, xyz, tag: int) -> int:
        if len(self._frames) + self._stats[0] >= self.max_queued:
            return ERR_BUSY
        self._frames.append((int(tag), np.ascontiguousarray(xyz, dtype=np.float32)))
        self._submit_ms[int(tag)] = self.clock_ms()
        return 0

    submit_pinned = submit  # the frame travels in the message either way

    def cancel(self, tag: int) -> int:
        for j, (t, _) in enumerate(self._frames):
            if t == tag:  # not sent yet
                del self._frames[j]
                self._submit_ms.pop(tag, None)
                return 0
        for j, r in enumerate(self._results):
            if r.tag == tag:  # finished, not yet polled
                del self._results[j]
                return 0
        self._cancels.append(int(tag))
        self._cancelled.add(int(tag))  # its result is dropped if it still comes
        return 0

    def step(self) -> int:
        import torch.distributed as dist
        msg = ("step", self._frames, self._cancels)
        self._frames, self._cancels = [], []
        dist.send_object_list([msg], dst=self.rank, group=self.group)
        reply = [None]
        dist.recv_object_list(reply, src=self.rank, group=self.group)
        advanced, results, self._stats = reply[0]
        now = self.clock_ms()
        for tag, status, levels, cancelled in results:
            sub = self._submit_ms.pop(tag, now)
            if cancelled or tag in self._cancelled:
                self._cancelled.discard(tag)
                continue
            self._results.append(_Result(tag, status, levels, sub, sub, now))
        return advanced

    def poll(self, copy: bool = True):
        out, self._results = self._results, []  # received by message: copies already
        return out

    def stats(self):
        return self._stats

    def close(self):
        import torch.distributed as dist
        dist.send_object_list([("stop", [], [])], dst=self.rank, group=self.group)


def replica_loop(server, src: int = 0, group=None) -> int:
    """Serve the front-end at rank `src` until it says stop: per message,
    submit its frames (a full queue keeps them for the next message), apply
    its cancellations, run one step and answer with the finished results
    (tag, status, levels, cancelled) and (queued, in-flight, arena bytes).
    Returns the number of requests served."""
    import torch.distributed as dist
    backlog = []
    served = 0
    while True:
        msg = [None]
        dist.recv_object_list(msg, src=src, group=group)
        kind, frames, cancels = msg[0]
        if kind == "stop":
            return served
        backlog.extend(frames)
        done = []
        for tag in cancels:
            before = len(backlog)
            backlog = [(t, x) for (t, x) in backlog if t != tag]
            if len(backlog) < before or server.cancel(tag) == 0:
                done.append((tag, ERR_INVALID_ARG, [], True))
        keep = []
        for tag, xyz in backlog:
            if keep or server.submit(xyz, tag) != 0:
                keep.append((tag, xyz))  # in order: once one waits, the rest wait
        backlog = keep
        advanced = server.step()
        for r in server.poll():
            done.append((r.tag, r.status, [np.asarray(v) for v in r.levels], False))
            served += 1
        q, f, u = server.stats()
        dist.send_object_list([(advanced, done, (q + len(backlog), f, u))], dst=src, group=group)
