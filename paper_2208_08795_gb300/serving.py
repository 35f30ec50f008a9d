"""Driving the serving runtime with a Poisson arrival stream.

`poisson_run` submits frames at exponentially spaced arrival times (a Poisson
process of the given rate), keeps calling `Server.step` and `Server.poll`,
and reports latency from each request's scheduled arrival to its completion
(queueing included) and the achieved frame rate.
"""
from __future__ import annotations

import time

import numpy as np


def poisson_arrivals(rate_hz: float, n: int, seed: int) -> np.ndarray:
    """Arrival times in ms of n requests of a Poisson process."""
    g = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(g.exponential(1000.0 / rate_hz, n))


def poisson_run(server, frames, rate_hz: float, n_requests: int, seed: int = 0,
                keep_results: bool = False, max_wall_s: float = 60.0, pinned: bool = False):
    """pinned=True: `frames` lie in page-locked memory and are submitted
    without a copy (Server.submit_pinned); they outlive the run."""
    arrivals = poisson_arrivals(rate_hz, n_requests, seed)
    submit = server.submit_pinned if pinned else server.submit
    t0 = server.clock_ms()
    done = {}
    i = 0
    steps = advanced = 0
    deadline = time.perf_counter() + max_wall_s
    while len(done) < n_requests:
        now = server.clock_ms() - t0
        while i < n_requests and arrivals[i] <= now:
            rc = submit(frames[i % len(frames)], i)
            if rc != 0:
                break  # queue full: retry on the next turn
            i += 1
        a = server.step()
        if a > 0:
            steps += 1
            advanced += a
        for r in server.poll(copy=keep_results):  # without a copy: views valid until the next poll
            done[r.tag] = r
        if a == 0 and i < n_requests and not server.stats()[1]:
            # idle: wait for the next arrival
            wait = arrivals[i] - (server.clock_ms() - t0)
            if wait > 0.2:
                time.sleep(min(wait, 5.0) / 1000.0 * 0.5)
        if time.perf_counter() > deadline:
            raise TimeoutError(f"serving run did not finish: {len(done)}/{n_requests} done")
    lat = np.array([done[t].done_ms - (t0 + arrivals[t]) for t in range(n_requests)])
    first, last = t0 + arrivals[0], max(r.done_ms for r in done.values())
    out = {
        "offered_frames_per_s": rate_hz,
        "achieved_frames_per_s": n_requests / ((last - first) / 1000.0),
        "requests": n_requests,
        "p50_ms": float(np.percentile(lat, 50)),
        "p99_ms": float(np.percentile(lat, 99)),
        "mean_ms": float(lat.mean()),
        "steps": steps,
        "mean_requests_per_step": advanced / max(steps, 1),
    }
    if keep_results:
        out["results"] = done
    return out
