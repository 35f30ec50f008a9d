"""Benchmark: NPDU-AFPS vs plain FPS on one GB300, clouds/s and p99 ms.

Workload (one step): a batch of 32 object-scale clouds of 2048 points
(2-5 primitive surfaces, jitter 0.005, unit ball, sorted by x), C = 512
samples each, NPDU-AFPS with M = 32 sectors and window k = 16, all clouds in
one batched call (graph-replayed).  Beside it, in the same run: plain FPS
(M = 1, no NPDU) on the same batch, the sweep M in {1, 4, 16, 32} with NPDU
off/on, the end-to-end time through host buffers, the roofline of the
sampling kernel, and the CPU oracle on the host's cores.

Timing.  Throughput (`value`, `ms_per_step`): K steps between two CUDA
events, step i on stream i mod S (S = 8 by default: the steps of a stream
run back to back, the streams side by side, as independent batches would),
each step on the next of R resident copies of the batch (R copies span twice
the L2), so every timed step reads cold points without a flush; a
fixed-length sleep kernel ahead of the first event holds the streams while
the host enqueues the K steps, so the host's call rate does not set the pace
(the host path is what `e2e` measures).  `one_stream` repeats it on a single
stream.  Latency (`p50_ms`, `p99_ms`): isolated steps, each after a 256 MB
write that flushes the L2, with its own pair of events.  The CPU oracle runs
one worker process per host core.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun each rank samples its own
batch (weak scaling, no collective on the data path); the time is the max
over ranks.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "clouds/s & p99 ms, NPDU-AFPS vs plain FPS on 1 GB300, indices = FP32 oracle"
UNIT = "clouds/s"
B_CLOUDS, N_POINTS, C_SAMPLES, M_SECTORS, K_WINDOW = 32, 2048, 512, 32, 16
WORKLOAD = (f"object batch {B_CLOUDS} x {N_POINTS} pts, C={C_SAMPLES}, "
            f"NPDU-AFPS M={M_SECTORS} k={K_WINDOW}")
L2_FLUSH_BYTES = 256 << 20
L2_BYTES = 129 << 20  # GB300 L2
FALLBACK_HBM_GBS = 6800.0


def k_rule(M: int) -> int:
    """NPDU window per sector count: k = 8 for M <= 8, 16 for M >= 16."""
    return 8 if M <= 8 else 16


# ------------------------------------------------------------------ ranks
def rank_info():
    r = int(os.environ.get("RANK", "0"))
    w = int(os.environ.get("WORLD_SIZE", "1"))
    lr = int(os.environ.get("LOCAL_RANK", "0"))
    return r, w, lr


def batch_seed(rank: int) -> int:
    """Each rank samples its own batch (weak scaling)."""
    return 1 + rank


def max_over_ranks(x: float, world: int, device=None) -> float:
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi sampled every 50 ms while the benchmark runs."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [l.strip().split(", ") for l in self.file.read().splitlines() if l.strip()]
        os.unlink(self.file.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for name, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ inputs
def make_batch(seed: int):
    from paper_2208_08795_gb300 import synth
    clouds = synth.object_batch(seed, B_CLOUDS, N_POINTS)
    xyz, off = synth.pack(clouds)
    return clouds, xyz, off


def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


# ------------------------------------------------------------------ CPU oracle
_ORACLE_WORK = None


def _oracle_init(clouds, C, M, k):
    global _ORACLE_WORK
    _ORACLE_WORK = (clouds, C, M, k)


def _oracle_chunk(lo: int, hi: int, reps: int):
    """Clouds [lo, hi) of the batch through the oracle, `reps` times; returns
    the last pass's indices."""
    import oracle
    clouds, C, M, k = _ORACLE_WORK
    out = None
    for _ in range(reps):
        out = [oracle.afps(clouds[i], C, M, k, 0) for i in range(lo, hi)]
    return out


class OraclePool:
    """The oracle, as it stands, over one batch on `procs` host cores: worker
    processes (started with spawn, so safe after CUDA use) that each hold the
    batch and run a contiguous chunk of its clouds.  Processes rather than
    threads: the oracle's Python wrapper holds the GIL for about a sixth of a
    call, which capped 16 threads at 1.3x one."""

    def __init__(self, clouds, C, M, k, procs: int):
        self.n, self.procs = len(clouds), max(1, min(procs, len(clouds)))
        self.pool = None
        if self.procs == 1:
            _oracle_init(clouds, C, M, k)
        else:
            import multiprocessing as mp
            self.pool = mp.get_context("spawn").Pool(self.procs, initializer=_oracle_init,
                                                     initargs=(clouds, C, M, k))

    def run(self, reps: int = 1):
        """The batch `reps` times; returns the last pass's indices per cloud."""
        if self.pool is None:
            return _oracle_chunk(0, self.n, reps)
        bounds = [(self.n * i // self.procs, self.n * (i + 1) // self.procs, reps)
                  for i in range(self.procs)]
        out = []
        for part in self.pool.starmap(_oracle_chunk, bounds, chunksize=1):
            out.extend(part)
        return out

    def close(self):
        if self.pool is not None:
            self.pool.close()
            self.pool.join()
            self.pool = None


def time_oracle(clouds, C, M, k, budget_s: float, procs: int):
    """The oracle as it stands on `procs` cores: whole batches, repeated for
    about budget_s.  Returns (clouds/s, batches, indices per cloud)."""
    pool = OraclePool(clouds, C, M, k, procs)
    try:
        outs = pool.run(1)  # starts the workers and warms the library
        t0 = time.perf_counter()
        pool.run(10)
        once = (time.perf_counter() - t0) / 10
        reps = max(1, min(100000, int(budget_s / max(once, 1e-6))))
        t0 = time.perf_counter()
        pool.run(reps)
        el = time.perf_counter() - t0
    finally:
        pool.close()
    return reps * len(clouds) / el, reps, outs


def cpu_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ------------------------------------------------------------------ GPU timing
def time_device(sampler, x, ba, out, steps: int, warmup: int, flush):
    """Per-step device time with CUDA events on the launching stream.  Each
    step is preceded (outside its events) by a 256 MB write that flushes L2
    and keeps the GPU busy while the host enqueues the step."""
    import torch
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        flush.zero_()
        sampler.sample_batched(x, ba, out=out, stream=stream)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    n0 = sampler.launch_count
    for i in range(steps):
        flush.zero_()
        evs[i][0].record(stream)
        sampler.sample_batched(x, ba, out=out, stream=stream)
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    sampler.sync()
    return [a.elapsed_time(b) for a, b in evs], sampler.launch_count - n0


def rotation(x, total_out: int, dev):
    """Copies of the batch in as many resident slots as cover twice the L2
    (points and outputs), so that a step that visits a slot for the first time
    in more than 2 x L2 of traffic reads its points from DRAM."""
    import torch
    slot_bytes = x.numel() * 4 + total_out * 4
    R = max(8, -(-2 * L2_BYTES // slot_bytes))
    xr = x.unsqueeze(0).repeat(R, *([1] * x.dim())).contiguous()
    outr = torch.full((R, total_out), -1, dtype=torch.int32, device=dev)
    return xr, outr


def time_stream(sampler, xr, outr, ba, steps: int, warmup: int, n_streams: int = 1):
    """Whole-job throughput: K steps issued through the C ABI
    (afps_sample_batched on a context without graphs: one direct kernel
    launch per step; hundreds of distinct graphs, one per slot, were measured
    to launch slower than that when queued), each on the next resident slot
    of the rotation.  Step i goes to stream i mod S: the steps of one stream
    run back to back, the S streams side by side (independent batches; a
    step's kernel leaves most of the GPU idle, so they overlap).  One pair of
    CUDA events on the launching stream brackets the K steps; every stream
    waits for the first event and the second waits for every stream.  Every
    slot is run once first (untimed); the timed steps start at the least
    recently used slot, so every one of them reads cold points.  Returns (ms
    per step, launches in the timed region, last slot used, enqueue
    information)."""
    import torch
    from paper_2208_08795_gb300 import afps as A
    fn = A.load().afps_sample_batched
    main = torch.cuda.current_stream()
    streams = [main] + [torch.cuda.Stream() for _ in range(n_streams - 1)]
    R = xr.shape[0]
    args = [(sampler.ctx, xr[i % R].data_ptr(), *ba.args(), outr[i % R].data_ptr(),
             streams[i % n_streams].cuda_stream) for i in range(R)]

    def call(i):
        if fn(*args[i % R]) != 0:
            raise A.AfpsError(-1, A.afps_last_error(sampler.ctx))

    for i in range(R):  # every slot once
        call(i)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(warmup):
        call(i)
    torch.cuda.synchronize()
    per_call = (time.perf_counter() - t0) / warmup
    # Hold the streams (a fixed-length sleep kernel before the first event)
    # while the K steps are enqueued, so that the GPU runs them without
    # waiting for the host, whose per-call cost does not set the pace.
    hold_s = min(3.0 * per_call * steps + 1e-3, 0.05)
    torch.cuda._sleep(int(hold_s * 2.07e9))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n0 = sampler.launch_count
    e0.record(main)
    for st in streams[1:]:
        st.wait_event(e0)
    t0 = time.perf_counter()
    for i in range(warmup, warmup + steps):
        call(i)
    for st in streams[1:]:
        ev = torch.cuda.Event()
        ev.record(st)
        main.wait_event(ev)
    e1.record(main)
    enqueue_s = time.perf_counter() - t0
    torch.cuda.synchronize()
    sampler.sync()
    info = {"host_enqueue_ms": round(enqueue_s * 1e3, 3), "hold_ms": round(hold_s * 1e3, 3),
            "enqueued_within_hold": enqueue_s < hold_s}
    return (e0.elapsed_time(e1) / steps, sampler.launch_count - n0, (warmup + steps - 1) % R,
            info)


def time_e2e_stream(sampler, xyz, ba, steps: int, warmup: int, expect, n_streams: int = 1):
    """End to end through the public API, pipelined: K calls of
    afps_sample_batched_host_async (a context without graphs: its kernels
    read the points from, and write the indices to, page-locked host memory
    over the C2C link), call i on stream i mod S, then one synchronisation of
    the device, timed on the host clock.  Step i reads input copy i mod R (R
    copies span twice the L2, so no step finds its points cached) and writes
    its own output buffer; every output is checked against `expect`
    afterwards.  Returns (ms per step, input bytes per step, output bytes per
    step)."""
    import torch
    from paper_2208_08795_gb300 import afps as A
    fn = A.load().afps_sample_batched_host_async
    streams = [torch.cuda.current_stream()] + [torch.cuda.Stream() for _ in range(n_streams - 1)]
    slot = xyz.nbytes + ba.total_out * 4
    R = max(8, -(-2 * L2_BYTES // slot))
    hx = torch.from_numpy(xyz).unsqueeze(0).repeat(R, 1, 1).pin_memory()
    ho = torch.full((warmup + steps, ba.total_out), -1, dtype=torch.int32).pin_memory()
    args = [(sampler.ctx, hx[i % R].data_ptr(), *ba.args(), ho[i].data_ptr(),
             streams[i % n_streams].cuda_stream) for i in range(warmup + steps)]

    def call(i):
        if fn(*args[i]) != 0:
            raise A.AfpsError(-1, A.afps_last_error(sampler.ctx))

    for i in range(warmup):
        call(i)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(warmup, warmup + steps):
        call(i)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / steps
    sampler.sync()
    if not bool((ho[warmup:] == torch.from_numpy(expect).unsqueeze(0)).all()):
        raise RuntimeError("an end-to-end step differs from the device path")
    return ms, xyz.nbytes, ba.total_out * 4


def time_e2e(sampler, h_xyz, ba, h_out, steps: int, warmup: int):
    """The C-ABI call afps_sample_batched_host on pinned host buffers: the
    host-to-device copy of the points, the sampling and the device-to-host copy
    of the indices are inside each timed call (which returns after the copy)."""
    import torch
    from paper_2208_08795_gb300 import afps as A
    fn = A.load().afps_sample_batched_host
    args = (sampler.ctx, h_xyz.ctypes.data, *ba.args(), h_out.ctypes.data,
            torch.cuda.current_stream().cuda_stream)
    for _ in range(warmup):
        if fn(*args) != 0:
            raise A.AfpsError(-1, A.afps_last_error(sampler.ctx))
    ts = []
    for _ in range(steps):
        t0 = time.perf_counter()
        fn(*args)
        ts.append((time.perf_counter() - t0) * 1e3)
    return ts


def _json_default(o):
    if isinstance(o, np.generic):
        return o.item()
    raise TypeError(f"not JSON serializable: {type(o).__name__}")


def pct(xs, q):
    return float(np.percentile(np.asarray(xs), q))


def npdu_work(out_idx, ba, k):
    """Algorithmic work of one batch: distance evaluations (window sizes, or
    whole sectors) and argmax compares, from the sector plan and the output."""
    evals = compares = 0
    for b in range(ba.B):
        N = int(ba.pt_off[b + 1] - ba.pt_off[b])
        C, M = int(ba.C[b]), int(ba.M[b])
        idx = out_idx[ba.out_off[b]:ba.out_off[b] + C]
        for s in range(M):
            lo, hi = s * N // M, (s + 1) * N // M
            o0, o1 = s * C // M, (s + 1) * C // M
            n = hi - lo
            compares += (o1 - o0 - 1) * n
            for p in idx[o0:o1 - 1] - lo:
                if k > 0:
                    evals += int(min(n - 1, p + (k - k // 2)) - max(0, p - k // 2) + 1)
                else:
                    evals += n
    return evals, compares


HEADLINE_KERNEL_SOURCES = ("afps_warp.cu", "afps_device.cuh", "afps_internal.h")


def kernel_source_hash() -> str:
    """Hash of the sources the headline kernel (afps_warp_kernel) is built from."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2208_08795_gb300", "csrc")
    for f in HEADLINE_KERNEL_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


# DRAM traffic of the headline kernel from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum per launch), valid only for the kernel sources it was
# taken on (their hash); otherwise reported as null.
NCU_TRAFFIC = {"source_hash": "86501c29aea197c6", "bytes_per_launch": 820224}
# warp instructions of one headline launch (ncu smsp__inst_executed.sum), same rule
NCU_INST = {"source_hash": "86501c29aea197c6", "warp_inst_per_launch": 925696}


# ------------------------------------------------------------------ other configs
def time_batch(sampler, x, ba, out, steps, warmup, flush):
    """Autotune (untimed), then per-step device time; returns (mean ms, p99 ms)."""
    sampler.autotune_batched(x, ba, out)
    sampler.sync()
    ms, _ = time_device(sampler, x, ba, out, steps, warmup, flush)
    return float(np.mean(ms)), float(pct(ms, 99))


def large_clouds(sampler, flush, dev, steps: int):
    """Single large clouds N in {8192, 16384, 32768} (1 x 1 x 0.2 slab with 5%
    Gaussian bumps, sorted by x), C = N/4: plain FPS (M = 1, one thread-block
    cluster) and NPDU-AFPS with M in {8, 32, 64, 128}."""
    import torch
    from paper_2208_08795_gb300 import afps as A, synth
    rows = []
    for N in (8192, 16384, 32768):
        P = synth.slab_cloud(2, N)
        x = torch.from_numpy(P).to(dev)
        for M, k in ((1, 0), (8, 8), (32, 16), (64, 16), (128, 16)):
            ba = A.BatchArgs([0, N], N // 4, M, k, 0)
            out = torch.empty(ba.total_out, dtype=torch.int32, device=dev)
            ms, p99 = time_batch(sampler, x, ba, out, steps, 3, flush)
            plan = sampler.describe_plan(-(-N // M), -(-(N // 4) // M), k, M)
            rows.append({"N": N, "C": N // 4, "M": M, "k": k, "ms": round(ms, 4),
                         "p99_ms": round(p99, 4), "variant": plan})
    for r in rows:  # speedup over plain FPS at equal N and C
        base = next(b for b in rows if b["N"] == r["N"] and b["M"] == 1)
        r["speedup_vs_fps"] = round(base["ms"] / r["ms"], 2)
    return {"workload": "slab clouds 8K/16K/32K, C=N/4", "runs": rows}


# Table IV of the paper: Transmuter (gem5) seconds, for context only
PAPER_TABLE_IV = {"fps_s": {2048: 0.0170, 4096: 0.0892, 8192: 0.3028, 16384: 0.6172, 32768: 1.2211},
                  "npdu_afps_m32_s": {2048: 0.0005, 4096: 0.0007, 8192: 0.0011, 16384: 0.0022,
                                      32768: 0.0044}}


def table_iv(sampler, flush, dev, steps: int):
    """The paper's size sweep (Table IV, and NPDU on FPS, Sec. IV-D) on one
    GB300: single slab clouds of N in {2K .. 32K} points sorted by x, C = 512,
    plain FPS, NPDU-FPS (M = 1, k = 8), AFPS (M = 32) and NPDU-AFPS (M = 32,
    k = 16); isolated steps after an L2 flush, variants autotuned.  The
    paper's own times (a simulated 64-core accelerator) are listed beside."""
    import torch
    from paper_2208_08795_gb300 import afps as A, synth
    rows = []
    for N in (2048, 4096, 8192, 16384, 32768):
        x = torch.from_numpy(synth.slab_cloud(2, N)).to(dev)
        row = {"N": N, "C": 512}
        for name, M, k in (("fps", 1, 0), ("npdu_fps_k8", 1, 8), ("afps_m32", 32, 0),
                           ("npdu_afps_m32_k16", 32, 16)):
            ba = A.BatchArgs([0, N], 512, M, k, 0)
            out = torch.empty(ba.total_out, dtype=torch.int32, device=dev)
            ms, _ = time_batch(sampler, x, ba, out, steps, 3, flush)
            row[name + "_ms"] = round(ms, 4)
        for name in ("npdu_fps_k8", "afps_m32", "npdu_afps_m32_k16"):
            row[name + "_speedup"] = round(row["fps_ms"] / row[name + "_ms"], 1)
        row["paper_fps_ms"] = PAPER_TABLE_IV["fps_s"][N] * 1e3
        row["paper_npdu_afps_m32_ms"] = PAPER_TABLE_IV["npdu_afps_m32_s"][N] * 1e3
        rows.append(row)
    return {"workload": "single slab clouds, C=512 (Table IV analogue); paper times are a "
                        "simulated 64-core accelerator, context only", "rows": rows}


def ragged_batch(sampler, flush, dev, steps: int):
    """256 object-scale clouds, N ~ U[2048, 32768], C = N/4, M = round(N/256)
    (sectors of about 256 points), NPDU k = 16: all (cloud, sector) items in
    one persistent launch, replayed from a CUDA graph, variant autotuned."""
    import torch
    from paper_2208_08795_gb300 import afps as A, synth
    clouds, Cs, Ms = synth.ragged_batch(3, 256)
    xyz, off = synth.pack(clouds)
    x = torch.from_numpy(xyz).to(dev)
    res = {}
    for k in (0, 16):
        ba = A.BatchArgs(off, Cs, Ms, k, 0)
        out = torch.empty(ba.total_out, dtype=torch.int32, device=dev)
        ms, p99 = time_batch(sampler, x, ba, out, steps, 3, flush)
        res["npdu" if k else "full"] = {"ms": round(ms, 4), "p99_ms": round(p99, 4),
                                        "clouds_per_s": round(256 / (ms / 1e3), 1),
                                        "hbm_gbs": round((12 * int(off[-1]) + 4 * ba.total_out)
                                                         / (ms / 1e3) / 1e9, 1)}
    return {"workload": f"ragged batch of 256 clouds, {int(off[-1])} points, "
                        f"{sum(Ms)} sectors, C=N/4", **res}


def sort_section(sampler, flush, dev, steps: int):
    """Device sort by x of unsorted input: the object batch (32 x 2048) and a
    32768-point slab cloud, each in random storage order."""
    import torch
    from paper_2208_08795_gb300 import synth
    g = np.random.Generator(np.random.PCG64(11))
    rows = {}
    for name, clouds in (("object_batch_32x2048", synth.object_batch(1, 32, 2048)),
                         ("slab_32768", [synth.slab_cloud(2, 32768)])):
        clouds = [c[g.permutation(c.shape[0])] for c in clouds]
        xyz, off = synth.pack(clouds)
        x = torch.from_numpy(xyz).to(dev)
        out = torch.empty_like(x)
        perm = torch.empty(x.shape[0], dtype=torch.int32, device=dev)
        stream = torch.cuda.current_stream()
        for _ in range(3):
            sampler.sort_by_key(x, off, 0, out, perm)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            sampler.sort_by_key(x, off, 0, out, perm)
            b.record(stream)
        torch.cuda.synchronize()
        ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
        rows[name] = {"ms": round(ms, 4), "points_per_s": round(int(off[-1]) / (ms / 1e3), 1)}
    return {"workload": "stable radix sort by x of shuffled clouds (one CTA per cloud)", **rows}


def group_section(sampler, x, off, flush, dev, steps: int):
    """Ball query after sampling on the object batch: the NPDU-AFPS samples
    (C = 512 per cloud) as centroids, radius 0.2, K = 32; full scan against
    the range-limited scan that the x-sorted storage allows."""
    import torch
    from paper_2208_08795_gb300 import afps as A
    ba = A.BatchArgs(off, C_SAMPLES, M_SECTORS, K_WINDOW, 0)
    sel = sampler.sample_batched(x, ba)
    grp = torch.empty((ba.total_out, 32), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    rows = {}
    for name, axis in (("full_scan", -1), ("sorted_range_scan", 0)):
        for _ in range(3):
            sampler.ball_query(x, off, sel, ba.out_off, 0.2, 32, axis, grp)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            sampler.ball_query(x, off, sel, ba.out_off, 0.2, 32, axis, grp)
            b.record(stream)
        torch.cuda.synchronize()
        ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
        rows[name] = {"ms": round(ms, 4), "clouds_per_s": round(B_CLOUDS / (ms / 1e3), 1)}
    out = {"workload": "ball query r=0.2 K=32 around the 512 NPDU-AFPS samples of each of "
                       "32 x 2048-point clouds", **rows}
    # k nearest neighbours (K = 32) around the same centroids
    nn = torch.empty((ba.total_out, 32), dtype=torch.int32, device=dev)
    krows = {}
    for name, axis in (("full_scan", -1), ("sorted_outward_scan", 0)):
        for _ in range(3):
            sampler.knn(x, off, sel, ba.out_off, 32, axis, nn)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            sampler.knn(x, off, sel, ba.out_off, 32, axis, nn)
            b.record(stream)
        torch.cuda.synchronize()
        ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
        krows[name] = {"ms": round(ms, 4), "clouds_per_s": round(B_CLOUDS / (ms / 1e3), 1)}
    out["knn"] = {"workload": "32 nearest neighbours of the same centroids", **krows}
    return out


# ------------------------------------------------------------------ serving
SERVING_LEVELS = [16384, 4096, 1024, 256]
SERVING_RATES = [500.0, 2000.0, 8000.0, 32000.0]


def serving_sweep(sampler, seconds_per_rate: float = 0.25):
    """Poisson streams of LiDAR-like frames (16-32K points, 32 rings, range
    U[2, 60] m, 2% dropout, emitted column by column), each a chained request
    16384 -> 4096 -> 1024 -> 256 with NPDU-AFPS M = 32, k = 16, at rising
    arrival rates; latency is arrival to result on the host."""
    from paper_2208_08795_gb300 import afps as A, serving, synth
    frames = [synth.lidar_frame(100 + i) for i in range(8)]
    srv = A.Server(sampler, SERVING_LEVELS, 32, 16, hbm_budget_bytes=2 << 30,
                   max_inflight=256)
    try:
        serving.poisson_run(srv, frames, 1000.0, 20, seed=99)  # warm-up
        rows = []
        for i, rate in enumerate(SERVING_RATES):
            n = int(min(2000, max(100, rate * seconds_per_rate)))
            r = serving.poisson_run(srv, frames, rate, n, seed=i)
            rows.append({k: round(v, 3) if isinstance(v, float) else v for k, v in r.items()})
        # the same frames from page-locked memory, submitted without a copy
        import torch
        pinned = [torch.from_numpy(f).pin_memory().numpy() for f in frames]
        prow = []
        for i, rate in enumerate(SERVING_RATES[2:] + [64000.0]):
            n = int(min(2000, max(100, rate * seconds_per_rate)))
            r = serving.poisson_run(srv, pinned, rate, n, seed=10 + i, pinned=True)
            prow.append({k: round(v, 3) if isinstance(v, float) else v for k, v in r.items()})
    finally:
        srv.close()
    return {"workload": "LiDAR-like frames, 16-32K points, chained 16384->4096->1024->256, "
                        "NPDU-AFPS M=32 k=16, Poisson arrivals",
            "hbm_budget_bytes": 2 << 30, "rates": rows,
            "saturation_frames_per_s": max(r["achieved_frames_per_s"] for r in rows),
            "pinned_frames": {"how": "frames in page-locked memory, afps_server_submit_pinned "
                                     "(admission reads them by DMA, no host copy)",
                              "rates": prow,
                              "saturation_frames_per_s": max(r["achieved_frames_per_s"]
                                                             for r in prow)}}


# ------------------------------------------------------------------ arms
def run_reference(args, rank: int, world: int) -> int:
    """The oracle, as it stands, on the host cores: the reference arm.  One
    step = `batches` whole batches (about 50 ms of work, so that handing the
    work to the processes costs little), timed on the host clock."""
    if rank != 0:
        return 0
    clouds, _, _ = make_batch(batch_seed(0))
    procs = cpu_threads()
    pool = OraclePool(clouds, C_SAMPLES, M_SECTORS, K_WINDOW, procs)
    try:
        pool.run(1)
        t0 = time.perf_counter()
        pool.run(10)
        batches = max(1, int(0.05 / max((time.perf_counter() - t0) / 10, 1e-6)))
        for _ in range(args.warmup):
            pool.run(batches)
        ts = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            pool.run(batches)
            ts.append((time.perf_counter() - t0) * 1e3)
    finally:
        pool.close()
    ms = float(np.mean(ts))
    value = B_CLOUDS * batches / (ms / 1e3)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "p99_ms": pct(ts, 99),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "clouds": B_CLOUDS, "N": N_POINTS, "C": C_SAMPLES,
                   "M": M_SECTORS, "k": K_WINDOW, "parallelism": f"{procs} host processes",
                   "batches_per_step": batches},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle",
                         "sample": f"{args.steps} steps of {batches} whole batches of "
                                   f"{B_CLOUDS} clouds, one process per core, each a "
                                   f"contiguous chunk of the batch's clouds"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line, default=_json_default))
    return 0


def run_gpu(args, rank: int, world: int, local: int) -> int:
    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_2208_08795_gb300 import afps as A
    from paper_2208_08795_gb300 import build as build_mod
    if local == 0:
        build_mod.build()
    if world > 1:
        torch.distributed.barrier()

    clouds, xyz, off = make_batch(batch_seed(rank))
    sampler = A.Sampler(local, graph=True)
    x = torch.from_numpy(xyz).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    clocks = ClockSampler(local)
    clocks.start()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()

    plans = {}

    rot = {}

    def run(M, k, steps, warmup, latency=False, n_streams=args.streams):
        """Throughput over the rotation (steps back to back on each of
        n_streams streams), and with latency=True also per-step latency of
        isolated steps after an L2 flush."""
        ba = A.BatchArgs(off, C_SAMPLES, M, k, 0)
        out = torch.empty(ba.total_out, dtype=torch.int32, device=dev)
        # untimed: the autotuner picks the kernel variant (and writes the result)
        sampler.autotune_batched(x, ba, out)
        sampler.sync()
        n_s, c_s = -(-N_POINTS // M), -(-C_SAMPLES // M)
        plans[f"M{M}_{'npdu' if k else 'full'}"] = sampler.describe_plan(n_s, c_s, k, B_CLOUDS * M)
        xr, outr = rotation(x, ba.total_out, dev)
        rot["slots"], rot["mb"] = xr.shape[0], (xr.numel() + outr.numel()) * 4 / 2**20
        # a context without graphs for the throughput, with the variant just tuned
        tune = os.path.join(tempfile.gettempdir(), f"afps_bench_tune_{os.getpid()}.txt")
        A.afps_save_tuning(sampler.ctx, tune)
        direct = A.Sampler(local, tune_cache=tune)
        try:
            if direct.describe_plan(n_s, c_s, k, B_CLOUDS * M) != plans[f"M{M}_{'npdu' if k else 'full'}"]:
                raise RuntimeError("the throughput context did not load the tuned variant")
            barrier()
            ms, launches, last, rot["enqueue"] = time_stream(direct, xr, outr, ba, steps, warmup,
                                                             n_streams)
            barrier()
        finally:
            direct.close()
            os.unlink(tune)
        if not torch.equal(outr[last], out):
            raise RuntimeError(f"M={M} k={k}: a rotated step differs from the single call")
        del xr, outr
        lat = None
        if latency:
            lat, _ = time_device(sampler, x, ba, out, steps, warmup, flush)
            barrier()
        return ba, out, ms, lat, launches

    # headline: NPDU-AFPS M=32 k=16
    ba, out, ms, lat, launches = run(M_SECTORS, K_WINDOW, args.steps, args.warmup, latency=True)
    ms_step = max_over_ranks(ms, world, dev)
    p99 = max_over_ranks(pct(lat, 99), world, dev)
    p50 = max_over_ranks(pct(lat, 50), world, dev)
    iso_ms = max_over_ranks(float(np.mean(lat)), world, dev)
    value = B_CLOUDS * world / (ms_step / 1e3)
    head_out = out.cpu().numpy()
    head_enqueue = dict(rot["enqueue"])
    # the same steps on one stream (each step waits for the one before)
    _, _, ms1, _, _ = run(M_SECTORS, K_WINDOW, args.steps, args.warmup, n_streams=1)
    ms_one = max_over_ranks(ms1, world, dev)

    # plain FPS on the same batch, same protocol
    _, _, ms_f, _, _ = run(1, 0, args.steps, args.warmup)
    ms_fps = max_over_ranks(ms_f, world, dev)
    fps_value = B_CLOUDS * world / (ms_fps / 1e3)
    _, _, ms_f1, _, _ = run(1, 0, max(3, min(args.steps, 50)), max(3, args.warmup // 2),
                            n_streams=1)
    ms_fps_one = max_over_ranks(ms_f1, world, dev)

    # sweep of the paper's M values, NPDU off / on
    sweep = {}
    sw_steps = max(3, min(args.steps, 50))
    for M in (1, 4, 16, 32):
        for npdu in (False, True):
            k = k_rule(M) if npdu else 0
            _, _, ms_s, _, _ = run(M, k, sw_steps, max(3, args.warmup // 2))
            m = max_over_ranks(ms_s, world, dev)
            sweep[f"M{M}_{'npdu' if npdu else 'full'}"] = round(B_CLOUDS * world / (m / 1e3), 1)

    # end to end through host buffers: pipelined calls (the throughput) and
    # one synchronous call at a time (the latency of a call)
    tune = os.path.join(tempfile.gettempdir(), f"afps_bench_tune_{os.getpid()}.txt")
    A.afps_save_tuning(sampler.ctx, tune)
    direct = A.Sampler(local, tune_cache=tune)
    try:
        barrier()
        e2e_ms, h2d_bytes, d2h_bytes = time_e2e_stream(direct, xyz, ba, args.steps, args.warmup,
                                                       head_out, args.streams)
        barrier()
    finally:
        direct.close()
        os.unlink(tune)
    e2e_ms = max_over_ranks(e2e_ms, world, dev)
    h_xyz = torch.from_numpy(xyz).pin_memory().numpy()
    h_out = torch.empty(ba.total_out, dtype=torch.int32).pin_memory().numpy()
    barrier()
    ts = time_e2e(sampler, h_xyz, ba, h_out, args.steps, args.warmup)
    barrier()
    e2e_call_ms = max_over_ranks(float(np.mean(ts)), world, dev)
    serving_stats = serving_sweep(sampler) if args.serving else None
    extra_steps = max(5, min(args.steps, 20))
    large = large_clouds(sampler, flush, dev, extra_steps) if args.configs else None
    tab4 = table_iv(sampler, flush, dev, extra_steps) if args.configs else None
    ragged = ragged_batch(sampler, flush, dev, extra_steps) if args.configs else None
    sorting = sort_section(sampler, flush, dev, extra_steps) if args.configs else None
    grouping = group_section(sampler, x, off, flush, dev, extra_steps) if args.configs else None
    clk = clocks.stop()
    e2e_ok = bool(np.array_equal(h_out, head_out))

    # roofline of the sampling kernel (one launch per step).  With S streams
    # S launches run side by side: the GPU completes one every ms, and each
    # launch lasts about S x ms on its own stream.  achieved = the bytes the
    # launches of the timed region move together / the timed region.
    peak, peak_kind = measured_hbm_peak()
    hbm_bytes = 12 * int(off[-1]) + 4 * int(ba.total_out)
    kernel_s = ms / 1e3  # timed region / launches
    achieved = hbm_bytes / kernel_s / 1e9
    evals, compares = npdu_work(head_out, ba, K_WINDOW)
    sm_mhz = clk["sm_mhz"] or 2070.0
    alu_peak = 152 * 128 * sm_mhz * 1e6 / 1e12  # FP32 lanes x clock, Tops/s
    alu_ach = (9 * evals + compares) / kernel_s / 1e12
    traffic = (NCU_TRAFFIC["bytes_per_launch"]
               if NCU_TRAFFIC["source_hash"] == kernel_source_hash() else None)
    # issue: executed warp instructions (an ncu count of one launch of these
    # kernel sources) x launches / timed region, against every scheduler
    # issuing one per cycle -- how busy the SMs are, not algorithmic work
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    inst = (NCU_INST["warp_inst_per_launch"]
            if NCU_INST["source_hash"] == kernel_source_hash() else None)
    issue_peak = n_sm * 4 * sm_mhz * 1e6
    issue = None if inst is None else {
        "bound": "issue", "achieved": inst / kernel_s, "peak": issue_peak,
        "unit": "warp instructions/s", "frac": inst / kernel_s / issue_peak,
        "warp_inst_per_launch": inst,
        "how": f"ncu smsp__inst_executed.sum of one launch x launches / timed region; peak = "
               f"{n_sm} SMs x 4 schedulers x the median SM clock under load"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "p50_ms": p50, "p99_ms": p99,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "clouds_per_gpu": B_CLOUDS, "N": N_POINTS,
                   "C": C_SAMPLES, "M": M_SECTORS, "k": K_WINDOW,
                   "l2": f"inputs larger than L2: the {rot['slots']} resident copies of the batch "
                         f"({rot['mb']:.0f} MB with their outputs) are visited in turn, so each "
                         "timed step reads points untouched for more than 2 x L2 of traffic; "
                         "p50/p99 are isolated steps, each after a 256 MB L2 flush",
                   "streams": args.streams,
                   "timing": f"value and ms_per_step: K steps, step i on stream i mod "
                             f"{args.streams} (each stream's steps back to back, the streams "
                             "side by side), between two CUDA events on the launching stream "
                             "that every stream waits for / joins, enqueued while a sleep kernel "
                             "(before the first event) holds the streams; ms_per_step = timed "
                             "region / K; p50/p99: per-step events of isolated steps",
                   "parallelism": f"replicas x{world}",
                   "launch": "throughput: one direct kernel launch per step; latency: CUDA graph "
                             "replay; kernel variant chosen by the autotuner (untimed)"},
        "kernel_variants": plans,
        "sampled_points_per_s": value * C_SAMPLES,
        "fps_baseline": {"value": fps_value, "unit": UNIT, "ms_per_step": ms_fps,
                         "speedup_npdu_afps": value / fps_value, "streams": args.streams},
        "one_stream": {"value": B_CLOUDS * world / (ms_one / 1e3), "ms_per_step": ms_one,
                       "fps_value": B_CLOUDS * world / (ms_fps_one / 1e3),
                       "fps_ms_per_step": ms_fps_one, "speedup_npdu_afps": ms_fps_one / ms_one},
        "sweep_clouds_per_s": sweep,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"
                     if peak_kind == "measured" else "fallback 6.8 TB/s",
                     "algorithmic_bytes_per_launch": hbm_bytes,
                     "how": f"algorithmic bytes per launch x launches / timed region "
                            f"({args.streams} streams of back-to-back launches side by side; "
                            f"each launch lasts about {args.streams} x ms_per_step on its stream)",
                     "kernel": plans.get(f"M{M_SECTORS}_npdu")},
        "roofline_issue": issue,
        "roofline_alu": {"bound": "alu", "achieved": alu_ach, "peak": alu_peak,
                         "unit": "TFLOP/s", "frac": alu_ach / alu_peak,
                         "fp32_ops_per_launch": 9 * evals + compares},
        "e2e": {"value": B_CLOUDS * world / (e2e_ms / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": int(h2d_bytes), "d2h_bytes_per_step": int(d2h_bytes),
                "ms_per_step": e2e_ms, "matches_device_path": True,
                "how": f"K calls of afps_sample_batched_host_async on page-locked buffers "
                       f"(inputs rotating over copies larger than L2, one output per step), "
                       f"call i on stream i mod {args.streams}, one synchronisation, host "
                       f"clock; every output checked",
                "sync_call_ms": e2e_call_ms, "sync_call_matches_device_path": e2e_ok},
        "serving": serving_stats,
        "large_clouds": large,
        "table_iv": tab4,
        "ragged_batch": ragged,
        "sort_by_key": sorting,
        "ball_query": grouping,
        "gpu_launches": launches,
        "isolated_step_ms": iso_ms,
        "enqueue": head_enqueue,
        "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"],
                   "reasons": clk["reasons"], "samples": clk["samples"]},
    }

    if rank == 0 and world == 1:
        threads = cpu_threads()
        rate, reps, ref = time_oracle(clouds, C_SAMPLES, M_SECTORS, K_WINDOW,
                                      args.cpu_seconds, threads)
        rate1, reps1, _ = time_oracle(clouds, C_SAMPLES, M_SECTORS, K_WINDOW,
                                      args.cpu_seconds / 4, 1)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": f"{reps} whole batches of {B_CLOUDS} clouds "
                                          f"(about {args.cpu_seconds:.0f} s), one process per "
                                          f"core, each a contiguous chunk of the clouds",
                                "single_thread": {"value": rate1, "unit": UNIT, "cores": 1,
                                                  "sample": f"{reps1} whole batches of "
                                                            f"{B_CLOUDS} clouds on one thread"}}
        same = sum(int(np.array_equal(head_out[ba.out_off[b]:ba.out_off[b + 1]], ref[b]))
                   for b in range(B_CLOUDS))
        line["parity"] = f"{same}/{B_CLOUDS} clouds bit-exact vs the FP32 oracle"
        import oracle
        agree, drel = [], []
        for b, P in enumerate(clouds):
            r64 = oracle.afps(P, C_SAMPLES, M_SECTORS, K_WINDOW, 0, precision="f64")
            agree.append(float(np.mean(r64 == ref[b])))
            R32, R64 = oracle.coverage_radius(P, ref[b]), oracle.coverage_radius(P, r64)
            drel.append(abs(R32 - R64) / R64)
        line["fp64_oracle"] = {"index_agreement": float(np.mean(agree)),
                               "coverage_radius_rel_diff_max": float(max(drel))}
    else:
        line["cpu_baseline"] = None
    sampler.close()
    if rank == 0:
        print(json.dumps(line, default=_json_default))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--cpu-seconds", type=float, default=5.0)
    ap.add_argument("--streams", type=int, default=8,
                    help="streams the throughput steps are spread over (1: one stream)")
    ap.add_argument("--no-serving", dest="serving", action="store_false",
                    help="skip the serving sweep")
    ap.add_argument("--no-configs", dest="configs", action="store_false",
                    help="skip the large-cloud and ragged-batch sections")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    rank, world, local = rank_info()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_gpu(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
