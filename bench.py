"""Benchmark: NPDU-AFPS vs plain FPS on one GB300, clouds/s and p99 ms.

Headline workload (one step): the ragged batch of 256 object-scale clouds
(N ~ U[2048, 32768], seed 3; 2-5 primitive surfaces, jitter 0.005, unit
ball, sorted by x), C = N/4, M = max(1, round(N/256)) sectors of about 256
points, NPDU window k = 8 for M <= 8 and 16 for M >= 16 (Sec. IV-D); all
17,576 (cloud, sector) items in one batched call through the C ABI, replayed
from a CUDA graph, kernel variant chosen by the autotuner (untimed).  Beside
it, on the same batch and in the same run: plain FPS (M = 1, no NPDU) and
AFPS without NPDU, the end-to-end time through host buffers, the roofline of
the sampling kernel and the CPU oracle on the host's cores.

Timing.  Throughput (`value`, `ms_per_step`): K steps back to back on one
stream between two CUDA events on that stream; step i runs on the next of R
resident copies of the batch (the copies span twice the L2), so every timed
step reads cold points without a flush; a fixed-length sleep kernel ahead of
the first event holds the stream while the host enqueues the K steps.
Latency (`p50_ms`, `p99_ms`): isolated steps, each after a 256 MB write that
flushes the L2, with its own pair of events.  The end-to-end number (`e2e`)
is the same metric through host buffers on the host clock.  The CPU oracle
runs one worker process per host core.

Secondary sections: the object batch of 32 x 2048 points (M in {1, 4, 16,
32}, NPDU off and on, one stream), single large clouds, the paper's Table IV
sweep, sorting, grouping and the serving runtime.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun each rank samples its own
batch (weak scaling, no collective on the data path); the time is the max
over ranks.
"""
from __future__ import annotations

import argparse
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
RAGGED_CLOUDS, RAGGED_SECTOR = 256, 256
WORKLOAD = ("ragged batch of 256 clouds, N ~ U[2048, 32768] (seed 3), C = N/4, "
            "M = round(N/256), NPDU-AFPS k = 8 (M <= 8) / 16 (M >= 16)")
# the object batch (secondary section): 32 x 2048 points, C = 512
B_CLOUDS, N_POINTS, C_SAMPLES, M_SECTORS, K_WINDOW = 32, 2048, 512, 32, 16
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
    """Each rank samples its own ragged batch (weak scaling)."""
    return 3 + rank


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
def make_ragged(seed: int):
    """The ragged batch: clouds, per-cloud C, M and NPDU window."""
    from paper_2208_08795_gb300 import synth
    clouds, Cs, Ms = synth.ragged_batch(seed, RAGGED_CLOUDS, sector_points=RAGGED_SECTOR)
    ks = [k_rule(M) for M in Ms]
    return clouds, Cs, Ms, ks


def make_batch(seed: int):
    """The object batch (32 x 2048 points)."""
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


def _oracle_init(clouds, Cs, Ms, ks):
    global _ORACLE_WORK
    _ORACLE_WORK = (clouds, Cs, Ms, ks)


def _oracle_chunk(lo: int, hi: int, reps: int):
    """Clouds [lo, hi) of the batch through the oracle, `reps` times; returns
    the last pass's indices."""
    import oracle
    clouds, Cs, Ms, ks = _ORACLE_WORK
    out = None
    for _ in range(reps):
        out = [oracle.afps(clouds[i], Cs[i], Ms[i], ks[i], 0) for i in range(lo, hi)]
    return out


def balanced_chunks(sizes, parts: int):
    """Contiguous ranges of the clouds with about equal total points each."""
    total = float(sum(sizes))
    bounds, acc, b = [0], 0.0, 1
    for i, s in enumerate(sizes):
        acc += s
        if b < parts and acc >= total * b / parts and i + 1 < len(sizes):
            bounds.append(i + 1)
            b += 1
    bounds.append(len(sizes))
    return [(bounds[i], bounds[i + 1]) for i in range(len(bounds) - 1)
            if bounds[i + 1] > bounds[i]]


class OraclePool:
    """The oracle, as it stands, over one batch on `procs` host cores: worker
    processes (started with spawn, so safe after CUDA use) that each hold the
    batch and run a contiguous chunk of its clouds (chunks of about equal
    points).  Processes rather than threads: the oracle's Python wrapper
    holds the GIL for part of each call."""

    def __init__(self, clouds, Cs, Ms, ks, procs: int):
        self.n = len(clouds)
        self.chunks = balanced_chunks([c.shape[0] for c in clouds], max(1, procs))
        self.procs = len(self.chunks)
        self.pool = None
        if self.procs == 1:
            _oracle_init(clouds, Cs, Ms, ks)
        else:
            import multiprocessing as mp
            self.pool = mp.get_context("spawn").Pool(self.procs, initializer=_oracle_init,
                                                     initargs=(clouds, Cs, Ms, ks))

    def run(self, reps: int = 1):
        """The batch `reps` times; returns the last pass's indices per cloud."""
        if self.pool is None:
            return _oracle_chunk(0, self.n, reps)
        out = []
        for part in self.pool.starmap(_oracle_chunk, [(a, b, reps) for a, b in self.chunks],
                                      chunksize=1):
            out.extend(part)
        return out

    def close(self):
        if self.pool is not None:
            self.pool.close()
            self.pool.join()
            self.pool = None


def time_oracle(clouds, Cs, Ms, ks, budget_s: float, procs: int):
    """The oracle as it stands on `procs` cores: whole batches, repeated for
    about budget_s.  Returns (clouds/s, batches, indices per cloud, processes)."""
    pool = OraclePool(clouds, Cs, Ms, ks, procs)
    try:
        t0 = time.perf_counter()
        outs = pool.run(1)  # starts the workers and warms the library
        once = time.perf_counter() - t0
        reps = max(1, min(100000, int(budget_s / max(once, 1e-6))))
        t0 = time.perf_counter()
        pool.run(reps)
        el = time.perf_counter() - t0
    finally:
        pool.close()
    return reps * len(clouds) / el, reps, outs, pool.procs


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
    R = max(4, -(-2 * L2_BYTES // slot_bytes))
    xr = x.unsqueeze(0).repeat(R, *([1] * x.dim())).contiguous()
    outr = torch.full((R, total_out), -1, dtype=torch.int32, device=dev)
    return xr, outr


def time_steps(sampler, xr, outr, ba, steps: int, warmup: int):
    """Whole-job throughput on one stream: K steps issued through the C ABI
    (afps_sample_batched: a graph replay on a graph context, a direct launch
    otherwise), each on the next resident slot of the rotation, back to back.
    One pair of CUDA events on the stream brackets the K steps.  Every slot
    is run once first (untimed; a graph context captures its graphs there);
    the timed steps start at the least recently used slot, so every one of
    them reads cold points.  A fixed-length sleep kernel before the first
    event holds the stream while the host enqueues the steps, so the host's
    call rate does not set the pace.  Returns (ms per step, launches in the
    timed region, last slot used, enqueue information)."""
    import torch
    from paper_2208_08795_gb300 import afps as A
    fn = A.load().afps_sample_batched
    stream = torch.cuda.current_stream()
    R = xr.shape[0]
    args = [(sampler.ctx, xr[i].data_ptr(), *ba.args(), outr[i].data_ptr(), stream.cuda_stream)
            for i in range(R)]

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
    hold_s = min(3.0 * per_call * steps + 1e-3, 0.2)
    torch.cuda._sleep(int(hold_s * 2.07e9))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n0 = sampler.launch_count
    e0.record(stream)
    t0 = time.perf_counter()
    for i in range(warmup, warmup + steps):
        call(i)
    e1.record(stream)
    enqueue_s = time.perf_counter() - t0
    torch.cuda.synchronize()
    sampler.sync()
    info = {"host_enqueue_ms": round(enqueue_s * 1e3, 3), "hold_ms": round(hold_s * 1e3, 3),
            "enqueued_within_hold": enqueue_s < hold_s}
    return (e0.elapsed_time(e1) / steps, sampler.launch_count - n0, (warmup + steps - 1) % R,
            info)


def time_e2e_stream(sampler, xyz, ba, steps: int, warmup: int, expect):
    """End to end through the public API: K calls of
    afps_sample_batched_host_async on page-locked host buffers (a graph
    context: one replay per call; the kernels read the points from, and write
    the indices to, host memory over the C2C link), one stream, then one
    synchronisation, timed on the host clock.  Step i reads input copy i mod R
    and writes output copy i mod R (the copies span twice the L2); every
    output is checked against `expect` afterwards.  Returns (ms per step,
    input bytes per step, output bytes per step)."""
    import torch
    from paper_2208_08795_gb300 import afps as A
    fn = A.load().afps_sample_batched_host_async
    stream = torch.cuda.current_stream()
    slot = xyz.nbytes + ba.total_out * 4
    R = max(4, -(-2 * L2_BYTES // slot))
    hx = torch.from_numpy(xyz).unsqueeze(0).repeat(R, 1, 1).pin_memory()
    ho = torch.full((R, ba.total_out), -1, dtype=torch.int32).pin_memory()
    args = [(sampler.ctx, hx[i].data_ptr(), *ba.args(), ho[i].data_ptr(), stream.cuda_stream)
            for i in range(R)]

    def call(i):
        if fn(*args[i % R]) != 0:
            raise A.AfpsError(-1, A.afps_last_error(sampler.ctx))

    for i in range(max(R, warmup)):  # captures every slot's graph, then warms
        call(i)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(steps):
        call(i)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / steps
    sampler.sync()
    if not bool((ho == torch.from_numpy(expect).unsqueeze(0)).all()):
        raise RuntimeError("an end-to-end step differs from the device path")
    return ms, xyz.nbytes, ba.total_out * 4


def c2c_copy_gbs(nbytes: int, reps: int = 10) -> float:
    """Host-to-device bandwidth of the C2C link as the copy engine sees it:
    page-locked host memory to device memory, one cudaMemcpyAsync of nbytes
    per repetition, CUDA events on the stream (the ceiling of the end-to-end
    path, whose kernels read the same bytes over the same link)."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    for _ in range(3):
        d.copy_(h, non_blocking=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        d.copy_(h, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    return nbytes * reps / (e0.elapsed_time(e1) / 1e3) / 1e9


def time_e2e_sync(sampler, h_xyz, ba, h_out, steps: int, warmup: int):
    """One synchronous afps_sample_batched_host call at a time (page-locked
    buffers): the latency a caller sees for a single batch."""
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


def npdu_work(out_idx, ba, k=None):
    """Algorithmic work of one batch: distance evaluations (window sizes, or
    whole sectors) and argmax compares, from the sector plan and the output.
    k: the window of every cloud, or None for each cloud's own (ba.k)."""
    evals = compares = 0
    for b in range(ba.B):
        N = int(ba.pt_off[b + 1] - ba.pt_off[b])
        C, M = int(ba.C[b]), int(ba.M[b])
        kb = int(ba.k[b]) if k is None else k
        idx = out_idx[ba.out_off[b]:ba.out_off[b] + C]
        for s in range(M):
            lo, hi = s * N // M, (s + 1) * N // M
            o0, o1 = s * C // M, (s + 1) * C // M
            n = hi - lo
            compares += (o1 - o0 - 1) * n
            p = idx[o0:o1 - 1].astype(np.int64) - lo
            if kb > 0:
                evals += int((np.minimum(n - 1, p + (kb - kb // 2))
                              - np.maximum(0, p - kb // 2) + 1).sum())
            else:
                evals += n * len(p)
    return evals, compares


HEADLINE_KERNEL_SOURCES = ("afps_win.cu", "afps_device.cuh", "afps_internal.h")


def kernel_source_hash() -> str:
    """Hash of the sources the headline kernel (afps_win_kernel) is built from."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2208_08795_gb300", "csrc")
    for f in HEADLINE_KERNEL_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


# DRAM traffic of the headline kernel from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum of one launch over the ragged batch), valid only for
# the kernel sources it was taken on (their hash); otherwise reported as null.
NCU_TRAFFIC = {"source_hash": "f6dfa383e566b02e", "bytes_per_launch": 54947840}
# warp instructions of one headline launch (ncu smsp__inst_executed.sum), same rule
NCU_INST = {"source_hash": "f6dfa383e566b02e", "warp_inst_per_launch": 55554431}
# shared-memory wavefronts of one headline launch (ncu
# l1tex__data_pipe_lsu_wavefronts_mem_shared.sum; 128 bytes each), same rule
NCU_SMEM = {"source_hash": "f6dfa383e566b02e", "wavefronts_per_launch": 7709770}


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
            rounds = -(-(N // 4) // M)  # iterations of the longest sector's chain
            rows.append({"N": N, "C": N // 4, "M": M, "k": k, "ms": round(ms, 4),
                         "p99_ms": round(p99, 4), "variant": plan,
                         "iterations_per_sector": rounds,
                         "ns_per_iteration": round(ms * 1e6 / rounds, 1)})
    for r in rows:  # speedup over plain FPS at equal N and C
        base = next(b for b in rows if b["N"] == r["N"] and b["M"] == 1)
        r["speedup_vs_fps"] = round(base["ms"] / r["ms"], 2)
    return {"workload": "slab clouds 8K/16K/32K, C=N/4", "runs": rows,
            "latency": "few sectors: each launch is the latency of its longest sector's chain "
                       "of iterations, so each run also gives the step time per iteration "
                       "(ns_per_iteration; cycles_per_iteration at the median SM clock), "
                       "stage-in and launch included"}


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
    return {"workload": "stable radix sort by x of shuffled clouds", **rows}


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
        for i, rate in enumerate(SERVING_RATES + [64000.0, 128000.0]):  # past saturation
            n = int(min(2000, max(100, rate * seconds_per_rate)))
            r = serving.poisson_run(srv, frames, rate, n, seed=i)
            rows.append({k: round(v, 3) if isinstance(v, float) else v for k, v in r.items()})
        # the same frames from page-locked memory, submitted without a copy
        import torch
        pinned = [torch.from_numpy(f).pin_memory().numpy() for f in frames]
        prow = []
        for i, rate in enumerate(SERVING_RATES[2:] + [64000.0, 128000.0, 256000.0]):
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
    """The oracle, as it stands, on the host cores: the reference arm, on the
    headline workload.  One step = `batches` whole ragged batches (at least
    one; about 50 ms of work), timed on the host clock."""
    if rank != 0:
        return 0
    clouds, Cs, Ms, ks = make_ragged(batch_seed(0))
    procs = cpu_threads()
    pool = OraclePool(clouds, Cs, Ms, ks, procs)
    try:
        t0 = time.perf_counter()
        pool.run(1)
        once = time.perf_counter() - t0
        batches = max(1, int(0.05 / max(once, 1e-6)))
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
    value = RAGGED_CLOUDS * batches / (ms / 1e3)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "p99_ms": pct(ts, 99),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "clouds": RAGGED_CLOUDS,
                   "points": int(sum(c.shape[0] for c in clouds)), "samples": int(sum(Cs)),
                   "sectors": int(sum(Ms)), "parallelism": f"{pool.procs} host processes",
                   "batches_per_step": batches},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.procs, "kind": "oracle",
                         "sample": f"{args.steps} steps of {batches} whole ragged batch(es) of "
                                   f"{RAGGED_CLOUDS} clouds, one process per core, each a "
                                   f"contiguous chunk of the clouds (about equal points)"},
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
    from paper_2208_08795_gb300 import synth
    if local == 0:
        build_mod.build()
    if world > 1:
        torch.distributed.barrier()

    clouds, Cs, Ms, ks = make_ragged(batch_seed(rank))
    xyz, off = synth.pack(clouds)
    n_clouds = len(clouds)
    sampler = A.Sampler(local, graph=True)
    x = torch.from_numpy(xyz).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    clocks = ClockSampler(local)
    clocks.start()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()

    # ---------------------------------------------------------- headline
    ba = A.BatchArgs(off, Cs, Ms, ks, 0)
    out = torch.empty(ba.total_out, dtype=torch.int32, device=dev)
    sampler.autotune_batched(x, ba, out)  # untimed: every shape class tuned
    sampler.sync()
    head_out = sampler.sample_batched(x, ba).cpu().numpy()
    xr, outr = rotation(x, ba.total_out, dev)
    slots, rot_mb = xr.shape[0], (xr.numel() + outr.numel()) * 4 / 2**20
    barrier()
    ms, launches, last, enqueue = time_steps(sampler, xr, outr, ba, args.steps, args.warmup)
    barrier()
    if not np.array_equal(outr[last].cpu().numpy(), head_out):
        raise RuntimeError("a timed step differs from the single call")
    del xr, outr
    ms_step = max_over_ranks(ms, world, dev)
    value = n_clouds * world / (ms_step / 1e3)
    lat, _ = time_device(sampler, x, ba, out, args.steps, args.warmup, flush)
    barrier()
    p50 = max_over_ranks(pct(lat, 50), world, dev)
    p99 = max_over_ranks(pct(lat, 99), world, dev)
    iso_ms = max_over_ranks(float(np.mean(lat)), world, dev)
    launches_per_step = launches / args.steps

    # plain FPS and AFPS without NPDU on the same batch, same protocol
    def arm(M, k, steps, warmup):
        b = A.BatchArgs(off, Cs, M, k, 0)
        o = torch.empty(b.total_out, dtype=torch.int32, device=dev)
        sampler.autotune_batched(x, b, o)
        sampler.sync()
        xr2, outr2 = rotation(x, b.total_out, dev)
        barrier()
        m, _, _, _ = time_steps(sampler, xr2, outr2, b, steps, warmup)
        barrier()
        del xr2, outr2
        return max_over_ranks(m, world, dev)

    fps_steps, fps_warm = max(3, min(args.steps, 5)), 3
    ms_fps = arm(1, 0, fps_steps, fps_warm)
    ms_full = arm(Ms, 0, max(3, min(args.steps, 20)), 3)
    # the same windows under the full-first-pass reading (Sec. III-C): every
    # round after the first updates a window, none is decided by the stride
    # phase of the literal reading; isolated steps, as p50/p99
    ba_ff = A.BatchArgs(off, Cs, Ms, ks, 0, method=A.AFPS_METHOD_FULL_FIRST_PASS)
    out_ff = torch.empty(ba_ff.total_out, dtype=torch.int32, device=dev)
    lat_ff, _ = time_device(sampler, x, ba_ff, out_ff, max(3, min(args.steps, 20)), 3, flush)
    iso_ff = max_over_ranks(float(np.mean(lat_ff)), world, dev)

    # end to end through host buffers: pipelined calls (the throughput) and
    # one synchronous call at a time (the latency of a call)
    e2e_ms, h2d_bytes, d2h_bytes = time_e2e_stream(sampler, xyz, ba, args.steps, args.warmup,
                                                   head_out)
    e2e_ms = max_over_ranks(e2e_ms, world, dev)
    h_xyz = torch.from_numpy(xyz).pin_memory().numpy()
    h_out = torch.empty(ba.total_out, dtype=torch.int32).pin_memory().numpy()
    barrier()
    ts = time_e2e_sync(sampler, h_xyz, ba, h_out, max(3, min(args.steps, 10)), 3)
    barrier()
    e2e_call_ms = max_over_ranks(float(np.mean(ts)), world, dev)
    e2e_ok = bool(np.array_equal(h_out, head_out))
    link_gbs = c2c_copy_gbs(int(h2d_bytes))

    # ---------------------------------------------------------- object batch (config 2)
    obj = object_batch_section(args, sampler, dev, world, barrier) if args.configs else None
    serving_stats = serving_sweep(sampler) if args.serving else None
    extra_steps = max(5, min(args.steps, 20))
    large = large_clouds(sampler, flush, dev, extra_steps) if args.configs else None
    tab4 = table_iv(sampler, flush, dev, extra_steps) if args.configs else None
    sorting = sort_section(sampler, flush, dev, extra_steps) if args.configs else None
    grouping = None
    if args.configs:
        _, oxyz, ooff = make_batch(1 + rank)
        grouping = group_section(sampler, torch.from_numpy(oxyz).to(dev), ooff, flush, dev,
                                 extra_steps)
    clk = clocks.stop()

    # roofline of the sampling kernel: one launch per step (the merged
    # window-kernel class; `launches_per_step` says so), its duration the
    # timed region / K on the launching stream
    peak, peak_kind = measured_hbm_peak()
    hbm_bytes = 12 * int(off[-1]) + 4 * int(ba.total_out)
    kernel_s = ms / 1e3 / max(launches_per_step, 1.0)
    achieved = hbm_bytes / (ms / 1e3) / 1e9
    evals, compares = npdu_work(head_out, ba)
    sm_mhz = clk["sm_mhz"] or 2070.0
    if large:
        for r in large["runs"]:
            r["cycles_per_iteration"] = round(r["ns_per_iteration"] * sm_mhz / 1e3)
    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count
    alu_peak = n_sm * 128 * sm_mhz * 1e6 / 1e12  # FP32 lanes x clock, Tops/s
    alu_ach = (9 * evals + compares) / (ms / 1e3) / 1e12
    src = kernel_source_hash()
    traffic = NCU_TRAFFIC["bytes_per_launch"] if NCU_TRAFFIC["source_hash"] == src else None
    inst = NCU_INST["warp_inst_per_launch"] if NCU_INST["source_hash"] == src else None
    issue_peak = n_sm * 4 * sm_mhz * 1e6
    issue = None if inst is None else {
        "bound": "issue", "achieved": inst / kernel_s, "peak": issue_peak,
        "unit": "warp instructions/s", "frac": inst / kernel_s / issue_peak,
        "warp_inst_per_launch": inst,
        "how": f"ncu smsp__inst_executed.sum of one launch / the launch's duration; peak = "
               f"{n_sm} SMs x 4 schedulers x the median SM clock under load"}
    waves = NCU_SMEM["wavefronts_per_launch"] if NCU_SMEM["source_hash"] == src else None
    smem_peak = n_sm * 128 * sm_mhz * 1e6 / 1e9  # 128 bytes a clock per SM, GB/s
    smem = None if waves is None else {
        "bound": "smem", "achieved": waves * 128 / kernel_s / 1e9, "peak": smem_peak,
        "unit": "GB/s", "frac": waves * 128 / kernel_s / 1e9 / smem_peak,
        "wavefronts_per_launch": waves,
        "how": f"ncu l1tex__data_pipe_lsu_wavefronts_mem_shared.sum of one launch x 128 bytes / "
               f"the launch's duration; peak = {n_sm} SMs x 128 bytes x the median SM clock"}
    plan_desc = sampler.describe_batched(ba)

    sum_c = int(ba.total_out)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "p50_ms": p50, "p99_ms": p99,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "clouds_per_gpu": n_clouds,
                   "points": int(off[-1]), "samples": sum_c, "sectors": int(sum(Ms)),
                   "l2": f"inputs larger than L2: the {slots} resident copies of the batch "
                         f"({rot_mb:.0f} MB with their outputs) are visited in turn, so each "
                         "timed step reads points untouched for more than 2 x L2 of traffic; "
                         "p50/p99 are isolated steps, each after a 256 MB L2 flush",
                   "timing": "value and ms_per_step: K steps back to back on one stream between "
                             "two CUDA events on that stream, enqueued while a sleep kernel "
                             "(before the first event) holds the stream; ms_per_step = timed "
                             "region / K; p50/p99: per-step events of isolated steps",
                   "parallelism": f"replicas x{world}",
                   "launch": "one afps_sample_batched call per step: a CUDA graph replay (one "
                             "graph per resident copy); kernel variants chosen by the "
                             "autotuner (untimed)"},
        "kernel_launches": plan_desc,
        "launches_per_step": launches_per_step,
        "sampled_points_per_s": sum_c * world / (ms_step / 1e3),
        "fps_baseline": {"value": n_clouds * world / (ms_fps / 1e3), "unit": UNIT,
                         "ms_per_step": ms_fps, "speedup_npdu_afps": ms_fps / ms_step,
                         "steps": fps_steps, "what": "plain FPS (M = 1, k = 0) on the same "
                                                     "batch, same C, same protocol"},
        "afps_no_npdu": {"value": n_clouds * world / (ms_full / 1e3), "unit": UNIT,
                         "ms_per_step": ms_full, "speedup_npdu_afps": ms_full / ms_step,
                         "what": "AFPS with the same M and no NPDU window"},
        "npdu_no_stride": {"isolated_step_ms": iso_ff, "vs_isolated_headline": iso_ff / iso_ms,
                           "what": "the same windows under the full-first-pass reading: no round "
                                   "is decided by the stride phase of the literal reading; "
                                   "isolated steps after an L2 flush, as p50/p99"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"
                     if peak_kind == "measured" else "fallback 6.8 TB/s",
                     "algorithmic_bytes_per_launch": hbm_bytes,
                     "launch_ms": kernel_s * 1e3,
                     "how": "algorithmic bytes of one step (12 bytes a point read, 4 bytes a "
                            "sample written) / the step's duration (timed region / K on the "
                            "launching stream; one kernel launch per step)"},
        "roofline_issue": issue,
        "roofline_smem": smem,
        "roofline_alu": {"bound": "alu", "achieved": alu_ach, "peak": alu_peak,
                         "unit": "TFLOP/s", "frac": alu_ach / alu_peak,
                         "fp32_ops_per_launch": 9 * evals + compares,
                         "peak_how": f"{n_sm} SMs x 128 FP32 lanes x the median SM clock"},
        "e2e": {"value": n_clouds * world / (e2e_ms / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": int(h2d_bytes), "d2h_bytes_per_step": int(d2h_bytes),
                "ms_per_step": e2e_ms, "matches_device_path": True,
                "how": "K calls of afps_sample_batched_host_async on page-locked buffers "
                       "(graph context; the kernels read the points and write the indices in "
                       "host memory over the C2C link; inputs rotating over copies larger "
                       "than L2, one output per step), one stream, one synchronisation, host "
                       "clock; every output checked",
                "sync_call_ms": e2e_call_ms, "sync_call_matches_device_path": e2e_ok,
                "link": {"bound": "c2c", "unit": "GB/s",
                         "achieved": h2d_bytes / (e2e_ms / 1e3) / 1e9,
                         "peak": link_gbs,
                         "frac": h2d_bytes / (e2e_ms / 1e3) / 1e9 / link_gbs,
                         "how": "the step's input bytes (host to device over the C2C link) / "
                                "the end-to-end step; peak: a cudaMemcpyAsync of those bytes "
                                "from page-locked memory to the device, measured in this run "
                                "(the indices go the other way, which the link carries "
                                "separately)"}},
        "object_batch": obj,
        "serving": serving_stats,
        "large_clouds": large,
        "table_iv": tab4,
        "sort_by_key": sorting,
        "ball_query": grouping,
        "gpu_launches": launches,
        "isolated_step_ms": iso_ms,
        "enqueue": enqueue,
        "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"],
                   "reasons": clk["reasons"], "samples": clk["samples"]},
    }

    if rank == 0 and world == 1:
        threads = cpu_threads()
        rate, reps, ref, procs = time_oracle(clouds, Cs, Ms, ks, args.cpu_seconds, threads)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": procs, "kind": "oracle",
                                "sample": f"{reps} whole ragged batch(es) of {n_clouds} clouds "
                                          f"(about {args.cpu_seconds:.0f} s), one process per "
                                          f"core, each a contiguous chunk of the clouds"}
        same = sum(int(np.array_equal(head_out[ba.out_off[b]:ba.out_off[b + 1]], ref[b]))
                   for b in range(n_clouds))
        line["parity"] = f"{same}/{n_clouds} clouds bit-exact vs the FP32 oracle"
        import oracle
        agree, drel = [], []
        for b in range(0, n_clouds, 16):  # every 16th cloud in FP64
            P = clouds[b]
            r64 = oracle.afps(P, Cs[b], Ms[b], ks[b], 0, precision="f64")
            agree.append(float(np.mean(r64 == ref[b])))
            R32, R64 = oracle.coverage_radius(P, ref[b]), oracle.coverage_radius(P, r64)
            drel.append(abs(R32 - R64) / R64)
        line["fp64_oracle"] = {"index_agreement": float(np.mean(agree)),
                               "coverage_radius_rel_diff_max": float(max(drel)),
                               "clouds": len(agree)}
    else:
        line["cpu_baseline"] = None
    sampler.close()
    if rank == 0:
        print(json.dumps(line, default=_json_default))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def object_batch_section(args, sampler, dev, world, barrier):
    """The object batch (32 x 2048 points, C = 512), the paper's part-
    segmentation shape (Sec. IV-B): one call per step on one stream, the
    rotation over resident copies as for the headline, on a context without
    graphs (direct launches chain through programmatic dependent launch);
    NPDU-AFPS M = 32, k = 16, plain FPS and the sweep M in {1, 4, 16, 32}
    with NPDU off and on."""
    import torch
    from paper_2208_08795_gb300 import afps as A
    clouds, xyz, off = make_batch(1)
    x = torch.from_numpy(xyz).to(dev)
    res = {"workload": f"object batch {B_CLOUDS} x {N_POINTS} pts, C={C_SAMPLES}"}
    steps = max(3, min(args.steps * 10, 200))

    def run(M, k):
        ba = A.BatchArgs(off, C_SAMPLES, M, k, 0)
        out = torch.empty(ba.total_out, dtype=torch.int32, device=dev)
        sampler.autotune_batched(x, ba, out)
        sampler.sync()
        tune = os.path.join(tempfile.gettempdir(), f"afps_bench_tune_{os.getpid()}.txt")
        A.afps_save_tuning(sampler.ctx, tune)
        direct = A.Sampler(sampler.device, tune_cache=tune)
        xr, outr = rotation(x, ba.total_out, dev)
        try:
            barrier()
            ms, _, last, _ = time_steps(direct, xr, outr, ba, steps, 5)
            barrier()
        finally:
            direct.close()
            os.unlink(tune)
        if not torch.equal(outr[last], out):
            raise RuntimeError(f"object batch M={M} k={k}: a step differs from the single call")
        return max_over_ranks(ms, world, dev), sampler.describe_plan(
            -(-N_POINTS // M), -(-C_SAMPLES // M), k, B_CLOUDS * M)

    sweep = {}
    for M in (1, 4, 16, 32):
        for npdu in (False, True):
            k = k_rule(M) if npdu else 0
            ms, plan = run(M, k)
            sweep[f"M{M}_{'npdu' if npdu else 'full'}"] = {
                "clouds_per_s": round(B_CLOUDS * world / (ms / 1e3), 1),
                "ms_per_step": round(ms, 5), "variant": plan}
    head = sweep[f"M{M_SECTORS}_npdu"]
    res.update({"npdu_afps_m32_k16": head, "fps": sweep["M1_full"],
                "speedup_npdu_afps_vs_fps": round(sweep["M1_full"]["ms_per_step"]
                                                  / head["ms_per_step"], 2),
                "sweep": sweep, "steps": steps,
                "timing": "one call per step, steps back to back on one stream between two "
                          "CUDA events, each on the next resident copy (copies span 2 x L2)"})
    return res


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--cpu-seconds", type=float, default=5.0)
    ap.add_argument("--no-serving", dest="serving", action="store_false",
                    help="skip the serving sweep")
    ap.add_argument("--no-configs", dest="configs", action="store_false",
                    help="skip the object-batch, large-cloud, Table IV, sort and grouping "
                         "sections")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    rank, world, local = rank_info()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_gpu(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
