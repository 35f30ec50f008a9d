"""Single sampling workloads, run a few times, for profiling with ncu.

    python -m paper_2208_08795_gb300.profile_cases <case> [--reps R] [--tune-cache PATH]

With --tune-cache, a batched case whose cache file does not exist yet is
autotuned (as bench.py does) and the choice saved; a later run with the same
file replays the tuned variant without autotuning, so a profiler can capture
the exact kernel the benchmark times.

Cases (inputs from `synth`; kernel variants from the planner or the cache):
  headline     32 object clouds x 2048 points, C = 512, NPDU-AFPS M = 32, k = 16 (batched)
  fps2048      the same batch, plain FPS (M = 1)
  cluster32k   one 32768-point slab cloud, C = 8192, plain FPS (one thread-block cluster)
  clusters     plain FPS on slab clouds of 8K / 16K / 32K points, C = N/4, every cluster shape
               (P, W, CS) the autotuner tries, forced one by one; prints each one's time
  npdu32k      the same cloud, NPDU-AFPS M = 32, k = 16
  ragged       256 clouds of 2K-32K points, C = N/4, sectors of ~256 points, k = 8 / 16 (persistent)
  chain        one LiDAR-like frame, levels 16384 -> 4096 -> 1024 -> 256, M = 32, k = 16
  sort         the object batch in random storage order, sorted by x
  group        ball query (r = 0.2, K = 32) around the headline samples of the batch
  knn          32 nearest neighbours of the same centroids (outward scan of the x-sorted clouds)
  coverage     coverage radius of the headline samples of the batch
"""
from __future__ import annotations

import argparse
import sys

import torch

from . import afps, build, synth

CASES = ("headline", "fps2048", "cluster32k", "clusters", "npdu32k", "ragged", "chain", "sort",
         "group", "knn", "coverage")


def run(case: str, reps: int, tune_cache: str | None = None) -> None:
    import os
    build.build()
    tune = bool(tune_cache) and not os.path.exists(tune_cache)
    s = afps.Sampler(0, tune_cache=tune_cache)
    dev = torch.device("cuda", 0)
    if case in ("headline", "fps2048", "ragged"):
        if case == "ragged":
            clouds, C, M = synth.ragged_batch(3, 256)
            k = [8 if m <= 8 else 16 for m in M]  # Sec. IV-D: k = 8 for M <= 8, else 16
        else:
            clouds, C = synth.object_batch(1, 32, 2048), 512
            M, k = (32, 16) if case == "headline" else (1, 0)
        xyz, off = synth.pack(clouds)
        x = torch.from_numpy(xyz).to(dev)
        ba = afps.BatchArgs(off, C, M, k, 0)
        out = torch.empty(ba.total_out, dtype=torch.int32, device=dev)
        if tune:
            s.autotune_batched(x, ba, out)
            s.sync()
            afps.afps_save_tuning(s.ctx, None)
        for _ in range(reps):
            s.sample_batched(x, ba, out=out)
        if case != "ragged":
            print("variant:", s.describe_plan(-(-2048 // M), -(-C // M), k, 32 * M))
    elif case == "clusters":
        import tempfile
        for N in (8192, 16384, 32768):
            x = torch.from_numpy(synth.slab_cloud(2, N)).to(dev)
            C = N // 4
            for P in (4, 8, 16):
                for W in (4, 8, 16, 32):
                    CS = -(-N // (32 * W * P))
                    if CS < 2 or CS > 16:
                        continue
                    path = os.path.join(tempfile.gettempdir(), "afps_profile_cluster.txt")
                    with open(path, "w") as f:
                        f.write(f"full:n{N}:c{C}:i1 1 {P} {W} {CS} 0 0\n")
                    sc = afps.Sampler(0, tune_cache=path)
                    out = sc.sample(x, C, 1, 0, 0)
                    sc.sync()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    for _ in range(reps):
                        sc.sample(x, C, 1, 0, 0, out=out)
                    e1.record()
                    sc.sync()
                    ms = e0.elapsed_time(e1) / reps
                    print(f"N={N} {sc.describe_plan(N, C, 0, 1):28s} {ms:8.3f} ms "
                          f"{ms * 1e6 / C:7.1f} ns/iteration", flush=True)
                    sc.close()
    elif case in ("cluster32k", "npdu32k"):
        x = torch.from_numpy(synth.slab_cloud(2, 32768)).to(dev)
        M, k = (1, 0) if case == "cluster32k" else (32, 16)
        for _ in range(reps):
            s.sample(x, 8192, M, k, 0)
    elif case in ("sort", "group", "knn", "coverage"):
        clouds = synth.object_batch(1, 32, 2048)
        if case == "sort":
            g = synth.rng(11)
            clouds = [c[g.permutation(c.shape[0])] for c in clouds]
        xyz, off = synth.pack(clouds)
        x = torch.from_numpy(xyz).to(dev)
        if case == "sort":
            for _ in range(reps):
                s.sort_by_key(x, off, afps.AFPS_KEY_X)
        else:
            ba = afps.BatchArgs(off, 512, 32, 16, 0)
            sel = s.sample_batched(x, ba)
            for _ in range(reps):
                if case == "group":
                    s.ball_query(x, off, sel, ba.out_off, 0.2, 32, 0)
                elif case == "knn":
                    s.knn(x, off, sel, ba.out_off, 32, 0)
                else:
                    s.coverage_radius(x, off, sel, ba.out_off)
    elif case == "chain":
        frame = torch.from_numpy(synth.lidar_frame(5)).to(dev)
        for _ in range(reps):
            cloud, fidx = frame, None
            for C in (16384, 4096, 1024, 256):
                n = cloud.shape[0]
                sel = s.sample(cloud, C, 32, 16, 0)
                nxt = torch.empty((C, 3), dtype=torch.float32, device=dev)
                nfr = torch.empty(C, dtype=torch.int32, device=dev)
                s.gather_levels([0, n], cloud, fidx, [0, C], sel, nxt, nfr)
                cloud, fidx = nxt, nfr
    else:
        raise SystemExit(f"unknown case {case!r}; one of {', '.join(CASES)}")
    s.sync()
    s.close()
    print(f"{case}: {reps} runs ok")


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("case", choices=CASES)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--tune-cache", default=None)
    a = ap.parse_args(argv)
    run(a.case, a.reps, a.tune_cache)
    return 0


if __name__ == "__main__":
    sys.exit(main())
