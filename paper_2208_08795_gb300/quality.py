"""Sampling quality without a trained network: coverage radius on synthetic
clouds, for AFPS (Sec. III-B) and NPDU (Sec. III-C) against plain FPS.

The paper scores its variants by the mIoU of a pretrained PointNet++ on
ShapeNet (Table II, Fig. 6, Fig. 7); neither is available.  The coverage
radius R(S) = max_j min_{s in S} |p_j - p_s| is the quantity FPS greedily
shrinks (property P1), so R(variant) / R(FPS) on the same cloud measures how
much of FPS's coverage a variant keeps (1.0 = as good as FPS, larger =
worse).  Clouds are the object-scale generator of `synth` (2-5 primitive
surfaces, 2048 points, C = 512).  All sampling and radii run on the GPU
through the library.

    python -m paper_2208_08795_gb300.quality [--clouds 32]
"""
from __future__ import annotations

import argparse
import json
import sys

import numpy as np
import torch

from . import afps, build, synth

ORDERS = ("unsorted", "approx_x", "exact_x", "exact_z")


def storage_orders(clouds, seed: int = 7):
    """The clouds in the four storage orders of Table II."""
    g = synth.rng(seed)
    out = {}
    for name in ORDERS:
        res = []
        for P in clouds:
            if name == "unsorted":
                res.append(synth.shuffled(P, g))
            elif name == "approx_x":
                res.append(synth.approx_sort_by_axis(synth.shuffled(P, g), g, 0, 128))
            elif name == "exact_x":
                res.append(synth.sort_by_axis(P, 0))
            else:
                res.append(synth.sort_by_axis(P, 2))
        out[name] = res
    return out


def radii(sampler, clouds, C: int, M: int, k: int, method: int = 0) -> np.ndarray:
    """Coverage radius of NPDU-AFPS(C, M, k) on each cloud (start index 0)."""
    xyz, off = synth.pack(clouds)
    x = torch.from_numpy(xyz).cuda()
    ba = afps.BatchArgs(off, C, M, k, 0, method=method if method else None)
    sel = sampler.sample_batched(x, ba)
    r = sampler.coverage_radius(x, off, sel, ba.out_off)
    sampler.sync()
    return r.cpu().numpy()


def table_ii(sampler, clouds, C=512, Ms=(2, 8, 32)):
    """Mean R(AFPS)/R(FPS) per storage order and M (no NPDU)."""
    rows = {}
    for name, cl in storage_orders(clouds).items():
        base = radii(sampler, cl, C, 1, 0)
        rows[name] = {f"M={M}": float(np.mean(radii(sampler, cl, C, M, 0) / base)) for M in Ms}
    return rows


def fig6(sampler, clouds, C=512, ks=(4, 8, 16, 32, 64)):
    """NPDU on plain FPS (M = 1), mean R/R(FPS) per k and reading."""
    cl = storage_orders(clouds)["exact_x"]
    base = radii(sampler, cl, C, 1, 0)
    readings = {"default": 0, "full_first_pass": afps.AFPS_METHOD_FULL_FIRST_PASS,
                "window_has_sample": afps.AFPS_METHOD_WINDOW_HAS_SAMPLE}
    return {r: {f"k={k}": float(np.mean(radii(sampler, cl, C, 1, k, m) / base)) for k in ks}
            for r, m in readings.items()}


def fig7(sampler, clouds, C=512, Ms=(4, 8, 16, 32), ks=(4, 8, 16, 32)):
    """NPDU on AFPS, mean R/R(FPS) per (M, k); k = 0 is AFPS without NPDU."""
    cl = storage_orders(clouds)["exact_x"]
    base = radii(sampler, cl, C, 1, 0)
    return {f"M={M}": {f"k={k}": float(np.mean(radii(sampler, cl, C, M, k) / base))
                       for k in (0,) + tuple(ks)} for M in Ms}


def markdown(title, table) -> str:
    cols = list(next(iter(table.values())).keys())
    lines = [f"**{title}**", "", "| | " + " | ".join(cols) + " |",
             "|---|" + "---:|" * len(cols)]
    for r, vals in table.items():
        lines.append(f"| {r} | " + " | ".join(f"{vals[c]:.3f}" for c in cols) + " |")
    return "\n".join(lines)


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--clouds", type=int, default=32)
    ap.add_argument("--seed", type=int, default=1)
    a = ap.parse_args(argv)
    build.build()
    s = afps.Sampler(0)
    clouds = synth.object_batch(a.seed, a.clouds, 2048)
    res = {"table_ii": table_ii(s, clouds), "fig6": fig6(s, clouds), "fig7": fig7(s, clouds)}
    s.close()
    print(markdown("R(AFPS) / R(FPS) by storage order (Table II analogue)", res["table_ii"]))
    print()
    print(markdown("R(NPDU-FPS) / R(FPS) by window, M = 1 (Fig. 6 analogue)", res["fig6"]))
    print()
    print(markdown("R(NPDU-AFPS) / R(FPS), x-sorted (Fig. 7 analogue)", res["fig7"]))
    print(json.dumps(res))
    return 0


if __name__ == "__main__":
    sys.exit(main())
