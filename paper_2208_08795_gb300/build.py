"""Build libafps.so (the CUDA kernels and the C ABI of include/afps.h) for
sm_103a with nvcc.  Translation units compile in parallel into _build/ and
link into paper_2208_08795_gb300/libafps.so.  Run ``python -m
paper_2208_08795_gb300.build`` or call :func:`build`."""
from __future__ import annotations

import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD_DIR = os.path.join(PKG, "_build")
LIBRARY = os.path.join(PKG, "libafps.so")
# debug build: device-side index checks (AFPS_DEBUG_CHECKS), a library of its own
BUILD_DIR_DEBUG = os.path.join(PKG, "_build_debug")
LIBRARY_DEBUG = os.path.join(PKG, "libafps_debug.so")
HEADER = os.path.join(ROOT, "include", "afps.h")
SOURCES = ["afps_warp.cu", "afps_win.cu", "afps_cta.cu", "afps_gather.cu", "afps_api.cu", "afps_noalloc.cu",
           "afps_server.cu", "afps_sort.cu", "afps_coverage.cu", "afps_group.cu",
           "afps_knn.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-Xcompiler", "-Wall", "-I", os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _deps():
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    return hdrs + [HEADER]


def _stale(target: str, inputs) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(i) > t for i in inputs)


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compile and link libafps.so (debug=True: libafps_debug.so, with the
    device-side index checks) if any source changed; returns its path."""
    build_dir = BUILD_DIR_DEBUG if debug else BUILD_DIR
    library = LIBRARY_DEBUG if debug else LIBRARY
    flags = NVCC_FLAGS + (["-DAFPS_DEBUG_CHECKS"] if debug else [])
    os.makedirs(build_dir, exist_ok=True)
    nvcc = _nvcc()
    deps = _deps()
    objs, procs = [], []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(build_dir, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + deps):
            cmd = [nvcc] + flags + ["-c", s, "-o", o]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE,
                                                stderr=subprocess.STDOUT, text=True)))
    errors = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errors.append(f"{src}:\n{out}")
        elif verbose and out:
            print(out, file=sys.stderr)
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
    if force or procs or _stale(library, objs):
        tmp = library + ".tmp"
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
        os.replace(tmp, library)
    return library


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, debug="--debug" in sys.argv))
