"""The debug build (AFPS_DEBUG_CHECKS): every sampling kernel checks its
sector sizes and indices on the device and records a failure in the status
word, which afps_sync reports as AFPS_ERR_DEVICE_CHECK.  Run across the
kernel paths (warp, CTA, cluster; computed items and tables; the stride phase;
the window readings; host-resident points), no check may fail and every
result must still equal the oracle's.  The library is loaded in a child
process (one libafps per process)."""
import os
import subprocess
import sys

import pytest

from paper_2208_08795_gb300 import build as build_mod

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

CHILD = r'''
import sys
sys.path[:0] = [{root!r}, {tests!r}]
import numpy as np
import torch
import oracle
from paper_2208_08795_gb300 import afps as B, synth
B.load({lib!r})
s = B.Sampler(0)
n_ok = 0

def check(got, ref, what):
    global n_ok
    got = np.asarray(got)
    assert np.array_equal(got, ref), what
    n_ok += 1

objs = synth.object_batch(1, 16, 2048)
xyz, off = synth.pack(objs)
x = torch.from_numpy(xyz).cuda()
for M, k, start, method in ((32, 16, 0, 0), (4, 8, 3, 0), (1, 0, 0, 0), (16, 16, 2, 2), (8, 8, 0, 1)):
    ba = B.BatchArgs(off, 512, M, k, start, method=method if method else None)
    o = s.sample_batched(x, ba)
    s.sync()
    o = o.cpu().numpy()
    for b in (0, 15):
        check(o[ba.out_off[b]:ba.out_off[b + 1]],
              oracle.afps(objs[b], 512, M, k, start, method=method), ("batch", M, k, method, b))
mixed = [synth.uniform_cloud(3, 300), synth.slab_cloud(4, 9000), objs[2]]
xm, om = synth.pack(mixed)
ba = B.BatchArgs(om, [100, 2000, 512], [3, 1, 32], [5, 0, 16], 0)
o = s.sample_batched(torch.from_numpy(xm).cuda(), ba)
s.sync()
o = o.cpu().numpy()
for b, (P, C, M, k) in enumerate(zip(mixed, [100, 2000, 512], [3, 1, 32], [5, 0, 16])):
    check(o[ba.out_off[b]:ba.out_off[b + 1]], oracle.afps(P, C, M, k, 0), ("mixed", b))
big = synth.slab_cloud(2, 20000)
for C, M, k in ((1500, 1, 0), (5000, 8, 8), (5000, 1, 16)):
    o = s.sample(torch.from_numpy(big).cuda(), C, M, k, 7)
    s.sync()
    check(o.cpu().numpy(), oracle.afps(big, C, M, k, 7), ("single", C, M, k))
hx = torch.from_numpy(xyz).pin_memory().numpy()
ba = B.BatchArgs(off, 512, 32, 16, 0)
ho = torch.full((ba.total_out,), -1, dtype=torch.int32).pin_memory().numpy()
s.sample_batched_host_async(hx, ba, ho)
s.sync()
check(ho[ba.out_off[3]:ba.out_off[4]], oracle.afps(objs[3], 512, 32, 16, 0), "host-resident")
s.close()
print("debug checks ok", n_ok)
'''


def test_debug_build_kernels_pass_their_checks():
    lib = build_mod.build(debug=True)
    code = CHILD.format(root=ROOT, tests=HERE, lib=lib)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "debug checks ok" in r.stdout, r.stdout[-2000:]
