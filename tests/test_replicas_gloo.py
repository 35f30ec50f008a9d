"""Multi-GPU layout of the benchmark, on CPU with gloo (world size 2): every
rank samples its own batch (weak scaling, no collective on the data path) and
only the step time is reduced, by max over ranks."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    from paper_2208_08795_gb300 import synth
    r, w, lr = bench.rank_info()
    seed = bench.batch_seed(r)
    clouds = synth.object_batch(seed, 2, 512)  # this rank's own shard
    idx = [oracle.afps(P, 128, 1, 0) for P in clouds]
    slowest = bench.max_over_ranks(float(10 * (rank + 1)), w)
    q.put((r, w, seed, slowest, [int(i[1:].sum()) for i in idx]))
    dist.destroy_process_group()


def test_two_ranks_shard_and_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, s0, m0, i0), (r1, w1, s1, m1, i1) = out
    assert (r0, r1) == (0, 1) and w0 == w1 == 2
    assert s0 != s1  # different batches per rank
    assert m0 == m1 == 20.0  # max over ranks
    assert i0 != i1
