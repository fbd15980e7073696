"""The N > 1 benchmark path on CPU: two gloo ranks pick disjoint problem ranges (weak scaling,
no data-path collective) and agree on the slowest rank's time."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    from paper_2207_09442_b300 import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    first, n = bench.rank_problems(rank, 4)
    b = synth.workload("pgo_se3_b256", batch=n, first=first)
    t = bench.max_over_ranks(10.0 + rank, dist, torch.device("cpu"))
    out.put((rank, first, n, float(b.theta_init[5, 3]), t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_problems_and_reduce_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    (r0, f0, n0, x0, t0), (r1, f1, n1, x1, t1) = res
    assert (f0, n0, f1, n1) == (0, 4, 4, 4)          # disjoint, contiguous problem ranges
    assert x0 != x1                                  # different seeded problems
    assert t0 == t1 == 11.0                          # max over ranks
    from paper_2207_09442_b300 import synth
    ref = synth.workload("pgo_se3_b256", batch=8)
    assert np.allclose(ref.theta_init[ref.pose_offsets[4] + 5, 3], x1)
