"""The N > 1 benchmark path on CPU: two gloo ranks pick disjoint problem ranges (weak scaling,
no data-path collective), agree on the slowest rank's time and on the summed work, and compute
the same flops-balanced partition of one uneven batch (strong scaling)."""
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
    tot = bench.sum_over_ranks(100.0 + rank, dist, torch.device("cpu"))
    # strong scaling of the uneven workload: every rank computes the same balanced partition
    u = synth.workload("pgo_se3_uneven_b1024", batch=64)
    n_b = np.diff(u.pose_offsets).astype(np.float64)
    parts, load = bench.balanced_partition(6.0 * n_b ** 3 / 3.0, world)
    out.put((rank, first, n, float(b.theta_init[5, 3]), t, tot, parts, load))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_problems_and_reduce_time():
    from paper_2207_09442_b300 import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    (r0, f0, n0, x0, t0, s0, P0, L0), (r1, f1, n1, x1, t1, s1, P1, L1) = res
    assert (f0, n0, f1, n1) == (0, 4, 4, 4)          # disjoint, contiguous problem ranges
    assert x0 != x1                                  # different seeded problems
    assert t0 == t1 == 11.0                          # max over ranks
    assert s0 == s1 == 201.0                         # units summed over ranks
    # the balanced partition: identical on both ranks, disjoint, complete, loads within 1 %
    assert P0 == P1 and L0 == L1
    assert sorted(P0[0] + P0[1]) == list(range(64)) and not set(P0[0]) & set(P0[1])
    assert max(L0) / (sum(L0) / 2) < 1.01
    # equal counts would not be balanced on this uneven batch
    u = synth.workload("pgo_se3_uneven_b1024", batch=64)
    c = 6.0 * np.diff(u.pose_offsets).astype(np.float64) ** 3 / 3.0
    assert max(c[:32].sum(), c[32:].sum()) / (c.sum() / 2) > 1.05
    ref = synth.workload("pgo_se3_b256", batch=8)
    assert np.allclose(ref.theta_init[ref.pose_offsets[4] + 5, 3], x1)
