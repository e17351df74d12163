"""Host logic of bench.py's multi-process path with world_size 2 over gloo on
CPU: each rank docks its own replica (distinct seeds, no data exchange), the
step time is the max over ranks and the throughput the sum of all ranks'
evaluations over that time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    my_time = 1.5 + rank          # rank 1 is the slower one
    my_evals = 1000.0 * (rank + 1)
    t = bench.max_over_ranks(my_time)
    n = bench.sum_over_ranks(my_evals)
    bench.barrier()
    q.put((rank, bench.replica_seed(7, rank), t, n, bench.dist_env()[:2]))
    dist.destroy_process_group()


def test_two_rank_timing_and_replicas():
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
    (r0, s0, t0, n0, e0), (r1, s1, t1, n1, e1) = out
    assert s0 != s1                       # independent replicas
    assert t0 == t1 == 2.5                # max over ranks
    assert n0 == n1 == 3000.0             # whole-job evaluations
    assert e0 == (0, 2) and e1 == (1, 2)
