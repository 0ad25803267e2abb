"""The multi-GPU path of the benchmark is replicas only: every rank solves its
own independent subproblem and the job's numbers add the units over the ranks
and take the slowest rank's time.  This runs that aggregation (and the seed
of each replica) as two gloo processes on the CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sums, maxes = bench.reduce_over_ranks(world, "cpu", [1000 * (rank + 1), 2],
                                          [10.0 + 5 * rank, 3.0 - rank])
    out.put((rank, sums, maxes, bench.replica_seed(rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, sums, maxes, seed in res:
        assert sums == [3000.0, 4.0]        # units of both replicas
        assert maxes == [15.0, 3.0]         # the slowest rank's times
        assert seed == rank                 # independent subproblems
    assert res[0][3] != res[1][3]


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(1, "cpu", [5, 6], [7]) == ([5.0, 6.0], [7.0])
