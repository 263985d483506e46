"""The multi-GPU path of the benchmark is replicas only (the traversal of one
target does not shard): every rank runs the same workload and rank 0
reports the slowest rank's time and the sum of all ranks' work.  This checks
that reduction with two gloo ranks on the CPU."""
import os
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    times, work = bench.reduce_over_ranks([10.0 + rank, 3.0 * (rank + 1)], [100 * (rank + 1), rank, 7], "cpu")
    out[rank] = (times, work)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_max_time_sum_work():
    port = 29500 + os.getpid() % 1000
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
        got = dict(out)
    for r in (0, 1):
        times, work = got[r]
        assert times == [11.0, 6.0]
        assert work == [300, 1, 14]
