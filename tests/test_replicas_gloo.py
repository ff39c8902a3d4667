"""The multi-process path of bench.py on the CPU: two ranks over gloo (the
bench runs one replica per GPU with no data-path collective, so the only
exchange is the timing rule: the job's time is the maximum over the ranks,
and its value counts the pairs of all replicas)."""
import os
import sys

import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = [3.25, 7.5][rank]
    ms = bench.job_ms(local, world, "cpu")
    out[rank] = (ms, bench.job_value(world, 1000, 50, ms / 10))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest():
    world, port = 2, 29500 + os.getpid() % 1000
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 7.5
    # value: both replicas' pairs over the slowest rank's step time
    assert abs(res[0][1] - 2 * 1000 * 50 / (0.75e-3)) <= 1e-6 * res[0][1]


def test_single_process_is_its_own_time():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_ms(4.0, 1, "cpu") == 4.0
    assert bench.job_value(1, 10, 3, 2.0) == 10 * 3 / 2e-3
