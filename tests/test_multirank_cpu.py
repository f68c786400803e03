"""The multi-rank (replicas) timing path of bench.py on CPU: two gloo ranks, barrier, max over
ranks, whole-job value = units of all ranks / max time."""
import os

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    dist.barrier()
    t_local = [2.0, 5.0][rank]
    t_max = bench.reduce_max(t_local, "cpu", world)
    units = 100.0 * world
    q.put((rank, t_max, units / t_max))
    dist.destroy_process_group()


def test_two_rank_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29531
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    assert [o[1] for o in out] == [5.0, 5.0]
    assert out[0][2] == pytest.approx(40.0)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.reduce_max(3.5, "cpu", 1) == 3.5
