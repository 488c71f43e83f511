"""The N > 1 path of the bench on CPU: two gloo ranks plan their replicas
(disjoint chain ranges, distinct start clouds) and aggregate the whole-job
throughput over the slowest rank, as bench.py does over NCCL."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    C, steps = 64, 5
    plan = bench.replica_plan(rank, world, C)
    my_ms = 100.0 + 50.0 * rank  # rank 1 is the slower one
    g = [torch.zeros(1) for _ in range(world)]
    dist.all_gather(g, torch.tensor([my_ms]))
    value, t_max = bench.aggregate([float(t.item()) for t in g], world, C, steps)
    ranges = [None] * world
    dist.all_gather_object(ranges, (plan["chain0"], plan["chain0"] + plan["chains"],
                                    plan["start_seed"]))
    if rank == 0:
        out.put((value, t_max, ranges))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_replicas_and_aggregate():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    value, t_max, ranges = out.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert t_max == 150.0                            # the slowest rank's time
    assert value == pytest.approx(2 * 64 * 5 / 0.150)  # all ranks' chain-steps
    (a0, a1, s0), (b0, b1, s1) = ranges
    assert (a0, a1) == (0, 64) and (b0, b1) == (64, 128)  # disjoint chain ranges
    assert s0 != s1                                     # distinct start clouds
