"""Host logic of the replica (multi-GPU) path on CPU ranks: gloo, world size 2."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1904_06376_b300 import replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, costs, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        share = replicas.rank_share(costs, rank, world)
        mine = sum(costs[i] for i in share)
        slowest = replicas.max_over_ranks(10.0 + rank, dist)  # rank 1 is the slower one
        gathered = [None] * world
        dist.all_gather_object(gathered, share)
        out.put((rank, share, mine, slowest, gathered))
    finally:
        dist.destroy_process_group()


def test_two_ranks_partition_and_max():
    world = 2
    costs = [replicas.solve_cost(n) for n in (64, 4096, 300, 1024, 2000, 77, 512, 3000, 900)]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, costs, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    shares = [r[1] for r in res]
    # the ranks agree on the assignment without exchanging it ...
    assert res[0][4] == res[1][4] == shares
    # ... which covers every unit exactly once
    assert sorted(i for s in shares for i in s) == list(range(len(costs)))
    # the slowest rank's time reaches every rank
    assert res[0][3] == res[1][3] == 11.0
    # longest-first greedy: no rank carries more than the largest unit above the mean
    loads = [r[2] for r in res]
    assert max(loads) - sum(loads) / world <= max(costs)


def test_partition_deterministic_and_balanced():
    costs = [float(c) for c in range(1, 101)]
    a = replicas.partition_by_cost(costs, 4)
    assert a == replicas.partition_by_cost(costs, 4)
    loads = [sum(costs[i] for i in s) for s in a]
    assert max(loads) - min(loads) <= 4.0
    assert replicas.partition_by_cost(costs, 1) == [list(range(100))]
    with pytest.raises(ValueError):
        replicas.partition_by_cost(costs, 0)


def test_max_over_ranks_without_group():
    assert replicas.max_over_ranks(3.5) == 3.5


def test_reference_arm_other_ranks_do_no_work(capsys):
    """Under torchrun only rank 0 runs and prints the reference line."""
    import bench

    class A:
        steps, warmup, m, n, k, mode = 1, 0, 64, 64, 64, 6

    assert bench.run_reference(A(), 1, 2) is None
    assert capsys.readouterr().out == ""
    torch.manual_seed(0)
