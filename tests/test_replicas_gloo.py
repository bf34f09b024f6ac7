"""The multi-GPU replica logic on CPU: two gloo ranks, no GPU.

Independent problems shard across ranks with no data-path exchange; only the
timing (max over ranks) and the item counts (sum) are combined. The same
functions run under NCCL when bench.py is launched with one rank per GPU.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1011_5964_gb300.replicas import reduce_over_ranks, shard, whole_job_rate


def test_shard_covers_every_item_once_and_balances():
    sizes = [128 ** 2, 512 ** 2, 256 ** 2, 384 ** 2, 192 ** 2, 512 ** 2, 128 ** 2]
    for world in (1, 2, 3, 8):
        parts = [shard(sizes, r, world) for r in range(world)]
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(sizes)
    with pytest.raises(ValueError):
        shard(sizes, 2, 2)


def test_without_a_process_group_it_is_one_rank():
    assert reduce_over_ranks(3.5, "max") == 3.5
    assert whole_job_rate(10, 2000.0) == pytest.approx(5.0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sizes = [100, 400, 400, 100, 300]
        mine = shard(sizes, rank, world)
        ms = 1000.0 + 500.0 * rank          # rank 1 is the slower one
        rate = whole_job_rate(len(mine), ms)
        mx = reduce_over_ranks(ms, "max")
        q.put((rank, mine, rate, mx))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine_counts_and_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    items = sorted(i for _, mine, _, _ in out for i in mine)
    assert items == list(range(5))
    for _, _, rate, mx in out:
        assert mx == 1500.0
        assert rate == pytest.approx(1000.0 * 5 / 1500.0)
