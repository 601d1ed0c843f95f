"""Multi-rank host logic on CPU: two gloo ranks shard signals without overlap and reduce timings."""
import os

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1606_07407_gb300 import dist as D


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, lr = D.world_info()
        seeds = D.rank_seed_offsets(r, 8)
        gathered = [None] * world
        dist.all_gather_object(gathered, seeds)
        t_max = D.max_over_ranks(1.0 + r, device="cpu")
        m_sum = D.sum_over_ranks(1000.0 * (r + 1), device="cpu")
        D.barrier()
        out.put((r, w, gathered, t_max, m_sum))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 2000)
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, gathered, t_max, m_sum in res:
        assert w == 2
        flat = [s for g in gathered for s in g]
        assert len(flat) == len(set(flat)) == 16          # no signal recovered twice
        assert t_max == 2.0 and m_sum == 3000.0           # max of times, sum of modes


def test_single_process_reductions_are_identity():
    assert D.max_over_ranks(3.5, device="cpu") == 3.5
    assert D.sum_over_ranks(7.0, device="cpu") == 7.0
    assert D.rank_seed_offsets(2, 3) == [2000, 2001, 2002]
    with pytest.raises(ValueError):
        D.rank_seed_offsets(0, 5000)
