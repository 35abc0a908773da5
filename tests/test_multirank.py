"""Multi-rank host logic on CPU (gloo, world size 2): the split of the starts over ranks, the
winner over ranks, and the max/sum reductions bench.py uses for its whole-job numbers."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1212_4137_gb300.replicas import best_over_ranks, rank_starts


def test_rank_starts_partition():
    for r in (1, 5, 1024, 1027):
        for world in (1, 2, 3, 8):
            seen = []
            for rank in range(world):
                off, cnt = rank_starts(r, rank, world)
                seen.extend(range(off, off + cnt))
            assert seen == list(range(r))
    with pytest.raises(ValueError):
        rank_starts(4, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, objectives, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        win, val = best_over_ranks(objectives[rank], world, dist)
        import bench
        bench._dist = dist
        mx = bench.reduce_max(10.0 + rank, world)
        sm = bench.reduce_sum(1.5 * (rank + 1), world)
        bench.barrier(world)
        out[rank] = (win, val, mx, sm)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("objectives,winner", [((3.0, 5.0), 1), ((7.0, 7.0), 0), ((9.0, -1.0), 0)])
def test_best_over_ranks_gloo(objectives, winner):
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), objectives, out), nprocs=world, join=True,
                       start_method="spawn")
    for rank in range(world):
        win, val, mx, sm = out[rank]
        assert win == winner and val == max(objectives)
        assert mx == 11.0 and sm == 4.5
