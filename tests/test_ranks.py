"""Multi-rank host logic on CPU: instance shares partition the list, and the timing
reduction (barrier + max over ranks) works across two gloo processes."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2609_26332_b300 import ranks


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_instance_shares_partition_the_list(world):
    from paper_2609_26332_b300 import inputs
    specs = inputs.batch_instances(512, seed=3)
    cells = [s["nx"] * s["ny"] for s in specs]
    shares = [ranks.instance_share(cells, r, world) for r in range(world)]
    assert shares[0][0] == 0 and shares[-1][1] == len(cells)
    for (a, b), (c, d) in zip(shares, shares[1:]):
        assert b == c and a <= b
    load = [sum(cells[a:b]) for a, b in shares]
    assert max(load) - min(load) <= max(cells)          # balanced to within one instance
    assert all(b > a for a, b in shares)


def test_fewer_instances_than_ranks():
    shares = [ranks.instance_share([10, 20], r, 4) for r in range(4)]
    covered = sorted(i for a, b in shares for i in range(a, b))
    assert covered == [0, 1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    t = ranks.max_over_ranks(10.0 + rank, dist)
    r, w, _ = ranks.rank_world()
    out[rank] = (t, r, w)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_processes():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    assert dict(out) == {0: (11.0, 0, 2), 1: (11.0, 1, 2)}
    assert ranks.max_over_ranks(3.5) == 3.5
