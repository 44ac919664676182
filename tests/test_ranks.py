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


def _tiny_instances():
    from paper_2609_26332_b300 import inputs
    out = []
    for i, (nx, ny) in enumerate([(16, 8), (24, 12), (40, 20), (32, 16), (16, 10), (48, 24), (20, 10)]):
        out.append(dict(nx=nx, ny=ny, R=0.35 * ny, theta=40.0 + 15.0 * i, psi0=0.005 + 0.004 * i))
    return out


def _step_instance(sp, steps=6):
    """One instance on the oracle (stands in for the GPU batch on CPU ranks)."""
    from oracle import Oracle, OracleParams, Wall
    from paper_2609_26332_b300 import inputs
    pb = inputs.bulk_phi(sp["psi0"], 1.0)
    phi0, psi0 = inputs.sessile_drop(sp["nx"], sp["ny"], sp["R"], 4.0, phi_b=pb, psi0=sp["psi0"])
    o = Oracle(OracleParams(nx=sp["nx"], ny=sp["ny"], psi_b=sp["psi0"], walls=[Wall(sp["theta"]), Wall(90.0)]),
               phi0, psi0)
    o.step(steps)
    return o.fields()["phi"]


def _shard_worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    specs = _tiny_instances()
    lo, hi = ranks.instance_share([s["nx"] * s["ny"] for s in specs], rank, world)
    mine = {i: _step_instance(specs[i]) for i in range(lo, hi)}
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    if rank == 0:
        merged = {}
        for part in gathered:
            assert not set(part) & set(merged)          # disjoint shares
            merged.update(part)
        out["merged"] = merged
        out["shares"] = [ranks.instance_share([s["nx"] * s["ny"] for s in specs], r, world) for r in range(world)]
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_step_disjoint_shares_of_one_list():
    """Two gloo ranks each step their share of one global instance list (the batch
    workload's split); gathered, the shares cover every instance once and reproduce the
    single-rank results exactly."""
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    mp.start_processes(_shard_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    merged = out["merged"]
    specs = _tiny_instances()
    assert sorted(merged) == list(range(len(specs)))
    (a0, b0), (a1, b1) = out["shares"]
    assert a0 == 0 and b0 == a1 and b1 == len(specs) and b0 > 0 and b1 > b0
    for i, sp in enumerate(specs):
        assert np.array_equal(merged[i], _step_instance(sp))
