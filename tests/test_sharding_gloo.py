"""Multi-rank site sharding on CPU: two gloo ranks partition the 64 uneven sites.

Each rank computes its own share (no data-path collective); the test gathers
the shares and the per-rank loads to check that the partition is disjoint,
complete, identical on every rank and balanced, and that the max-over-ranks
time reduction used by the benchmark agrees.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2005_07834_gb300 import sharding, synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = synth.batched_64_sites()
    K = wl.orbitals.nk * wl.orbitals.nbands
    mine = sharding.shard_sites(wl.sites, K, wl.nfreq, rank, world)
    load = sum(sharding.site_cost(wl.sites[i].npts, K, wl.nfreq) for i in mine)
    shares = [None] * world
    dist.all_gather_object(shares, mine)
    t = torch.tensor([float(rank + 1)])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    loads = [None] * world
    dist.all_gather_object(loads, load)
    if rank == 0:
        out.put((shares, loads, float(t.item())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_site_sharding():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    shares, loads, tmax = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    allsites = sorted(shares[0] + shares[1])
    assert allsites == list(range(64))
    assert not set(shares[0]) & set(shares[1])
    assert max(loads) / min(loads) < 1.05
    assert tmax == 2.0


def test_lpt_partition_properties():
    costs = [5.0, 1.0, 4.0, 3.0, 3.0, 2.0]
    parts = sharding.lpt_partition(costs, 3)
    assert sorted(sum(parts, [])) == list(range(6))
    loads = [sum(costs[i] for i in p) for p in parts]
    assert max(loads) == 6.0
    assert sharding.lpt_partition(costs, 1) == [list(range(6))]
    with pytest.raises(ValueError):
        sharding.lpt_partition(costs, 0)
