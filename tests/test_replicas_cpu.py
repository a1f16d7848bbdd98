"""Replica sharding across ranks, on CPU with gloo (world size 2).

The multi-GPU path runs independent problems on each rank with no data-path
collective.  Here two CPU ranks compute their shares of a 64-problem batch
mix, solve them with the float64 oracle (standing in for each rank's GPU),
and exchange only host metadata: the shares must be disjoint, cover every
problem, be byte-balanced, and the gathered per-problem results must equal a
single-process run.
"""

import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2412_12308_gb300 import replicas, workloads as wl


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _solve(p):
    import oracle

    f = p.field(np.float64)
    if p.op == "poisson":
        u = oracle.poisson(f, p.lx, p.ly)
    elif p.op == "diffusion":
        u = oracle.diffusion(f, p.D, p.t, p.lx, p.ly)
    else:
        u = oracle.wave(f, None, p.c, p.t, p.lx, p.ly)
    return float(np.sum(u * u)), float(u.mean())


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    probs = wl.batch_mix(seed=21, count=64, sizes=(8, 16, 24, 32, 40, 48, 64))
    mine = replicas.my_share([replicas.problem_cost(p.n) for p in probs], rank, world)
    results = {i: _solve(probs[i]) for i in mine}
    gathered = [None] * world
    dist.all_gather_object(gathered, {"rank": rank, "idx": mine, "res": results})
    if rank == 0:
        q.put(gathered)
    dist.barrier()
    dist.destroy_process_group()


def test_shard_is_deterministic_disjoint_and_balanced():
    costs = [replicas.problem_cost(n) for n in (2048, 1024, 1024, 512, 512, 512, 256, 128, 64, 64, 8192)]
    for world in (1, 2, 3, 4, 8):
        a = replicas.shard(costs, world)
        assert a == replicas.shard(costs, world)
        flat = sorted(i for lst in a for i in lst)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in lst) for lst in a]
        assert max(loads) - min(loads) <= max(costs)
    with pytest.raises(ValueError):
        replicas.shard(costs, 0)


def test_two_gloo_ranks_match_single_process():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    probs = wl.batch_mix(seed=21, count=64, sizes=(8, 16, 24, 32, 40, 48, 64))
    idx = [g["idx"] for g in sorted(gathered, key=lambda g: g["rank"])]
    assert not set(idx[0]) & set(idx[1])
    assert sorted(idx[0] + idx[1]) == list(range(64))
    merged = {}
    for g in gathered:
        merged.update(g["res"])
    for i in (0, 7, 31, 63):
        assert merged[i] == _solve(probs[i])


def _assembly_worker(rank, world, port, q):
    """Each rank assembles the request array of its share through the product
    code (replicas.batch_share_requests); plans and fields are stand-in
    handles and addresses, so nothing reaches a GPU."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    probs = wl.batch_mix()
    plans = {n: 0x1000 + n for n in sorted({p.n for p in probs})}
    inputs = {i: 0x10_0000_0000 + (i << 24) for i in range(len(probs))}
    outputs = {i: 0x20_0000_0000 + (i << 24) for i in range(len(probs))}
    arr, idx = replicas.batch_share_requests(probs, rank, world, plans, inputs, outputs)
    rows = [(r.op, r.plan, r.in_u, r.out_u, r.D, r.c, r.t, r.keep, r.parent, r.state, r.in_v, r.out_v)
            for r in arr]
    gathered = [None] * world
    dist.all_gather_object(gathered, {"rank": rank, "idx": idx, "rows": rows})
    if rank == 0:
        q.put(gathered)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_batch_share_request_assembly_on_gloo_ranks(world):
    """The 512-problem mix split across gloo ranks: shares are disjoint and
    cover every problem, each rank's requests carry its problems' operator,
    parameters, plan and field addresses in share order, and the shares'
    grid points are balanced to within the largest problem."""
    from paper_2412_12308_gb300 import fsolve

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_assembly_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    gathered = sorted(q.get(timeout=300), key=lambda g: g["rank"])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    probs = wl.batch_mix()
    ops = {"poisson": fsolve.FS_OP_POISSON, "diffusion": fsolve.FS_OP_DIFFUSION, "wave": fsolve.FS_OP_WAVE}
    seen = []
    for g in gathered:
        assert g["idx"] == sorted(g["idx"])
        assert len(g["rows"]) == len(g["idx"])
        for i, row in zip(g["idx"], g["rows"]):
            p = probs[i]
            assert row == (ops[p.op], 0x1000 + p.n, 0x10_0000_0000 + (i << 24), 0x20_0000_0000 + (i << 24),
                           p.D, p.c, p.t, 0, 0, None, None, None)
        seen += g["idx"]
    assert sorted(seen) == list(range(len(probs)))
    loads = [sum(probs[i].n ** 2 for i in g["idx"]) for g in gathered]
    assert max(loads) - min(loads) <= max(p.n ** 2 for p in probs)
