"""Multi-GPU by replicas: independent problems dealt across ranks.

A single solve does not shard here (one GPU holds even an 8192^2 problem);
what scales across GPUs is a stream or batch of independent problems.  Each
rank takes a deterministic share -- longest-processing-time order by bytes
moved (problem points), assigned greedily to the least-loaded rank -- and
runs it through its own GPU with no collective on the data path.  Ranks only
exchange host metadata (e.g. per-rank timings or checksums) at the end.
"""

import heapq


def problem_cost(n_x, n_y=None):
    """Relative cost of one problem: its grid points (all passes are linear in them)."""
    return n_x * (n_x if n_y is None else n_y)


def shard(costs, world):
    """Assign item indices to `world` ranks; returns a list of index lists.

    Greedy LPT: items in decreasing cost (ties by index) go to the rank with
    the smallest load so far (ties by rank).  Deterministic, so every rank
    computes the same assignment without communicating.
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0, r) for r in range(world)]
    out = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    for lst in out:
        lst.sort()
    return out


def my_share(costs, rank, world):
    """Indices this rank runs."""
    return shard(costs, world)[rank]


def batch_share_requests(problems, rank, world, plans, inputs, outputs):
    """This rank's share of `problems` (workloads.Problem list) as a request
    array for one persistent batch, and the indices it covers.  `plans[n]`,
    `inputs[i]`, `outputs[i]` are this rank's plan handles and fields (device
    tensors, or raw device addresses); nothing is launched."""
    from . import fsolve

    ops = {"poisson": fsolve.FS_OP_POISSON, "diffusion": fsolve.FS_OP_DIFFUSION, "wave": fsolve.FS_OP_WAVE}
    idx = my_share([problem_cost(p.n) for p in problems], rank, world)
    reqs = [fsolve.fs_request(ops[problems[i].op], plan=plans[problems[i].n], in_u=inputs[i], out_u=outputs[i],
                              D=problems[i].D, c=problems[i].c, t=problems[i].t) for i in idx]
    return (fsolve.fs_request_array(reqs) if reqs else None), idx


def run_batch_share(problems, rank, world, plans, inputs, outputs, stream=None):
    """Submit this rank's share of `problems` as one persistent batch on the
    current GPU; returns the batch ticket (0 for an empty share) and the
    indices it covers."""
    from . import fsolve

    arr, idx = batch_share_requests(problems, rank, world, plans, inputs, outputs)
    ticket = fsolve.fs_batch_submit(arr, stream) if arr is not None else 0
    return ticket, idx
