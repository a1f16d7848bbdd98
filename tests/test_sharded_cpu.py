"""One solve split across ranks by slabs (sharded.py), on CPU.

The decomposition and the two all-to-all exchanges are the product code; the
local steps of each rank (x transforms of its rows, column transforms with the
operator of its x frequencies, inverse x transforms) are done here by a
float64 stand-in built from the oracle's direct DFT (Eq. DFT along one axis)
and the Sec. III multipliers, since the CPU ranks have no GPU.  The gathered
result must equal the oracle's unsharded solve.  Runs as gloo process groups
of 2 and 4 ranks, and single-process emulations of 1 to 5 ranks; uneven
slabs (ny or nx/2+1 not divisible by the rank count) are included.
"""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from oracle.solve import omega_axis
from paper_2412_12308_gb300 import sharded


class OracleSteps:
    """Per-rank local steps in float64 on the host (test stand-in for the GPU)."""

    def __init__(self, nx, ny, lx, ly):
        self.nx, self.ny = nx, ny
        self.wx, self.wy = omega_axis(nx, lx), omega_axis(ny, ly)

    def rows_forward(self, f_slab):
        X = oracle.dft1(f_slab.numpy(), axis=1, sign=-1)[:, : self.nx // 2 + 1]
        return torch.from_numpy(np.ascontiguousarray(X.T))  # [nx/2+1][rows]

    def columns_apply(self, a0, cols, op, D, c, t):
        na = cols.shape[0]
        Y = oracle.dft1(cols.numpy(), axis=1, sign=-1)  # along y
        w2 = self.wx[a0:a0 + na, None] ** 2 + self.wy[None, :] ** 2
        if op == "poisson":
            m = np.zeros_like(w2)
            m[w2 > 0] = -1.0 / w2[w2 > 0]
        elif op == "diffusion":
            m = np.exp(-D * t * w2)
        else:
            m = np.cos(c * np.sqrt(w2) * t)
        out = oracle.dft1(Y * m / (self.nx * self.ny), axis=1, sign=+1)
        cols.copy_(torch.from_numpy(out))

    def rows_inverse(self, spec):
        S = spec.numpy().T  # [rows][nx/2+1]
        full = np.concatenate([S, np.conj(S[:, 1:self.nx // 2][:, ::-1])], axis=1)
        full[:, 0] = full[:, 0].real
        full[:, self.nx // 2] = full[:, self.nx // 2].real
        return torch.from_numpy(np.ascontiguousarray(oracle.dft1(full, axis=1, sign=+1).real))


def _want(f, op, lx, ly, D, c, t):
    if op == "poisson":
        return oracle.poisson(f, lx, ly)
    if op == "diffusion":
        return oracle.diffusion(f, D, t, lx, ly)
    return oracle.wave(f, None, c, t, lx, ly)


CASES = [(32, 24, "poisson"), (40, 30, "diffusion"), (16, 48, "wave"), (24, 20, "poisson")]


def _field(nx, ny, seed):
    return np.random.default_rng(seed).standard_normal((ny, nx))


def test_partition():
    assert sharded.partition(10, 3) == [(0, 4), (4, 3), (7, 3)]
    for n in (1, 7, 64, 1025):
        for w in (1, 2, 3, 8):
            if w > n:
                continue
            p = sharded.partition(n, w)
            assert sum(c for _, c in p) == n
            assert all(p[i][0] + p[i][1] == p[i + 1][0] for i in range(w - 1))
            assert max(c for _, c in p) - min(c for _, c in p) <= 1
    with pytest.raises(ValueError):
        sharded.partition(4, 0)
    with pytest.raises(ValueError):
        sharded.Layout(8, 2, 4)  # more ranks than rows


@pytest.mark.parametrize("world", [1, 2, 3, 5])
@pytest.mark.parametrize("nx,ny,op", CASES)
def test_emulated_ranks_match_oracle(nx, ny, op, world):
    lx, ly, D, c, t = 1.0, 1.4, 0.02, 1.3, 0.37
    f = _field(nx, ny, nx + ny)
    got = sharded.emulate(OracleSteps(nx, ny, lx, ly), torch.from_numpy(f), world, op, D, c, t).numpy()
    want = _want(f, op, lx, ly, D, c, t)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 1e-12


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lx, ly, D, c, t = 1.0, 1.4, 0.02, 1.3, 0.37
    res = {}
    for nx, ny, op in CASES:
        lay = sharded.Layout(nx, ny, world)
        f = _field(nx, ny, nx + ny)
        y0, cnt = lay.rows[rank]
        u = sharded.solve_rank(OracleSteps(nx, ny, lx, ly), lay, rank, torch.from_numpy(f[y0:y0 + cnt].copy()),
                               op, D, c, t)
        res[(nx, ny, op)] = (y0, u.numpy())
    gathered = [None] * world
    dist.all_gather_object(gathered, res)
    if rank == 0:
        q.put(gathered)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_gloo_ranks_match_oracle(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    gathered = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    lx, ly, D, c, t = 1.0, 1.4, 0.02, 1.3, 0.37
    for nx, ny, op in CASES:
        parts = sorted((g[(nx, ny, op)] for g in gathered), key=lambda x: x[0])
        got = np.concatenate([u for _, u in parts], axis=0)
        want = _want(_field(nx, ny, nx + ny), op, lx, ly, D, c, t)
        assert got.shape == want.shape
        assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 1e-12, (nx, ny, op, world)
