"""One solve split by slabs, on the GPU (sharded.py with the library's slab
entry points fs_rows_forward / fs_columns_apply / fs_rows_inverse).

One GPU is available, so every rank of a 1-, 2- or 4-way split runs in this
process (sharded.emulate: the all-to-all exchanges become copies; no kernel
waits on another).  The result must match the float64 oracle at the dtype's
bar (rel-L2 <= 1e-5 FP32, <= 1e-12 FP64), and the unsharded solve of the same
plan within the same bar.
"""

import numpy as np
import pytest
import torch

import oracle
from paper_2412_12308_gb300 import fsolve, sharded

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-12}


@pytest.mark.parametrize("nx,ny,dtype", [(256, 192, 0), (1024, 1024, 0), (160, 96, 1), (64, 64, 1)])
@pytest.mark.parametrize("op", ["poisson", "diffusion", "wave"])
def test_emulated_shards_match_oracle(gpu_lib, nx, ny, dtype, op):
    lx, ly, D, c, t = 1.0, 1.3, 0.002, 1.1, 0.41
    rng = np.random.default_rng(nx * 3 + ny)
    f = rng.standard_normal((ny, nx)).astype(np.float32).astype(np.float64)
    if op == "poisson":
        want = oracle.poisson(f, lx, ly)
    elif op == "diffusion":
        want = oracle.diffusion(f, D, t, lx, ly)
    else:
        want = oracle.wave(f, None, c, t, lx, ly)
    tdt = torch.float32 if dtype == 0 else torch.float64
    fd = torch.tensor(f, dtype=tdt, device="cuda")
    plan = fsolve.fs_plan_create(nx, ny, lx, ly, dtype)
    try:
        whole = torch.empty_like(fd)
        if op == "poisson":
            fsolve.fs_poisson_solve(plan, fd, whole)
        elif op == "diffusion":
            fsolve.fs_diffusion_solve(plan, fd, D, t, whole)
        else:
            fsolve.fs_wave_solve(plan, fd, None, c, t, whole)
        back = sharded.Library(plan, nx, ny, dtype)
        for world in (1, 2, 4):
            got = sharded.emulate(back, fd, world, op, D, c, t)
            torch.cuda.synchronize()
            g = got.double().cpu().numpy()
            assert np.linalg.norm(g - want) / np.linalg.norm(want) <= TOL[dtype], (world, op)
            w = whole.double().cpu().numpy()
            assert np.linalg.norm(g - w) / np.linalg.norm(w) <= TOL[dtype], (world, op)
    finally:
        fsolve.fs_plan_destroy(plan)


def test_slab_entry_points_reject_bad_ranges(gpu_lib):
    plan = fsolve.fs_plan_create(64, 64, 1.0, 1.0, 0)
    try:
        cols = torch.zeros((8, 64), dtype=torch.complex64, device="cuda")
        with pytest.raises(fsolve.FsError):
            fsolve.fs_columns_apply(plan, 30, 8, fsolve.FS_OP_POISSON, cols)  # 30 + 8 > 33
        with pytest.raises(fsolve.FsError):
            fsolve.fs_columns_apply(plan, 0, 8, 7, cols)  # not an operator
        with pytest.raises(fsolve.FsError):
            fsolve.fs_columns_apply(plan, 0, 8, fsolve.FS_OP_WAVE, cols, c=0.0, t=1.0)
        f = torch.zeros((4, 64), device="cuda")
        spec = torch.zeros((33, 4), dtype=torch.complex64, device="cuda")
        with pytest.raises(fsolve.FsError):
            fsolve.fs_rows_forward(plan, 0, f[:0], spec[:0])
        with pytest.raises(fsolve.FsError):  # wrong element type for an FP32 plan
            fsolve.fs_rows_forward(plan, 4, f.double(), spec)
    finally:
        fsolve.fs_plan_destroy(plan)
