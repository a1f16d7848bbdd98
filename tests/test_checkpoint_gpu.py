"""State checkpoints (GPU): save, then load into a fresh state of another plan
with the same grid, domain and dtype; advances after the load are
bit-identical to advances of the saved state (the kept spectra fix the
solution at every t).  Mismatched checkpoints are rejected."""

import numpy as np
import pytest
import torch

from paper_2412_12308_gb300 import fsolve as fs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("n", [64, 384, 1024])
def test_state_checkpoint_roundtrip(gpu_lib, n, dtype):
    tdt = torch.float32 if dtype == 0 else torch.float64
    rng = np.random.default_rng(n + dtype)
    u0, v0, s = (torch.tensor(rng.standard_normal((n, n)), dtype=tdt, device="cuda") for _ in range(3))
    p1 = fs.fs_plan_create(n, n, 2.0, 1.5, dtype)
    p2 = fs.fs_plan_create(n, n, 2.0, 1.5, dtype)
    a = fs.fs_state_create(p1, u0, v0)
    b = fs.fs_state_create(p2, v0, u0)  # different initial data, overwritten by the load
    try:
        fs.fs_state_set_source(a, s)
        blob = fs.fs_state_save(a)
        fs.fs_state_load(b, blob)
        for args in ((1.0, 0.3), (0.7, 2.5)):
            ua, va, ub, vb = (torch.empty_like(u0) for _ in range(4))
            fs.fs_wave_advance(a, *args, ua, va)
            fs.fs_wave_advance(b, *args, ub, vb)
            torch.cuda.synchronize()
            assert torch.equal(ua, ub) and torch.equal(va, vb)
        ua, ub = torch.empty_like(u0), torch.empty_like(u0)
        fs.fs_diffusion_advance(a, 0.01, 0.4, ua)
        fs.fs_diffusion_advance(b, 0.01, 0.4, ub)
        torch.cuda.synchronize()
        assert torch.equal(ua, ub)
        # a checkpoint without a source detaches the loaded state's source
        fs.fs_state_set_source(a, None)
        fs.fs_state_load(b, fs.fs_state_save(a))
        fs.fs_diffusion_advance(a, 0.01, 0.4, ua)
        fs.fs_diffusion_advance(b, 0.01, 0.4, ub)
        torch.cuda.synchronize()
        assert torch.equal(ua, ub)
    finally:
        fs.fs_state_destroy(a)
        fs.fs_state_destroy(b)
        fs.fs_plan_destroy(p1)
        fs.fs_plan_destroy(p2)


def test_state_checkpoint_rejections(gpu_lib):
    u = torch.zeros((64, 64), device="cuda")
    p1 = fs.fs_plan_create(64, 64, 1.0, 1.0, 0)
    p2 = fs.fs_plan_create(64, 64, 2.0, 1.0, 0)
    a = fs.fs_state_create(p1, u, u)
    b = fs.fs_state_create(p2, u, u)
    c = fs.fs_state_create(p1, u)
    try:
        blob = fs.fs_state_save(a)
        with pytest.raises(fs.FsError):
            fs.fs_state_load(b, blob)  # other domain
        with pytest.raises(fs.FsError):
            fs.fs_state_load(c, blob)  # v0 presence differs
        with pytest.raises(fs.FsError):
            fs.fs_state_load(a, blob[:100])  # truncated
        with pytest.raises(fs.FsError):
            fs.fs_state_load(a, b"X" * len(blob))  # not a checkpoint
    finally:
        for st in (a, b, c):
            fs.fs_state_destroy(st)
        fs.fs_plan_destroy(p1)
        fs.fs_plan_destroy(p2)
