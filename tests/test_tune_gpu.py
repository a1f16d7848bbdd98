"""Autotuner (GPU): fs_tune times candidate register tiles and tile shapes of
a grid's passes and caches the fastest; later plans of that grid use it; a
tuned plan still matches the closed form; a stale cache entry falls back to
the defaults.  The cache is cleared afterwards so other tests see defaults."""

import json

import numpy as np
import pytest
import torch

from oracle import closed_forms as cf
from paper_2412_12308_gb300 import fsolve as fs
from paper_2412_12308_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture
def clean_cache(gpu_lib):
    fs.fs_tune_cache_clear()
    yield
    fs.fs_tune_cache_clear()


@pytest.mark.parametrize("n,dtype", [(4096, 0), (1536, 0), (640, 1)])
def test_tune_and_use(clean_cache, n, dtype):
    r = fs.fs_tune(n, n, 1.0, 1.0, dtype, reps=5)
    assert r["candidates"] > 1 and 0 < r["us_tuned"] <= r["us_default"] * 1.0001
    plan = fs.fs_plan_create(n, n, 1.0, 1.0, dtype)
    try:
        assert fs.fs_plan_tiles(plan) == (r["e_row"], r["e_col"], r["rows"], r["cols"])
        rng = np.random.default_rng(n)
        modes = wl.draw_modes(rng, 8, 40)
        f = wl.mode_sum(modes, n, n, 1.0, 1.0)
        tdt = torch.float32 if dtype == 0 else torch.float64
        fd = torch.tensor(f, dtype=tdt, device="cuda")
        ud = torch.empty_like(fd)
        fs.fs_poisson_solve(plan, fd, ud)
        torch.cuda.synchronize()
        want = cf.poisson_modes(modes, n, n, 1.0, 1.0)
        got = ud.double().cpu().numpy()
        assert np.linalg.norm(got - want) / np.linalg.norm(want) <= (1e-5 if dtype == 0 else 1e-12)
    finally:
        fs.fs_plan_destroy(plan)


def test_tune_cache_file_and_stale_entry(clean_cache, tmp_path):
    n = 1024
    default = fs.fs_plan_create(n, n, 1.0, 1.0, 0)
    d_tiles = fs.fs_plan_tiles(default)
    fs.fs_plan_destroy(default)
    r = fs.fs_tune(n, n, 1.0, 1.0, 0, reps=5)
    path = tmp_path / "tune.jsonl"
    assert fs.fs_tune_cache_save(str(path)) == 1
    fs.fs_tune_cache_clear()
    assert fs.fs_tune_cache_load(str(path)) == 1
    p = fs.fs_plan_create(n, n, 1.0, 1.0, 0)
    assert fs.fs_plan_tiles(p) == (r["e_row"], r["e_col"], r["rows"], r["cols"])
    fs.fs_plan_destroy(p)
    # an entry that no longer fits (register tile 7 does not exist): defaults
    gpu = torch.cuda.get_device_name()
    path.write_text(json.dumps({"gpu": gpu, "nx": n, "ny": n, "dtype": 0, "e_row": 7, "e_col": 16,
                                "rows": 4, "cols": 4, "us": 1.0}) + "\n")
    fs.fs_tune_cache_clear()
    assert fs.fs_tune_cache_load(str(path)) == 1
    p = fs.fs_plan_create(n, n, 1.0, 1.0, 0)
    assert fs.fs_plan_tiles(p) == d_tiles
    fs.fs_plan_destroy(p)


@pytest.mark.parametrize("n", [384, 640])
def test_tune_batch_and_use(clean_cache, n):
    """Batch-mode tuning picks register tiles for the grid inside a batch; a
    batch using them still matches the closed form for every problem."""
    r = fs.fs_tune_batch(n, n, 1.0, 1.0, 0, nprob=4, reps=2)
    assert r["candidates"] >= 1 and 0 < r["us_tuned"] <= r["us_default"] * 1.0001
    plan = fs.fs_plan_create(n, n, 1.0, 1.0, 0)
    try:
        rng = np.random.default_rng(n + 3)
        fields, outs, reqs, wants = [], [], [], []
        for _ in range(6):
            modes = wl.draw_modes(rng, 8, 30)
            f = torch.tensor(wl.mode_sum(modes, n, n, 1.0, 1.0), dtype=torch.float32, device="cuda")
            o = torch.empty_like(f)
            fields.append(f)
            outs.append(o)
            wants.append(cf.poisson_modes(modes, n, n, 1.0, 1.0))
            reqs.append(fs.fs_request(fs.FS_OP_POISSON, plan=plan, in_u=f, out_u=o))
        fs.fs_batch_wait(fs.fs_batch_submit(reqs), 30_000_000)
        torch.cuda.synchronize()
        for o, want in zip(outs, wants):
            got = o.double().cpu().numpy()
            assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 1e-5
    finally:
        fs.fs_plan_destroy(plan)

