"""The allocation-free Poisson entry point (GPU).

fs_poisson_solve_static serves callers that may not allocate device memory
while they run; its scratch is a fixed array inside the library.  It must
give the same answer as the plan-based fs_poisson_solve and as the float64
oracle (within the FP32 bar used everywhere, rel-L2 <= 1e-5) on consecutive
calls that reuse the shared array, must not change the device's free memory once set up, and
must refuse grids beyond its fixed 1024 x 1024 limit.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""

import numpy as np
import pytest
import torch

from paper_2412_12308_gb300 import fsolve, workloads

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(torch.linalg.vector_norm((a - b).double()) / torch.linalg.vector_norm(b.double()))


@pytest.mark.parametrize("nx,ny,lx,ly", [(64, 64, 1.0, 1.0), (1024, 1024, 1.0, 1.0),
                                         (96, 40, 2.0, 0.7), (640, 512, 1.0, 1.3), (8, 1024, 1.0, 3.0)])
def test_static_matches_plan_entry_point(gpu_lib, nx, ny, lx, ly):
    rng = np.random.default_rng(nx + 3 * ny)
    kmax = max(1, min(16, nx // 2 - 1, ny // 2 - 1))
    f_host = workloads.mode_sum(workloads.draw_modes(rng, 8, kmax), nx, ny, lx, ly)
    f_host = f_host + 0.1 * rng.standard_normal((ny, nx))
    f = torch.tensor(f_host, dtype=torch.float32, device="cuda")
    plan = fsolve.fs_plan_create(nx, ny, lx, ly, fsolve.FS_F32)
    try:
        ref = torch.empty_like(f)
        fsolve.fs_poisson_solve(plan, f, ref)
        # two calls in a row: the second reuses the array the first left behind
        for _ in range(2):
            out = torch.full_like(f, float("nan"))
            fsolve.fs_poisson_solve_static(nx, ny, lx, ly, f, out)
            torch.cuda.synchronize()
            assert torch.isfinite(out).all()
            assert _rel(out, ref) <= 1e-5
    finally:
        fsolve.fs_plan_destroy(plan)


@pytest.mark.parametrize("nx,ny,lx,ly", [(64, 64, 1.0, 1.0), (96, 40, 2.0, 0.7), (1024, 256, 1.0, 1.0)])
def test_static_matches_oracle(gpu_lib, nx, ny, lx, ly):
    """The static entry point shares its pass kernels with fs_poisson_solve, so
    it is also checked against the float64 oracle (an independent direct DFT,
    Eq. SolutionPoisson) on the same float32-rounded input."""
    import oracle

    rng = np.random.default_rng(7 * nx + ny)
    f_host = rng.standard_normal((ny, nx)).astype(np.float32)
    want = oracle.poisson(f_host.astype(np.float64), lx, ly)
    f = torch.tensor(f_host, device="cuda")
    for _ in range(2):
        out = torch.full_like(f, float("nan"))
        fsolve.fs_poisson_solve_static(nx, ny, lx, ly, f, out)
        got = out.double().cpu().numpy()
        assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 1e-5


def test_static_allocates_nothing_per_call(gpu_lib):
    n = 512
    f = torch.randn(n, n, device="cuda")
    u = torch.empty_like(f)
    fsolve.fs_poisson_solve_static(n, n, 1.0, 1.0, f, u)  # first call: set-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        fsolve.fs_poisson_solve_static(n, n, 1.0, 1.0, f, u)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_rejects_grids_beyond_its_limit(gpu_lib):
    f = torch.zeros(8, 2048, device="cuda")
    with pytest.raises(fsolve.FsError) as ei:
        fsolve.fs_poisson_solve_static(2048, 8, 1.0, 1.0, f, f)
    assert ei.value.status == -2
    assert "1024" in str(ei.value)
    with pytest.raises(fsolve.FsError):
        fsolve.fs_poisson_solve_static(1024, 1024, 1.0, 1.0, None, f)
