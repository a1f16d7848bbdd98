"""Guard words around every output (GPU).

compute-sanitizer is not available on this machine, so out-of-bounds stores are
checked directly: each output field is the middle of a larger buffer whose
margins hold a canary pattern, and after every entry point writes the field
the margins must be unchanged (and the field finite).  Sizes cover ragged row
tiles and column groups, the three radix families, the single-CTA path, the
three-pass path, batches, complex fields, kept states with sources and the
RK4 integrator.
"""

import numpy as np
import pytest
import torch

from paper_2412_12308_gb300 import fsolve as fs
from paper_2412_12308_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

MARGIN = 4096  # elements on each side
CANARY = -1.2345678e30


class Guarded:
    """A [ny][nx] field in the middle of a buffer with canary margins."""

    def __init__(self, nx, ny, dtype=torch.float32, complex_=False):
        n = nx * ny
        self.shape = (ny, nx)
        self.buf = torch.full((n + 2 * MARGIN,), CANARY, dtype=dtype, device="cuda")
        if complex_:
            self.buf = torch.complex(self.buf, self.buf)
        self.field = self.buf[MARGIN:MARGIN + n].view(ny, nx)

    def check(self, what):
        torch.cuda.synchronize()
        lo, hi = self.buf[:MARGIN], self.buf[-MARGIN:]
        want = torch.full_like(lo, CANARY) if not torch.is_complex(lo) else torch.complex(
            torch.full_like(lo.real, CANARY), torch.full_like(lo.real, CANARY))
        assert torch.equal(lo, want), f"{what}: store below the field"
        assert torch.equal(hi, want), f"{what}: store above the field"
        assert bool(torch.isfinite(self.field).all()), f"{what}: non-finite output"


SIZES = [(8, 8), (24, 40), (96, 80), (160, 12), (320, 192), (1280, 24), (1024, 1024), (2048, 256)]


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("nx,ny", SIZES)
def test_guard_solves_and_advances(gpu_lib, nx, ny, dtype):
    tdt = torch.float32 if dtype == 0 else torch.float64
    rng = np.random.default_rng(nx * 7 + ny)
    f = torch.tensor(rng.standard_normal((ny, nx)), dtype=tdt, device="cuda")
    g = torch.tensor(rng.standard_normal((ny, nx)), dtype=tdt, device="cuda")
    plan = fs.fs_plan_create(nx, ny, 1.0, 1.3, dtype)
    st = fs.fs_state_create(plan, f, g)
    try:
        out, vout = Guarded(nx, ny, tdt), Guarded(nx, ny, tdt)
        fs.fs_poisson_solve(plan, f, out.field)
        out.check("poisson")
        fs.fs_diffusion_solve(plan, f, 0.01, 0.1, out.field)
        out.check("diffusion")
        fs.fs_wave_solve(plan, f, g, 1.0, 0.3, out.field)
        out.check("wave v0")
        fs.fs_wave_advance(st, 1.0, 0.7, out.field, vout.field)
        out.check("wave advance u")
        vout.check("wave advance v")
        fs.fs_state_set_source(st, g)
        fs.fs_diffusion_advance(st, 0.01, 0.2, out.field)
        out.check("diffusion advance with source")
        fs.fs_wave_advance(st, 1.0, 0.2, out.field, vout.field)
        out.check("wave advance with source u")
        vout.check("wave advance with source v")
        # batch: the same outputs through the persistent launch
        reqs = [fs.fs_request(fs.FS_OP_POISSON, plan=plan, in_u=f, out_u=out.field),
                fs.fs_request(fs.FS_OP_WAVE_ADVANCE, state=st, out_u=vout.field, c=1.0, t=0.1)]
        fs.fs_batch_wait(fs.fs_batch_submit(reqs), 30_000_000)
        out.check("batch poisson")
        vout.check("batch wave advance")
    finally:
        fs.fs_state_destroy(st)
        fs.fs_plan_destroy(plan)


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("nx,ny", [(16, 16), (96, 80), (40, 512), (1024, 256)])
def test_guard_complex(gpu_lib, nx, ny, dtype):
    cdt = torch.complex64 if dtype == 0 else torch.complex128
    rdt = torch.float32 if dtype == 0 else torch.float64
    rng = np.random.default_rng(nx + 5 * ny)
    z = torch.tensor(rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx)), dtype=cdt,
                     device="cuda")
    plan = fs.fs_plan_create(nx, ny, 1.0, 1.0, dtype)
    try:
        out = Guarded(nx, ny, rdt, complex_=True)
        fs.fs_poisson_solve_c(plan, z, out.field)
        out.check("complex poisson")
        fs.fs_wave_solve_c(plan, z, z, 1.0, 0.4, out.field)
        out.check("complex wave v0")
        fs.fs_diffusion_solve_c(plan, z, 0.01, 0.2, out.field)
        out.check("complex diffusion")
    finally:
        fs.fs_plan_destroy(plan)


@pytest.mark.parametrize("n", [64, 96, 512])
def test_guard_rk4(gpu_lib, n):
    plan = fs.fs_plan_create(n, n, 4.0, 4.0, 0)
    rk = fs.fs_rk4_create(plan, 1.0, wl.OrbitSource())
    try:
        fs.fs_rk4_step(rk, 0.25 * 4.0 / n, 130)  # two chunks
        out, vout = Guarded(n, n), Guarded(n, n)
        fs.fs_rk4_output(rk, out.field, vout.field)
        out.check("rk4 u")
        vout.check("rk4 v")
    finally:
        fs.fs_rk4_destroy(rk)
        fs.fs_plan_destroy(plan)
