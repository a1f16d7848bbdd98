"""Complex-field solves vs the float64 oracle (GPU).

Sec. II.B allows complex samples p_jk: fs_*_solve_c take interleaved complex
fields and use the full spectrum.  Compared element by element with
oracle.poisson_complex / diffusion_complex / wave_complex on the same seeded
inputs (complex64 inputs rounded once, promoted for the oracle).  Bar:
rel-L2 <= 1e-5 (FP32), <= 1e-12 (FP64).  Large grids use complex plane-wave
sums, whose solutions are known on every grid point.
"""

import math

import numpy as np
import pytest
import torch

import oracle
from tests.test_parity_gpu import TOL, Plan, field, rel

pytestmark = pytest.mark.gpu

CDT = {0: torch.complex64, 1: torch.complex128}


def cfield(rng, nx, ny, dtype):
    z = field(rng, nx, ny) + 1j * field(rng, nx, ny, "noise")
    return z.astype(np.complex64).astype(np.complex128) if dtype == 0 else z


def cdev(z, dtype):
    return torch.tensor(np.ascontiguousarray(z), dtype=CDT[dtype], device="cuda")


def chost(t):
    torch.cuda.synchronize()
    return t.to(torch.complex128).cpu().numpy()


SIZES = [(16, 16), (64, 64), (96, 80), (40, 512), (256, 256), (320, 192), (1024, 512)]


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("nx,ny", SIZES)
def test_complex_solves_vs_oracle(gpu_lib, nx, ny, dtype):
    fs = gpu_lib
    rng = np.random.default_rng(500 + nx + 3 * ny)
    f, g = cfield(rng, nx, ny, dtype), cfield(rng, nx, ny, dtype)
    lx, ly = 2 * np.pi, 1.7 * np.pi
    with Plan(fs, nx, ny, lx, ly, dtype) as p:
        fd, gd = cdev(f, dtype), cdev(g, dtype)
        out = torch.empty_like(fd)
        fs.fs_poisson_solve_c(p.h, fd, out)
        assert rel(chost(out), oracle.poisson_complex(f, lx, ly)) <= TOL[dtype]
        for D, t in ((0.05, 0.3), (0.0, 1.0)):
            fs.fs_diffusion_solve_c(p.h, fd, D, t, out)
            assert rel(chost(out), oracle.diffusion_complex(f, D, t, lx, ly)) <= TOL[dtype], (D, t)
        for t in (0.0, 0.41, -1.3):
            fs.fs_wave_solve_c(p.h, fd, None, 1.2, t, out)
            assert rel(chost(out), oracle.wave_complex(f, None, 1.2, t, lx, ly)) <= TOL[dtype], t
            fs.fs_wave_solve_c(p.h, fd, gd, 1.2, t, out)
            assert rel(chost(out), oracle.wave_complex(f, g, 1.2, t, lx, ly)) <= TOL[dtype], t
        # in place
        fs.fs_poisson_solve_c(p.h, fd, fd)
        assert rel(chost(fd), oracle.poisson_complex(f, lx, ly)) <= TOL[dtype]


def test_complex_real_input_matches_real_solve(gpu_lib):
    """A real field through the complex path equals the real (R2C) path."""
    fs = gpu_lib
    n = 256
    rng = np.random.default_rng(9)
    f = field(rng, n, n)
    with Plan(fs, n, n, 1.0, 1.0, 1) as p:
        fr = torch.tensor(f, dtype=torch.float64, device="cuda")
        ur = torch.empty_like(fr)
        fs.fs_poisson_solve(p.h, fr, ur)
        fc = cdev(f + 0j, 1)
        uc = torch.empty_like(fc)
        fs.fs_poisson_solve_c(p.h, fc, uc)
        got = chost(uc)
    assert rel(got.real, ur.cpu().numpy()) <= 1e-12
    assert np.abs(got.imag).max() <= 1e-12 * np.abs(got.real).max()


@pytest.mark.parametrize("n", [2048, 4096])
def test_complex_large_plane_waves(gpu_lib, n):
    """FP32, large grids: a sum of complex plane waves exp(i(wx x + wy y)) with
    signed wavenumbers has closed-form solutions on every grid point."""
    fs = gpu_lib
    rng = np.random.default_rng(n + 1)
    lx = ly = 1.0
    x = np.arange(n) / n
    modes = [(int(rng.integers(-60, 61)), int(rng.integers(-60, 61)), complex(rng.standard_normal(), rng.standard_normal()))
             for _ in range(6)]
    modes = [(kx, ky, a) for kx, ky, a in modes if (kx, ky) != (0, 0)]

    def make(fn):
        z = np.zeros((n, n), np.complex128)
        for kx, ky, a in modes:
            w2 = (2 * math.pi) ** 2 * (kx * kx + ky * ky)
            z += a * fn(w2) * np.exp(2j * math.pi * (ky * x[:, None] + kx * x[None, :]))
        return z
    f = make(lambda w2: 1.0)
    with Plan(fs, n, n, lx, ly, 0) as p:
        fd = cdev(f, 0)
        out = torch.empty_like(fd)
        fs.fs_poisson_solve_c(p.h, fd, out)
        assert rel(chost(out), make(lambda w2: -1.0 / w2)) <= 1e-5
        fs.fs_diffusion_solve_c(p.h, fd, 1e-5, 0.5, out)
        assert rel(chost(out), make(lambda w2: math.exp(-1e-5 * w2 * 0.5))) <= 1e-5
        fs.fs_wave_solve_c(p.h, fd, None, 1.0, 0.37, out)
        assert rel(chost(out), make(lambda w2: math.cos(math.sqrt(w2) * 0.37))) <= 1e-5


def test_complex_rejections(gpu_lib):
    fs = gpu_lib
    with Plan(fs, 64, 64, 1.0, 1.0, 0) as p:
        z = torch.zeros((64, 64), dtype=torch.complex64, device="cuda")
        with pytest.raises(fs.FsError):
            fs.fs_diffusion_solve_c(p.h, z, -1.0, 0.1, z)
        with pytest.raises(fs.FsError):
            fs.fs_wave_solve_c(p.h, z, None, 0.0, 0.1, z)
        with pytest.raises(fs.FsError):
            fs.fs_poisson_solve_c(p.h, None, z)


def test_complex_unsupported_length_reports_size(gpu_lib):
    """FP64, nx = 1280: no length-1280 plan; the plan works for real fields and
    complex calls fail with FS_ERR_SIZE (no device work)."""
    fs = gpu_lib
    with Plan(fs, 1280, 24, 1.0, 1.0, 1) as p:
        z = torch.zeros((24, 1280), dtype=torch.complex128, device="cuda")
        with pytest.raises(fs.FsError) as ei:
            fs.fs_poisson_solve_c(p.h, z, z)
        assert ei.value.status == -2

