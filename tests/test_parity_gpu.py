"""CUDA path vs the float64 oracle, element by element (GPU).

Bar: rel-L2 <= 1e-5 for the FP32 path, <= 1e-12 for the FP64 path, both
against the float64 oracle on the same seeded inputs.  Sizes span the
single-kernel path and the three-pass path, all three radix families
(2^k, 3*2^k, 5*2^k), non-square grids and domains, ragged row tiles and
column groups, and the size limits.
"""

import os

import numpy as np
import pytest
import torch

import oracle
from oracle import closed_forms as cf
from paper_2412_12308_gb300 import fsolve, workloads as wl

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-12}  # FS_F32, FS_F64
TDT = {0: torch.float32, 1: torch.float64}


def rel(a, b):
    return float(np.linalg.norm((np.asarray(a) - np.asarray(b)).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


def field(rng, nx, ny, kind="modes"):
    """Seeded input, rounded to float32 so both sides see identical values."""
    if kind == "noise":
        f = rng.standard_normal((ny, nx))
    else:
        kmax = max(1, min(16, nx // 2 - 1, ny // 2 - 1))
        f = wl.mode_sum(wl.draw_modes(rng, 8, kmax), nx, ny, 1.0, 1.0)
        f = f + 0.05 * rng.standard_normal((ny, nx))
    return f.astype(np.float32).astype(np.float64)


class Plan:
    def __init__(self, lib, nx, ny, lx, ly, dtype, small=None):
        self.lib = lib
        old = os.environ.get("FS_SMALL_MAX")
        if small is not None:
            os.environ["FS_SMALL_MAX"] = str(10**9 if small else 0)
        try:
            self.h = lib.fs_plan_create(nx, ny, lx, ly, dtype)
        finally:
            if small is not None:
                if old is None:
                    os.environ.pop("FS_SMALL_MAX", None)
                else:
                    os.environ["FS_SMALL_MAX"] = old
        self.info = lib.fs_plan_info(self.h)
        self.dtype = dtype

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.lib.fs_plan_destroy(self.h)

    def dev(self, arr):
        return torch.tensor(np.ascontiguousarray(arr), dtype=TDT[self.dtype], device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


SIZES = [(8, 8), (10, 10), (12, 12), (16, 16), (20, 20), (24, 24), (40, 40), (48, 48), (64, 64),
         (80, 80), (96, 96), (128, 128), (160, 160), (192, 192), (256, 256), (320, 320), (384, 384),
         (512, 512), (640, 640), (768, 768), (1024, 1024), (96, 40), (256, 80), (40, 512), (8, 96),
         (1280, 24), (160, 12)]


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("nx,ny", SIZES)
def test_poisson_vs_oracle(gpu_lib, nx, ny, dtype):
    rng = np.random.default_rng(nx * 7 + ny)
    f = field(rng, nx, ny)
    lx, ly = 1.0, 1.7
    want = oracle.poisson(f, lx, ly)
    for small in (True, False):
        with Plan(gpu_lib, nx, ny, lx, ly, dtype, small=small) as p:
            fd = p.dev(f)
            ud = torch.full_like(fd, float("nan"))
            gpu_lib.fs_poisson_solve(p.h, fd, ud)
            got = host(ud)
            assert np.all(np.isfinite(got))
            err = rel(got, want)
            assert err <= TOL[dtype], (nx, ny, dtype, p.info["path"], err)


def test_poisson_64_fp64_closed_form(gpu_lib):
    """64 x 64 FP64 Poisson with an 8-mode source: exact solution known."""
    f, modes, (lx, ly) = wl.poisson_modes_64()
    with Plan(gpu_lib, 64, 64, lx, ly, 1) as p:
        fd = p.dev(f)
        ud = torch.empty_like(fd)
        gpu_lib.fs_poisson_solve(p.h, fd, ud)
        got = host(ud)
    assert rel(got, cf.poisson_modes(modes, 64, 64, lx, ly)) <= 1e-12
    assert rel(got, oracle.poisson(f, lx, ly)) <= 1e-12


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("nx,ny", [(64, 64), (96, 80), (256, 256), (320, 192), (1024, 512)])
def test_diffusion_solve_and_advance(gpu_lib, nx, ny, dtype):
    rng = np.random.default_rng(11 + nx)
    u0 = field(rng, nx, ny)
    lx, ly, D = 2 * np.pi, 2 * np.pi, 0.1
    F = oracle.state_spectrum(u0)
    for small in (True, False):
        with Plan(gpu_lib, nx, ny, lx, ly, dtype, small=small) as p:
            ud0 = p.dev(u0)
            out = torch.empty_like(ud0)
            st = gpu_lib.fs_state_create(p.h, ud0)
            try:
                for t in (0.0, 0.013, 0.5, 1.0, 7.0):
                    want = np.real(oracle.idft2(oracle.diffusion_spectrum(F, D, t, lx, ly)))
                    gpu_lib.fs_diffusion_advance(st, D, t, out)
                    assert rel(host(out), want) <= TOL[dtype], ("advance", t, small)
                    gpu_lib.fs_diffusion_solve(p.h, ud0, D, t, out)
                    assert rel(host(out), want) <= TOL[dtype], ("solve", t, small)
            finally:
                gpu_lib.fs_state_destroy(st)


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("nx,ny", [(64, 64), (80, 96), (256, 256), (384, 320), (512, 1024)])
def test_wave_solve_and_advance(gpu_lib, nx, ny, dtype):
    rng = np.random.default_rng(23 + ny)
    u0 = field(rng, nx, ny, "noise")
    v0 = field(rng, nx, ny)
    lx, ly, c = 1.0, 1.3, 1.2
    F, G = oracle.state_spectrum(u0), oracle.state_spectrum(v0)
    for small in (True, False):
        with Plan(gpu_lib, nx, ny, lx, ly, dtype, small=small) as p:
            ud0, vd0 = p.dev(u0), p.dev(v0)
            uo, vo = torch.empty_like(ud0), torch.empty_like(ud0)
            s1 = gpu_lib.fs_state_create(p.h, ud0)
            s2 = gpu_lib.fs_state_create(p.h, ud0, vd0)
            try:
                for t in (0.0, 0.21, 1.0, -0.4):
                    U0, V0 = oracle.wave_spectrum(F, None, c, t, lx, ly)
                    U1, V1 = oracle.wave_spectrum(F, G, c, t, lx, ly)
                    wu0, wv0 = np.real(oracle.idft2(U0)), np.real(oracle.idft2(V0))
                    wu1, wv1 = np.real(oracle.idft2(U1)), np.real(oracle.idft2(V1))
                    gpu_lib.fs_wave_advance(s1, c, t, uo, vo)
                    assert rel(host(uo), wu0) <= TOL[dtype], ("u, v0=0", t, small)
                    if t != 0.0:
                        assert rel(host(vo), wv0) <= TOL[dtype], ("v, v0=0", t, small)
                    gpu_lib.fs_wave_advance(s2, c, t, uo, vo)
                    assert rel(host(uo), wu1) <= TOL[dtype], ("u", t, small)
                    assert rel(host(vo), wv1) <= TOL[dtype], ("v", t, small)
                    gpu_lib.fs_wave_advance(s2, c, t, uo, None)
                    assert rel(host(uo), wu1) <= TOL[dtype], ("u only", t, small)
                    gpu_lib.fs_wave_solve(p.h, ud0, vd0, c, t, uo)
                    assert rel(host(uo), wu1) <= TOL[dtype], ("solve", t, small)
                    gpu_lib.fs_wave_solve(p.h, ud0, None, c, t, uo)
                    assert rel(host(uo), wu0) <= TOL[dtype], ("solve v0=0", t, small)
            finally:
                gpu_lib.fs_state_destroy(s1)
                gpu_lib.fs_state_destroy(s2)


def test_in_place_and_degenerate_inputs(gpu_lib):
    for dtype in (0, 1):
        for nx, ny in ((64, 64), (512, 256)):
            with Plan(gpu_lib, nx, ny, 1.0, 1.0, dtype) as p:
                rng = np.random.default_rng(3)
                f = field(rng, nx, ny)
                want = oracle.poisson(f, 1.0, 1.0)
                fd = p.dev(f)
                gpu_lib.fs_poisson_solve(p.h, fd, fd)  # u aliases f
                assert rel(host(fd), want) <= TOL[dtype]
                z = torch.zeros_like(fd)
                out = torch.full_like(fd, 5.0)
                gpu_lib.fs_poisson_solve(p.h, z, out)
                assert float(host(out).__abs__().max()) == 0.0
                const = torch.full_like(fd, 3.5)
                gpu_lib.fs_poisson_solve(p.h, const, out)
                assert float(np.abs(host(out)).max()) <= (1e-5 if dtype == 0 else 1e-12)
                gpu_lib.fs_diffusion_solve(p.h, const, 0.3, 2.0, out)
                assert np.allclose(host(out), 3.5, rtol=TOL[dtype] * 10, atol=0)


def test_rejections_on_device(gpu_lib):
    from paper_2412_12308_gb300 import fsolve

    with Plan(gpu_lib, 64, 64, 1.0, 1.0, 0) as p:
        x = p.dev(np.zeros((64, 64)))
        with pytest.raises(fsolve.FsError):
            gpu_lib.fs_diffusion_solve(p.h, x, -1.0, 1.0, x)
        with pytest.raises(fsolve.FsError):
            gpu_lib.fs_wave_solve(p.h, x, None, 0.0, 1.0, x)
        with pytest.raises(fsolve.FsError):
            gpu_lib.fs_poisson_solve(p.h, None, x)
        # FP32 wave phases beyond 2^20 (c |t| |omega|_max) are refused: the
        # two-float phase reduction would lose accuracy past that range
        with pytest.raises(fsolve.FsError) as ei:
            gpu_lib.fs_wave_solve(p.h, x, None, 1.0, 1.0e5, x)
        assert "phase" in str(ei.value)
        gpu_lib.fs_wave_solve(p.h, x, None, 1.0, 1000.0, x)  # 1000 * pi * 64 * sqrt(2) < 2^20
    with Plan(gpu_lib, 64, 64, 1.0, 1.0, 1) as p:  # FP64 plans take any phase
        x = p.dev(np.zeros((64, 64)))
        gpu_lib.fs_wave_solve(p.h, x, None, 1.0, 1.0e5, x)


@pytest.mark.parametrize("nx,ny", [(2048, 2048), (4096, 4096), (8192, 8192), (1536, 1536), (2560, 2560),
                                   (3072, 1280), (6144, 640), (5120, 384), (1280, 3072)])
def test_large_grids_sampled(gpu_lib, nx, ny):
    """Large FP32 grids (powers of two, 3 x 2^k and 5 x 2^k lengths, square
    and rectangular): mode-sum sources have exact closed forms on every grid
    point (O(modes * N^2)), so the whole output is checked, through the
    per-call entry points and through one batch."""
    rng = np.random.default_rng(nx + 7 * ny)
    modes = wl.draw_modes(rng, 8, 40)
    f = wl.mode_sum(modes, nx, ny, 1.0, 1.0)
    with Plan(gpu_lib, nx, ny, 1.0, 1.0, 0) as p:
        fd = p.dev(f)
        ud = torch.empty_like(fd)
        gpu_lib.fs_poisson_solve(p.h, fd, ud)
        u_p = cf.poisson_modes(modes, nx, ny, 1.0, 1.0)
        assert rel(host(ud), u_p) <= 1e-5
        # D t chosen so the output keeps most of the input energy (a heavily
        # decayed output is compared normwise in test_diffusion_heavy_decay)
        gpu_lib.fs_diffusion_solve(p.h, fd, 1e-5, 0.5, ud)
        u_d = cf.diffusion_modes(modes, 1e-5, 0.5, nx, ny, 1.0, 1.0)
        assert rel(host(ud), u_d) <= 1e-5
        st = gpu_lib.fs_state_create(p.h, fd)
        try:
            for t in (0.3, 1.0, 1.9):
                gpu_lib.fs_wave_advance(st, 1.0, t, ud)
                assert rel(host(ud), cf.wave_modes(modes, 1.0, t, nx, ny, 1.0, 1.0)) <= 1e-5
            outs = [torch.empty_like(fd) for _ in range(3)]
            reqs = [fsolve.fs_request(fsolve.FS_OP_POISSON, plan=p.h, in_u=fd, out_u=outs[0]),
                    fsolve.fs_request(fsolve.FS_OP_DIFFUSION, plan=p.h, in_u=fd, out_u=outs[1], D=1e-5, t=0.5),
                    fsolve.fs_request(fsolve.FS_OP_DIFFUSION_ADVANCE, state=st, out_u=outs[2], D=1e-5, t=0.5)]
            fsolve.fs_batch_wait(fsolve.fs_batch_submit(reqs), 60_000_000)
            assert rel(host(outs[0]), u_p) <= 1e-5
            assert rel(host(outs[1]), u_d) <= 1e-5
            assert rel(host(outs[2]), u_d) <= 1e-5
        finally:
            gpu_lib.fs_state_destroy(st)


def test_diffusion_heavy_decay_normwise(gpu_lib):
    """When diffusion shrinks the field by orders of magnitude, FP32 rounding
    at the input's scale dominates the tiny output, so the error is bounded
    normwise: ||u - u_ref|| <= 1e-5 * max(||u_ref||, ||f||) (the largest
    diffusion multiplier is 1).  The plain rel-L2 bound holds whenever the
    output keeps at least that fraction of the input norm."""
    n = 256
    rng = np.random.default_rng(5)
    f = field(rng, n, n)
    for D, t in ((0.5, 0.8), (1.0, 1.0), (0.01, 0.3)):
        want = oracle.diffusion(f, D, t, 1.0, 1.0)
        with Plan(gpu_lib, n, n, 1.0, 1.0, 0) as p:
            fd = p.dev(f)
            ud = torch.empty_like(fd)
            gpu_lib.fs_diffusion_solve(p.h, fd, D, t, ud)
            got = host(ud)
        den = max(np.linalg.norm(want), np.linalg.norm(f))
        assert np.linalg.norm(got - want) / den <= 1e-5, (D, t)


@pytest.mark.parametrize("nx,ny", [(2048, 2048), (4096, 4096), (8192, 8192), (8192, 640)])
def test_large_grids_fp64_closed_forms(gpu_lib, nx, ny):
    """The FP64 path on long axes (register tiles of 8 up to length 4096 and 16
    at 8192), square and rectangular: every operator, one-shot solves and
    advances from a kept spectrum, against the mode-sum closed forms on the
    whole grid at the FP64 bar rel-L2 <= 1e-12 (Eq. SolutionPoisson,
    Eq. solCalorFourier, Eq. OmegaNonZero and its time derivative)."""
    rng = np.random.default_rng(3 * nx + ny)
    modes = wl.draw_modes(rng, 8, 40)
    f = wl.mode_sum(modes, nx, ny, 1.0, 1.0)
    tol = TOL[1]
    with Plan(gpu_lib, nx, ny, 1.0, 1.0, 1) as p:
        fd = p.dev(f)
        ud = torch.full_like(fd, float("nan"))
        vd = torch.full_like(fd, float("nan"))
        gpu_lib.fs_poisson_solve(p.h, fd, ud)
        assert rel(host(ud), cf.poisson_modes(modes, nx, ny, 1.0, 1.0)) <= tol
        D, t = 1e-5, 0.5
        u_d = cf.diffusion_modes(modes, D, t, nx, ny, 1.0, 1.0)
        gpu_lib.fs_diffusion_solve(p.h, fd, D, t, ud)
        assert rel(host(ud), u_d) <= tol
        st = gpu_lib.fs_state_create(p.h, fd)
        try:
            gpu_lib.fs_diffusion_advance(st, D, t, ud)
            assert rel(host(ud), u_d) <= tol
            del u_d
            u_w, v_w = cf.wave_modes(modes, 1.3, 0.3, nx, ny, 1.0, 1.0, want_v=True)
            gpu_lib.fs_wave_advance(st, 1.3, 0.3, ud, vd)
            assert rel(host(ud), u_w) <= tol
            assert rel(host(vd), v_w) <= tol
            del u_w, v_w
            u_w = cf.wave_modes(modes, 1.0, 1.9, nx, ny, 1.0, 1.0)
            gpu_lib.fs_wave_advance(st, 1.0, 1.9, ud)
            assert rel(host(ud), u_w) <= tol
            gpu_lib.fs_wave_solve(p.h, fd, None, 1.0, 1.9, ud)
            assert rel(host(ud), u_w) <= tol
        finally:
            gpu_lib.fs_state_destroy(st)
