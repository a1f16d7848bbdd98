"""RK4 wave integration with an orbiting source vs the float64 oracle (GPU).

Sec. III.C, example with source: u_tt = c^2 lap u + s(t, x, y) with the
orbiting Gaussian, integrated per mode with classical RK4 on
Eq. SystemOfODEsForWaveEquation.  The CUDA path (fs_rk4_*) is compared with
oracle.wave_rk4_spectrum on the same source definition (workloads.OrbitSource)
and the same step times.  Bar: rel-L2 <= 1e-5 (FP32), <= 1e-12 (FP64).
"""

import math

import numpy as np
import pytest
import torch

import oracle
from paper_2412_12308_gb300 import workloads as wl
from tests.test_parity_gpu import TOL, Plan, field, host, rel

pytestmark = pytest.mark.gpu

L = 4.0  # the paper's [-2, 2]^2


def _oracle(nx, ny, src, c, dt, nsteps, u0=None, v0=None, lx=L, ly=L):
    F = np.zeros((ny, nx), complex) if u0 is None else oracle.state_spectrum(u0)
    G = None if v0 is None else oracle.state_spectrum(v0)
    U, V = oracle.wave_rk4_spectrum(F, G, lambda t: src.field(t, nx, ny, lx, ly), c, 0.0, dt, nsteps, lx, ly)
    return np.real(oracle.idft2(U)), np.real(oracle.idft2(V))


def _run(fs, p, c, src, dt, steps):
    """A new integrator from rest, advanced by successive fs_rk4_step calls."""
    rk = fs.fs_rk4_create(p.h, c, src)
    try:
        for n in steps:
            fs.fs_rk4_step(rk, dt, n)
    except Exception:
        fs.fs_rk4_destroy(rk)
        raise
    return rk


def _outputs(fs, rk, ny, nx, dtype):
    tdt = torch.float32 if dtype == 0 else torch.float64
    u = torch.empty((ny, nx), dtype=tdt, device="cuda")
    v = torch.empty_like(u)
    fs.fs_rk4_output(rk, u, v)
    return host(u), host(v)


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("nx,ny", [(64, 64), (96, 80), (128, 128)])
def test_rk4_orbit_vs_oracle(gpu_lib, nx, ny, dtype):
    """The paper's source and dt = h/4 from rest, 40 steps."""
    fs = gpu_lib
    src = wl.OrbitSource()
    dt = 0.25 * L / max(nx, ny)
    wu, wv = _oracle(nx, ny, src, 1.0, dt, 40)
    with Plan(fs, nx, ny, L, L, dtype) as p:
        rk = _run(fs, p, 1.0, src, dt, [40])
        try:
            u, v = _outputs(fs, rk, ny, nx, dtype)
            assert abs(fs.fs_rk4_time(rk) - 40 * dt) <= 1e-12
        finally:
            fs.fs_rk4_destroy(rk)
    assert rel(u, wu) <= TOL[dtype]
    assert rel(v, wv) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [0, 1])
def test_rk4_initial_data_and_split_calls(gpu_lib, dtype):
    """Non-zero u0, v0, wave speed c = 0.7, a non-square domain, and 13 + 1 + 26
    steps in three calls (three captured graphs) against 40 oracle steps."""
    fs = gpu_lib
    nx, ny, lx, ly = 80, 64, 4.0, 3.2
    rng = np.random.default_rng(77)
    u0, v0 = field(rng, nx, ny), field(rng, nx, ny)
    src = wl.OrbitSource(A=2.0, sigma=0.25, radius=0.6, Omega=3.0, gamma=7.0, x_min=-2.0, y_min=-1.6)
    dt, c = 0.01, 0.7
    wu, wv = _oracle(nx, ny, src, c, dt, 40, u0, v0, lx, ly)
    with Plan(fs, nx, ny, lx, ly, dtype) as p:
        rk = fs.fs_rk4_create(p.h, c, src, p.dev(u0), p.dev(v0))
        try:
            for n in (13, 1, 26):
                fs.fs_rk4_step(rk, dt, n)
            u, v = _outputs(fs, rk, ny, nx, dtype)
        finally:
            fs.fs_rk4_destroy(rk)
    assert rel(u, wu) <= TOL[dtype]
    assert rel(v, wv) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [0, 1])
def test_rk4_zero_steps_is_identity(gpu_lib, dtype):
    fs = gpu_lib
    n = 64
    rng = np.random.default_rng(3)
    u0, v0 = field(rng, n, n), field(rng, n, n)
    with Plan(fs, n, n, L, L, dtype) as p:
        rk = fs.fs_rk4_create(p.h, 1.0, wl.OrbitSource(), p.dev(u0), p.dev(v0))
        try:
            fs.fs_rk4_step(rk, 0.01, 0)
            u, v = _outputs(fs, rk, n, n, dtype)
        finally:
            fs.fs_rk4_destroy(rk)
    assert rel(u, u0) <= TOL[dtype]
    assert rel(v, v0) <= TOL[dtype]


def test_rk4_mean_self_convergence_fp64(gpu_lib):
    """FP64 on the GPU: the mean of u at t = 1 for dt = h/4 with h = 4/64, 4/128,
    4/256 (N = 64 grid) self-converges with factor ~16 (the paper's claim)
    and matches the exact mean A pi sigma^2 (1 - cos(gamma t)) / (L^2 gamma^2)
    within the RK4 error estimate."""
    from tests.golden import load_facts

    fs = gpu_lib
    src = wl.OrbitSource()
    means = []
    with Plan(fs, 64, 64, L, L, 1) as p:
        for N in (64, 128, 256):
            dt = 0.25 * L / N
            rk = fs.fs_rk4_create(p.h, 1.0, src)
            try:
                fs.fs_rk4_step(rk, dt, N)  # dt = 1/N: N steps reach t = 1
                means.append(fs.fs_rk4_mean(rk))
            finally:
                fs.fs_rk4_destroy(rk)
    u1, u2, u3 = means
    factor = (u2 - u1) / (u3 - u2)
    assert abs(factor - load_facts()["rk4_self_convergence_factor"]) <= 0.1 * 16
    exact = src.A * math.pi * src.sigma**2 * (1 - math.cos(src.gamma)) / (L**2 * src.gamma**2)
    assert abs(u3 - exact) <= 2 * abs(u3 - u2) / 15 + 1e-15


@pytest.mark.parametrize("n", [1024, 2048])
def test_rk4_large_grid_sublattice(gpu_lib, n):
    """FP32 on large grids: with sigma = 0.3 the source is band-limited to
    ~e^-56 at the 64 x 64 lattice's Nyquist, so the fine-grid RK4 solution on
    every (n/64)-th point equals the oracle's RK4 solution on the 64 x 64 grid
    with the same dt."""
    fs = gpu_lib
    src = wl.OrbitSource(sigma=0.3)
    dt, steps = 0.25 * L / n, 50
    wu, wv = _oracle(64, 64, src, 1.0, dt, steps)
    step = n // 64
    with Plan(fs, n, n, L, L, 0) as p:
        rk = fs.fs_rk4_create(p.h, 1.0, src)
        try:
            fs.fs_rk4_step(rk, dt, steps)
            u, v = _outputs(fs, rk, n, n, 0)
        finally:
            fs.fs_rk4_destroy(rk)
    assert rel(u[::step, ::step], wu) <= 1e-5
    assert rel(v[::step, ::step], wv) <= 1e-5


def test_rk4_rejections(gpu_lib):
    fs = gpu_lib
    with Plan(fs, 64, 64, L, L, 0) as p:
        with pytest.raises(fs.FsError):
            fs.fs_rk4_create(p.h, 0.0, wl.OrbitSource())
        with pytest.raises(fs.FsError):
            fs.fs_rk4_create(p.h, 1.0, wl.OrbitSource(sigma=0.0))
        rk = fs.fs_rk4_create(p.h, 1.0, wl.OrbitSource())
        try:
            with pytest.raises(fs.FsError):
                fs.fs_rk4_step(rk, 0.0, 1)
            with pytest.raises(fs.FsError):
                fs.fs_rk4_step(rk, 0.01, -1)
            with pytest.raises(fs.FsError):
                fs.fs_rk4_step(rk, float("nan"), 1)
        finally:
            fs.fs_rk4_destroy(rk)
