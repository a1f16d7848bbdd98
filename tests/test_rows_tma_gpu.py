"""The persistent TMA-staged row passes (GPU).

FP32 grids whose row transform has length nx/2 in {512, 1024, 2048, 4096}
run their R2C and C2R passes as persistent kernels that move tiles with the
tensor memory accelerator (bulk row copies, 2D tensor-map spectrum tiles).
They change the data movement only, so every output must equal, bit for bit,
the one computed by the plain-load row kernels (a child process with
FS_NO_TMA=1), and match the exact closed forms (mode-sum fields, Sec. III).
Two-field passes (a wave solve with an initial velocity: two R2C fields; an
advance that also returns v: two C2R fields) are covered too.
"""

import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from oracle import closed_forms as cf
from paper_2412_12308_gb300 import fsolve, workloads as wl

pytestmark = pytest.mark.gpu

GRIDS = [(1024, 1024), (2048, 2048), (4096, 4096), (8192, 512), (2048, 1536), (1024, 96)]


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _case(nx, ny):
    rng = np.random.default_rng(nx + 5 * ny)
    kmax = min(40, ny // 2 - 1)
    mu, mv = wl.draw_modes(rng, 8, kmax), wl.draw_modes(rng, 6, kmax)
    return mu, mv, wl.mode_sum(mu, nx, ny, 1.0, 1.0), wl.mode_sum(mv, nx, ny, 1.0, 1.0)


def run_case(nx, ny):
    """Outputs of every two-field and one-field path on one grid (host arrays)."""
    fsolve.load()
    mu, mv, f, g = _case(nx, ny)
    plan = fsolve.fs_plan_create(nx, ny, 1.0, 1.0, fsolve.FS_F32)
    fd = torch.tensor(f, dtype=torch.float32, device="cuda")
    gd = torch.tensor(g, dtype=torch.float32, device="cuda")
    outs = []
    try:
        u, v = torch.empty_like(fd), torch.empty_like(fd)
        fsolve.fs_poisson_solve(plan, fd, u)
        outs.append(u.cpu().numpy())
        fsolve.fs_wave_solve(plan, fd, gd, 1.1, 0.43, u)  # two R2C fields
        outs.append(u.cpu().numpy())
        st = fsolve.fs_state_create(plan, fd, gd)
        try:
            fsolve.fs_wave_advance(st, 1.1, 0.43, u, v)  # two C2R fields
            outs += [u.cpu().numpy(), v.cpu().numpy()]
        finally:
            fsolve.fs_state_destroy(st)
    finally:
        fsolve.fs_plan_destroy(plan)
    return outs


_PLAIN = """
import sys, numpy as np
sys.path.insert(0, '.')
from tests.test_rows_tma_gpu import run_case, GRIDS
res = {}
for nx, ny in GRIDS:
    for j, o in enumerate(run_case(nx, ny)):
        res[f"{nx}_{ny}_{j}"] = o
np.savez(sys.argv[1], **res)
"""


def _wave_closed(mu, mv, c, t, nx, ny):
    """u(t), v(t) for u0 = mode sum mu, v0 = mode sum mv (Eq. OmegaNonZero and
    its time derivative): each mode of u0 oscillates as cos(c|w|t), each mode
    of v0 as sin(c|w|t)/(c|w|)."""
    def cw(m):
        return c * 2 * np.pi * np.hypot(m[0], m[1])
    u = cf.mode_field(mu, nx, ny, 1.0, 1.0, [np.cos(cw(m) * t) for m in mu]) + \
        cf.mode_field(mv, nx, ny, 1.0, 1.0, [np.sin(cw(m) * t) / cw(m) for m in mv])
    v = cf.mode_field(mu, nx, ny, 1.0, 1.0, [-cw(m) * np.sin(cw(m) * t) for m in mu]) + \
        cf.mode_field(mv, nx, ny, 1.0, 1.0, [np.cos(cw(m) * t) for m in mv])
    return u, v


@pytest.mark.parametrize("nx,ny", GRIDS)
def test_rows_tma_closed_forms(gpu_lib, nx, ny):
    mu, mv, _f, _g = _case(nx, ny)
    up, uw, ua, va = run_case(nx, ny)
    assert _rel(up, cf.poisson_modes(mu, nx, ny, 1.0, 1.0)) <= 1e-5
    u_t, v_t = _wave_closed(mu, mv, 1.1, 0.43, nx, ny)
    assert _rel(uw, u_t) <= 1e-5
    assert _rel(ua, u_t) <= 1e-5
    assert _rel(va, v_t) <= 1e-5


def test_rows_tma_bit_identical_to_plain_rows(gpu_lib, tmp_path):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    path = tmp_path / "plain.npz"
    env = dict(os.environ, FS_NO_TMA="1")
    subprocess.run([sys.executable, "-c", _PLAIN, str(path)], env=env, cwd=root, check=True, timeout=900)
    ref = np.load(path)
    for nx, ny in GRIDS:
        for j, o in enumerate(run_case(nx, ny)):
            assert np.isfinite(o).all(), (nx, ny, j)
            assert np.array_equal(o, ref[f"{nx}_{ny}_{j}"]), (nx, ny, j)
