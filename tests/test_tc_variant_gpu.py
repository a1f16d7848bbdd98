"""Split-BF16 tensor-core first stage (measured variant, FS_COLUMN_VARIANT=bf16x3).

The variant replaces the first radix-16 stage of the inverse column
transform in advances by a tensor-core matmul with three-term BF16 operands.
It must stay within the FP32 bar against the float64 oracle (rel-L2 <= 1e-5)
on the 4096^2 wave snapshots the FP32 path is checked on, and it must
actually run (its rounding differs from the FP32 path's).
"""

import numpy as np
import pytest
import torch

import oracle
from oracle import closed_forms as cf
from paper_2412_12308_gb300 import fsolve, workloads as wl

pytestmark = pytest.mark.gpu


def _advance(plan, u0d, c, t, variant, monkeypatch):
    if variant:
        monkeypatch.setenv("FS_COLUMN_VARIANT", "bf16x3")
    else:
        monkeypatch.delenv("FS_COLUMN_VARIANT", raising=False)
    st = fsolve.fs_state_create(plan, u0d)
    out = torch.empty_like(u0d)
    try:
        fsolve.fs_wave_advance(st, c, t, out)
        torch.cuda.synchronize()
    finally:
        fsolve.fs_state_destroy(st)
    return out.double().cpu().numpy()


@pytest.mark.parametrize("n", [1024, 2048])
def test_tc_variant_modes(gpu_lib, n, monkeypatch):
    rng = np.random.default_rng(n)
    modes = wl.draw_modes(rng, 8, 30)
    f = wl.mode_sum(modes, n, n, 1.0, 1.0)
    plan = fsolve.fs_plan_create(n, n, 1.0, 1.0, fsolve.FS_F32)
    try:
        fd = torch.tensor(f, dtype=torch.float32, device="cuda")
        for t in (0.3, 1.7):
            want = cf.wave_modes(modes, 1.0, t, n, n, 1.0, 1.0)
            got = _advance(plan, fd, 1.0, t, True, monkeypatch)
            ref = _advance(plan, fd, 1.0, t, False, monkeypatch)
            assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 1e-5
            assert not np.array_equal(got, ref)
    finally:
        fsolve.fs_plan_destroy(plan)


def test_tc_variant_wave_4096(gpu_lib, monkeypatch):
    u0, (lx, ly), c, times, _ = wl.wave_pulse_4096()
    u0 = u0.astype(np.float32).astype(np.float64)
    n = u0.shape[0]
    plan = fsolve.fs_plan_create(n, n, lx, ly, fsolve.FS_F32)
    try:
        fd = torch.tensor(u0, dtype=torch.float32, device="cuda")
        F = oracle.state_spectrum(u0)
        # every 10th of the 50 snapshots (t = 0.2, 0.4, ..., 1), as for the FP32 path
        for t in [float(times[j]) for j in range(9, len(times), 10)]:
            U, _ = oracle.wave_spectrum(F, None, c, t, lx, ly)
            want = np.real(oracle.idft2(U))
            got = _advance(plan, fd, c, t, True, monkeypatch)
            assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 1e-5, t
    finally:
        fsolve.fs_plan_destroy(plan)
