"""Precision of the FP32 path's spectral factors against FP64-evaluated ones (GPU).

The FP32 column pass forms |omega|^2 = w_x^2 + w_y^2 and the Poisson factor
-1/(nx ny |omega|^2) in two-float (~44 bits) and rounds once; diffusion as
the two-float product of per-axis FP64 exponentials; the wave phase
c t |omega| in two-float, reduced modulo 2 pi with a two-part 2 pi, then the
hardware sine/cosine of the reduced angle (absolute error below 2^-21.4).
fs_operator_factors evaluates the same factors element by element both ways
(as the column pass does, and in FP64 rounded once); this checks the bounds
stated for them on every half-spectrum element, and the FP64 evaluation
against float64 NumPy of the Sec. III multipliers.
"""

import numpy as np
import pytest
import torch

from oracle.solve import omega_axis
from paper_2412_12308_gb300 import fsolve

pytestmark = pytest.mark.gpu

ULP = 2.0 ** -23  # float32 unit roundoff x 2


def _factors(plan, n, ny, op, fp64, **kw):
    out = torch.empty((n // 2 + 1) * ny, dtype=torch.float32, device="cuda")
    fsolve.fs_operator_factors(plan, op, out, fp64=fp64, **kw)
    torch.cuda.synchronize()
    return out.double().cpu().numpy().reshape(n // 2 + 1, ny)


@pytest.mark.parametrize("nx,ny,lx,ly", [(1024, 1024, 1.0, 1.0), (4096, 4096, 1.0, 1.0), (640, 384, 2.0, 0.7)])
def test_factor_precision(gpu_lib, nx, ny, lx, ly):
    plan = fsolve.fs_plan_create(nx, ny, lx, ly, fsolve.FS_F32)
    try:
        scale = 1.0 / (nx * ny)
        wx = omega_axis(nx, lx)[: nx // 2 + 1]
        wy = omega_axis(ny, ly)
        w2 = wx[:, None] ** 2 + wy[None, :] ** 2  # [a][b]
        th = 1.3 * 0.77 * np.sqrt(w2)
        # (op, parameters, float64 NumPy value, its float64 error bound: the
        # GPU's FP64 evaluation forms the argument in another order, ~1e-16
        # relative, which exp and cos pass on scaled by their argument)
        cases = [(fsolve.FS_OP_POISSON, {}, np.where(w2 > 0, -scale / np.where(w2 > 0, w2, 1.0), 0.0), None),
                 (fsolve.FS_OP_DIFFUSION, {"D": 0.013, "t": 0.41}, scale * np.exp(-0.013 * 0.41 * w2),
                  lambda e: 1e-15 * (1.0 + 0.013 * 0.41 * w2) * np.abs(e)),
                 (fsolve.FS_OP_WAVE, {"c": 1.3, "t": 0.77}, scale * np.cos(th), lambda e: 1e-15 * (1.0 + th) * scale)]
        tiny = np.finfo(np.float32).tiny
        for op, kw, exact, err64 in cases:
            f32 = _factors(plan, nx, ny, op, False, **kw)
            f64 = _factors(plan, nx, ny, op, True, **kw)
            e64 = (1e-13 * np.abs(exact)) if err64 is None else err64(exact)
            # FP64 rounded once: half an ulp from the float64 value, plus its error
            assert np.all(np.abs(f64 - exact) <= 0.5 * ULP * np.abs(exact) + e64 + tiny), op
            if op == fsolve.FS_OP_WAVE:
                # two-float phase, hardware sine/cosine of the reduced angle
                # (2^-21.4) plus one rounding of each side
                assert np.max(np.abs(f32 - f64)) <= 6e-7 * scale, op
            else:
                # two-float, rounded once: at most one ulp from FP64 rounded once
                assert np.all(np.abs(f32 - f64) <= ULP * np.abs(f64) + e64 + tiny), op
    finally:
        fsolve.fs_plan_destroy(plan)
