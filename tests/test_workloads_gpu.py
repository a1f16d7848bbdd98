"""The measured workloads at full size on the GPU.

* 512-problem uneven batch (N in {64..2048}, Poisson / diffusion / wave, 8-mode
  sources) in one persistent launch: every problem against its closed form
  (exact for mode sums), rel-L2 <= 1e-5 (normwise for strongly decayed
  diffusion, the largest diffusion multiplier being 1).
* Wave 4096^2 with a Gaussian pulse plus white noise, 50 snapshots from one
  kept spectrum in one batch: every 10th snapshot (t = 0.2, 0.4, ..., 1)
  against the float64 oracle (rel-L2 <= 1e-5), the mean invariant on all 50.
* Diffusion 1024^2, 100 output times: every output against the periodic heat
  kernel (exact on this grid: the narrowest blob's spectrum is e^-164 at
  Nyquist), rel-L2 <= 1e-5.
"""

import numpy as np
import pytest
import torch

import oracle
from oracle import closed_forms as cf
from paper_2412_12308_gb300 import fsolve, workloads as wl

pytestmark = pytest.mark.gpu


def test_batch_mix_512_closed_forms(gpu_lib):
    probs = wl.batch_mix()
    plans, ins, outs = {}, [], []
    try:
        for p in probs:
            if p.n not in plans:
                plans[p.n] = fsolve.fs_plan_create(p.n, p.n, p.lx, p.ly, fsolve.FS_F32)
            ins.append(torch.tensor(p.field(np.float32), device="cuda"))
            outs.append(torch.full_like(ins[-1], float("nan")))
        ops = {"poisson": fsolve.FS_OP_POISSON, "diffusion": fsolve.FS_OP_DIFFUSION, "wave": fsolve.FS_OP_WAVE}
        reqs = [fsolve.fs_request(ops[p.op], plan=plans[p.n], in_u=ins[i], out_u=outs[i], D=p.D, c=p.c, t=p.t)
                for i, p in enumerate(probs)]
        t = fsolve.fs_batch_submit(reqs)
        fsolve.fs_batch_wait(t, 60_000_000)
        worst = 0.0
        for i, p in enumerate(probs):
            got = outs[i].double().cpu().numpy()
            if p.op == "poisson":
                want = cf.poisson_modes(p.modes, p.n, p.n, p.lx, p.ly)
                den = np.linalg.norm(want)
            elif p.op == "diffusion":
                want = cf.diffusion_modes(p.modes, p.D, p.t, p.n, p.n, p.lx, p.ly)
                den = max(np.linalg.norm(want), np.linalg.norm(ins[i].double().cpu().numpy()))
            else:
                want = cf.wave_modes(p.modes, p.c, p.t, p.n, p.n, p.lx, p.ly)
                den = np.linalg.norm(want)
            err = float(np.linalg.norm(got - want) / den)
            worst = max(worst, err)
            assert err <= 1e-5, (i, p.op, p.n, err)
    finally:
        for h in plans.values():
            fsolve.fs_plan_destroy(h)


def test_wave_4096_snapshots_vs_oracle(gpu_lib):
    u0, (lx, ly), c, times, _ = wl.wave_pulse_4096()
    u0 = u0.astype(np.float32).astype(np.float64)
    n = u0.shape[0]
    plan = fsolve.fs_plan_create(n, n, lx, ly, fsolve.FS_F32)
    ud = torch.tensor(u0, dtype=torch.float32, device="cuda")
    st = fsolve.fs_state_create(plan, ud)
    outs = torch.empty((len(times), n, n), dtype=torch.float32, device="cuda")
    try:
        reqs = [fsolve.fs_request(fsolve.FS_OP_WAVE_ADVANCE, state=st, out_u=outs[j], c=c, t=float(t))
                for j, t in enumerate(times)]
        tk = fsolve.fs_batch_submit(reqs)
        fsolve.fs_batch_wait(tk, 60_000_000)
        F = oracle.state_spectrum(u0)
        m0 = u0.mean()
        for j in list(range(9, len(times), 10)):
            U, _ = oracle.wave_spectrum(F, None, c, float(times[j]), lx, ly)
            want = np.real(oracle.idft2(U))
            got = outs[j].double().cpu().numpy()
            err = float(np.linalg.norm(got - want) / np.linalg.norm(want))
            assert err <= 1e-5, (j, err)
        for j in range(len(times)):  # mean conserved (v0 = 0)
            assert abs(float(outs[j].double().mean()) - m0) <= 1e-5 * float(np.abs(u0).max())
    finally:
        fsolve.fs_state_destroy(st)
        fsolve.fs_plan_destroy(plan)


def test_diffusion_1024_heat_kernel_all_times(gpu_lib):
    u0, blobs, (lx, ly), D, times = wl.diffusion_blobs_1024()
    n = u0.shape[0]
    plan = fsolve.fs_plan_create(n, n, lx, ly, fsolve.FS_F32)
    ud = torch.tensor(u0.astype(np.float32), device="cuda")
    st = fsolve.fs_state_create(plan, ud)
    outs = torch.empty((len(times), n, n), dtype=torch.float32, device="cuda")
    try:
        reqs = [fsolve.fs_request(fsolve.FS_OP_DIFFUSION_ADVANCE, state=st, out_u=outs[j], D=D, t=float(t))
                for j, t in enumerate(times)]
        tk = fsolve.fs_batch_submit(reqs)
        fsolve.fs_batch_wait(tk, 60_000_000)
        assert len(times) == 100
        for j in range(len(times)):
            want = cf.gaussian_heat(blobs, D, float(times[j]), n, n, lx, ly, images=1)
            got = outs[j].double().cpu().numpy()
            err = float(np.linalg.norm(got - want) / np.linalg.norm(want))
            assert err <= 1e-5, (j, err)
    finally:
        fsolve.fs_state_destroy(st)
        fsolve.fs_plan_destroy(plan)
