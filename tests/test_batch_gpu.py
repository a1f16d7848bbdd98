"""Batch executor (one persistent launch per batch) on the GPU.

Checks: every problem of an uneven mixed batch matches the float64 oracle
(rel-L2 <= 1e-5; normwise for strongly decayed diffusion outputs); a request's
result is bit-identical alone and in a mix; batched results agree with the
per-call entry points; a repeated batch shape replays its CUDA graph with the
same results; staged column groups and C2R tiles (bulk / asynchronous
copies into shared memory) give results bit-identical to the unstaged units;
and an injected dependency that never completes ends the launch through the
bounded wait with FS_ERR_TIMEOUT, leaving the context usable.
"""

import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import oracle
from paper_2412_12308_gb300 import fsolve, workloads as wl

pytestmark = pytest.mark.gpu
F32 = fsolve.FS_F32


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


class Problems:
    """Device inputs/outputs and plans for a list of workloads.Problem."""

    def __init__(self, probs, dtype=F32):
        self.probs = probs
        self.dtype = dtype
        self.tdt = torch.float32 if dtype == F32 else torch.float64
        self.plans = {}
        self.inputs, self.outputs = [], []
        for p in probs:
            if p.n not in self.plans:
                self.plans[p.n] = fsolve.fs_plan_create(p.n, p.n, p.lx, p.ly, dtype)
            f = p.field(np.float64).astype(np.float32 if dtype == F32 else np.float64)
            self.inputs.append(torch.tensor(f, device="cuda"))
            self.outputs.append(torch.full_like(self.inputs[-1], float("nan")))

    def requests(self, idx=None):
        out = []
        for i in (range(len(self.probs)) if idx is None else idx):
            p = self.probs[i]
            op = {"poisson": fsolve.FS_OP_POISSON, "diffusion": fsolve.FS_OP_DIFFUSION,
                  "wave": fsolve.FS_OP_WAVE}[p.op]
            out.append(fsolve.fs_request(op, plan=self.plans[p.n], in_u=self.inputs[i], out_u=self.outputs[i],
                                         D=p.D, c=p.c, t=p.t))
        return out

    def close(self):
        for h in self.plans.values():
            fsolve.fs_plan_destroy(h)


def oracle_of(p, f64):
    if p.op == "poisson":
        return oracle.poisson(f64, p.lx, p.ly)
    if p.op == "diffusion":
        return oracle.diffusion(f64, p.D, p.t, p.lx, p.ly)
    return oracle.wave(f64, None, p.c, p.t, p.lx, p.ly)


def check_vs_oracle(P, i, got):
    p = P.probs[i]
    f = P.inputs[i].double().cpu().numpy()
    want = oracle_of(p, f)
    den = np.linalg.norm(want)
    if p.op == "diffusion":
        den = max(den, np.linalg.norm(f))
    return float(np.linalg.norm(got - want) / den)


def test_mixed_batch_vs_oracle_and_alone(gpu_lib):
    probs = wl.batch_mix(seed=99, count=48, sizes=(64, 80, 96, 128, 160, 192, 256, 320, 384, 512, 640, 768))
    P = Problems(probs)
    try:
        t = fsolve.fs_batch_submit(P.requests())
        fsolve.fs_batch_wait(t, 30_000_000)
        mixed = [o.clone() for o in P.outputs]
        for i in range(len(probs)):
            err = check_vs_oracle(P, i, mixed[i].double().cpu().numpy())
            assert err <= 1e-5, (i, probs[i].op, probs[i].n, err)
        # each request alone in its own batch: bit-identical
        for i in range(0, len(probs), 5):
            P.outputs[i].fill_(float("nan"))
            t = fsolve.fs_batch_submit(P.requests([i]))
            fsolve.fs_batch_wait(t, 30_000_000)
            assert torch.equal(P.outputs[i], mixed[i]), (i, probs[i].op, probs[i].n)
        # replay of the same batch shape (cached graph): same results
        for o in P.outputs:
            o.fill_(float("nan"))
        t = fsolve.fs_batch_submit(P.requests())
        fsolve.fs_batch_wait(t, 30_000_000)
        for i in range(len(probs)):
            assert torch.equal(P.outputs[i], mixed[i])
    finally:
        P.close()


def test_batch_matches_per_call_entry_points(gpu_lib):
    probs = wl.batch_mix(seed=7, count=12, sizes=(64, 128, 256, 512, 1024))
    P = Problems(probs)
    try:
        t = fsolve.fs_batch_submit(P.requests())
        fsolve.fs_batch_wait(t, 30_000_000)
        for i, p in enumerate(probs):
            ref = torch.empty_like(P.outputs[i])
            h = P.plans[p.n]
            if p.op == "poisson":
                fsolve.fs_poisson_solve(h, P.inputs[i], ref)
            elif p.op == "diffusion":
                fsolve.fs_diffusion_solve(h, P.inputs[i], p.D, p.t, ref)
            else:
                fsolve.fs_wave_solve(h, P.inputs[i], None, p.c, p.t, ref)
            torch.cuda.synchronize()
            d = float((P.outputs[i].double() - ref.double()).norm())
            den = max(float(ref.double().norm()), float(P.inputs[i].double().norm()) * 1e-2)
            assert d / den <= 1e-6, (i, p.op, p.n, d / den)
    finally:
        P.close()


@pytest.mark.parametrize("dtype", [0, 1])
def test_batched_advances_from_kept_states(gpu_lib, dtype):
    tdt = torch.float32 if dtype == 0 else torch.float64
    tol = 1e-5 if dtype == 0 else 1e-12
    n, lx = 256, 2 * np.pi
    u0, blobs, _, D, times = wl.diffusion_blobs_1024(n=n, n_times=12)
    v0 = np.random.default_rng(2).standard_normal((n, n)) * 0.1
    u0 = u0.astype(np.float32).astype(np.float64)
    v0 = v0.astype(np.float32).astype(np.float64)
    plan = fsolve.fs_plan_create(n, n, lx, lx, dtype)
    ud, vd = torch.tensor(u0, dtype=tdt, device="cuda"), torch.tensor(v0, dtype=tdt, device="cuda")
    s1 = fsolve.fs_state_create(plan, ud)
    s2 = fsolve.fs_state_create(plan, ud, vd)
    try:
        outs, reqs = [], []
        for t in times:
            o = torch.empty_like(ud)
            outs.append(("diff", float(t), o, None))
            reqs.append(fsolve.fs_request(fsolve.FS_OP_DIFFUSION_ADVANCE, state=s1, out_u=o, D=D, t=float(t)))
        for t in times[::3]:
            o, ov = torch.empty_like(ud), torch.empty_like(ud)
            outs.append(("wave", float(t), o, ov))
            reqs.append(fsolve.fs_request(fsolve.FS_OP_WAVE_ADVANCE, state=s2, out_u=o, out_v=ov, c=1.3, t=float(t)))
        tk = fsolve.fs_batch_submit(reqs)
        fsolve.fs_batch_wait(tk, 30_000_000)
        F, G = oracle.state_spectrum(u0), oracle.state_spectrum(v0)
        for kind, t, o, ov in outs:
            if kind == "diff":
                want = np.real(oracle.idft2(oracle.diffusion_spectrum(F, D, t, lx, lx)))
                assert rel(o.cpu().numpy(), want) <= tol, (kind, t)
            else:
                U, V = oracle.wave_spectrum(F, G, 1.3, t, lx, lx)
                assert rel(o.cpu().numpy(), np.real(oracle.idft2(U))) <= tol, (kind, t)
                assert rel(ov.cpu().numpy(), np.real(oracle.idft2(V))) <= tol, (kind, t)
    finally:
        fsolve.fs_state_destroy(s1)
        fsolve.fs_state_destroy(s2)
        fsolve.fs_plan_destroy(plan)


def test_outputs_in_pinned_host_memory(gpu_lib):
    """Output fields in pinned host memory (mapped into the device's address
    space) are stored by the kernels directly: identical to device outputs,
    for the batch (small and three-pass problems) and a per-call advance."""
    n1, n2 = 128, 1024
    rng = np.random.default_rng(44)
    plans, states, reqs_d, reqs_h, dev, hst = [], [], [], [], [], []
    try:
        for n in (n1, n2):
            plan = fsolve.fs_plan_create(n, n, 1.0, 1.0, F32)
            plans.append(plan)
            u0 = torch.tensor(rng.standard_normal((n, n)), dtype=torch.float32, device="cuda")
            st = fsolve.fs_state_create(plan, u0)
            states.append(st)
            for t in (0.001, 0.01):
                od = torch.empty((n, n), dtype=torch.float32, device="cuda")
                oh = torch.full((n, n), float("nan"), dtype=torch.float32).pin_memory()
                dev.append(od)
                hst.append(oh)
                reqs_d.append(fsolve.fs_request(fsolve.FS_OP_DIFFUSION_ADVANCE, state=st, out_u=od, D=0.1, t=t))
                reqs_h.append(fsolve.fs_request(fsolve.FS_OP_DIFFUSION_ADVANCE, state=st, out_u=oh.data_ptr(),
                                                D=0.1, t=t))
        fsolve.fs_batch_wait(fsolve.fs_batch_submit(reqs_d), 30_000_000)
        fsolve.fs_batch_wait(fsolve.fs_batch_submit(reqs_h), 30_000_000)
        torch.cuda.synchronize()
        for od, oh in zip(dev, hst):
            assert torch.equal(od.cpu(), oh)
        oh = torch.empty((n2, n2), dtype=torch.float32).pin_memory()
        fsolve.fs_diffusion_advance(states[1], 0.1, 0.01, oh.data_ptr())
        torch.cuda.synchronize()
        assert torch.equal(dev[3].cpu(), oh)
    finally:
        for st in states:
            fsolve.fs_state_destroy(st)
        for plan in plans:
            fsolve.fs_plan_destroy(plan)


def test_bounded_wait_expires_without_fault(gpu_lib, monkeypatch):
    # the 64^2 problems run as the small problems' second launch beside the
    # persistent one; the stall is injected into the persistent launch
    probs = wl.batch_mix(seed=5, count=8, sizes=(64, 512, 1024))
    P = Problems(probs)
    try:
        monkeypatch.setenv("FS_BATCH_INJECT_STALL", "1")
        monkeypatch.setenv("FS_BATCH_WAIT_NS", str(20_000_000))  # 20 ms
        t = fsolve.fs_batch_submit(P.requests())
        with pytest.raises(fsolve.FsError) as ei:
            fsolve.fs_batch_wait(t, 30_000_000)
        assert ei.value.status == -6  # FS_ERR_TIMEOUT
        monkeypatch.delenv("FS_BATCH_INJECT_STALL")
        monkeypatch.delenv("FS_BATCH_WAIT_NS")
        # the context is still usable and results are right afterwards
        for o in P.outputs:
            o.fill_(float("nan"))
        t = fsolve.fs_batch_submit(P.requests())
        fsolve.fs_batch_wait(t, 30_000_000)
        for i in range(len(probs)):
            assert check_vs_oracle(P, i, P.outputs[i].double().cpu().numpy()) <= 1e-5
    finally:
        P.close()


# (nx, ny): power-of-two rows and columns (staged), a ragged last C2R tile
# (ny = 40 with 16-row tiles), rows of 8192 (one-row tiles: unstaged),
# columns of 96 (no compiled length: unstaged columns, staged rows);
# 3 x 2^k and 5 x 2^k rows and columns (staged with tiles 24 / 20), one
# with a ragged last C2R tile (rows of 640 points, 16-row tiles, ny = 40)
STAGED_SHAPES = [(256, 40), (1024, 96), (2048, 256), (512, 512), (1024, 1024), (8192, 128),
                 (1536, 768), (1280, 1536), (768, 160), (640, 40)]


def staged_case():
    """One batch over STAGED_SHAPES: the three solves, diffusion and wave
    advances from kept spectra (the wave also with v).  Returns the outputs
    in request order."""
    rng = np.random.default_rng(321)
    plans, states, outs, reqs = [], [], [], []
    inputs = []  # the requests hold raw addresses: keep every input alive until the batch ends
    try:
        for nx, ny in STAGED_SHAPES:
            plan = fsolve.fs_plan_create(nx, ny, 1.0, 1.3, F32)
            plans.append(plan)
            f = torch.tensor(rng.standard_normal((ny, nx)), dtype=torch.float32, device="cuda")
            g = torch.tensor(rng.standard_normal((ny, nx)), dtype=torch.float32, device="cuda")
            inputs += [f, g]
            s1, s2 = fsolve.fs_state_create(plan, f), fsolve.fs_state_create(plan, f, g)
            states += [s1, s2]

            def out():
                outs.append(torch.full((ny, nx), float("nan"), dtype=torch.float32, device="cuda"))
                return outs[-1]
            reqs.append(fsolve.fs_request(fsolve.FS_OP_POISSON, plan=plan, in_u=f, out_u=out()))
            reqs.append(fsolve.fs_request(fsolve.FS_OP_DIFFUSION, plan=plan, in_u=f, out_u=out(), D=0.01, t=0.3))
            reqs.append(fsolve.fs_request(fsolve.FS_OP_WAVE, plan=plan, in_u=f, out_u=out(), c=1.0, t=0.4))
            reqs.append(fsolve.fs_request(fsolve.FS_OP_DIFFUSION_ADVANCE, state=s1, out_u=out(), D=0.01, t=0.2))
            reqs.append(fsolve.fs_request(fsolve.FS_OP_WAVE_ADVANCE, state=s1, out_u=out(), c=1.0, t=0.7))
            u, v = out(), out()
            reqs.append(fsolve.fs_request(fsolve.FS_OP_WAVE_ADVANCE, state=s2, out_u=u, out_v=v, c=1.0, t=0.7))
        fsolve.fs_batch_wait(fsolve.fs_batch_submit(reqs), 30_000_000)
        torch.cuda.synchronize()
        return [o.cpu().numpy() for o in outs]
    finally:
        for st in states:
            fsolve.fs_state_destroy(st)
        for plan in plans:
            fsolve.fs_plan_destroy(plan)


_UNSTAGED = """
import sys
import numpy as np
from tests.test_batch_gpu import staged_case
np.savez(sys.argv[1], *staged_case())
"""


def test_staged_units_bit_identical_to_unstaged(gpu_lib, tmp_path, monkeypatch):
    """Staging moves data only: the staged batch (this process) and the
    unstaged one (a child process with FS_NO_TMA=1) agree bit for bit, and
    every output is finite.  Problems run as units (no single-CTA path)."""
    monkeypatch.setenv("FS_BATCH_SMALL_MAX", "0")
    got = staged_case()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, FS_NO_TMA="1", FS_BATCH_SMALL_MAX="0")
    path = tmp_path / "unstaged.npz"
    subprocess.run([sys.executable, "-c", _UNSTAGED, str(path)], env=env, cwd=root, check=True, timeout=600)
    ref = np.load(path)
    assert len(ref.files) == len(got)
    for i, o in enumerate(got):
        assert np.isfinite(o).all(), i
        assert np.array_equal(o, ref[f"arr_{i}"]), (i, STAGED_SHAPES[i // 7])

