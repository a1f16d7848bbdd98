#!/usr/bin/env python
"""Benchmark of the 2D Fourier-space solve on GB300 (one JSON line on stdout).

Default workload (one "step"): diffusion u_t = D lap u on periodic
[0, 2 pi)^2, 1024 x 1024, FP32, D = 0.1, initial field = 16 seeded periodic
Gaussian blobs; the spectrum is computed once per step and kept on the
device, then u(t) is produced at 100 output times evenly spaced in [0, 1].
A step = 1 forward transform into the kept state + 100 advances (inverse
transforms), i.e. 100 solves; the 100 advances run as one persistent batch
launch.  The metric is solves per second.

Arms:
  --impl ours        this library through its C ABI (default)
  --impl reference   the float64 CPU oracle on the host cores (the whole step
                     of the same workload: 1 forward 2D DFT + 100 outputs)

Beside the headline the line carries `legs`, further workloads of the same
metric, each with its own roofline: the one-shot Poisson solve on 4096^2 with
the plain per-solve torch.fft path beside it, the 4096^2 wave with 50
snapshots from one kept spectrum, and the 512-problem uneven batch.  Their
accuracy against the float64 oracle (or exact closed forms) is computed in
the CPU-baseline leg.  `--leg NAME` runs one of them alone (for profilers).

Multi-GPU (torchrun, one rank per GPU): every rank runs its own copy of the
headline workload (replicas, weak scaling); the 512-problem batch is split
across ranks (replicas.shard); times are the max over ranks.
"""

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "2D solves/s & HBM GB/s vs plain GPU path at rel-L2≤1e-5; served p50/p99 latency"
N = 1024
N_TIMES = 100
WORKLOAD = ("diffusion u_t = D lap u, periodic [0,2pi)^2, 1024x1024 FP32, D=0.1, 16 seeded "
            "Gaussian blobs, spectrum kept on device, 100 output times evenly spaced in [0,1]")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle timing leg")
    ap.add_argument("--no-serving", action="store_true", help="skip the open-loop serving leg")
    ap.add_argument("--serve-requests", type=int, default=20000)
    ap.add_argument("--legs", default=",".join(LEGS),
                    help="comma-separated extra workloads reported beside the headline ('' for none)")
    ap.add_argument("--leg", choices=sorted(LEG_FNS), default=None,
                    help="run only this workload and print its JSON (e.g. under a profiler)")
    return ap.parse_args()


# ----------------------------------------------------------------------------- distributed
class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = False

    def init(self, backend):
        if self.world > 1:
            import torch.distributed as dist

            dist.init_process_group(backend)
            self.pg = True

    def barrier(self):
        if self.pg:
            import torch.distributed as dist

            dist.barrier()

    def max(self, x):
        if not self.pg:
            return x
        import torch
        import torch.distributed as dist

        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            import torch.distributed as dist

            dist.destroy_process_group()


# ----------------------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi sampled every 200 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="fs_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            out["reasons"] = ["nvidia-smi unavailable"]
            return out
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return out
        sm = [float(r[1]) for r in rows]
        out["samples"] = len(rows)
        out["sm_mhz"] = statistics.median(sm)
        out["sm_max_mhz"] = float(rows[0][2])
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = set()
        for r in rows:
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        out["reasons"] = sorted(reasons)
        out["power_w_max"] = max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())
        return out


# ----------------------------------------------------------------------------- workload
def workload():
    from paper_2412_12308_gb300 import workloads

    u0, blobs, (lx, ly), D, times = workloads.diffusion_blobs_1024(n=N, n_times=N_TIMES)
    return u0.astype(np.float32), blobs, lx, ly, D, times


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def cpu_baseline(u0, lx, ly, D, times, gpu_out=None, n_snap=None):
    """The float64 oracle as it stands on the host cores: one forward 2D DFT
    (the kept spectrum) and n_snap of the output times (default: all of them,
    i.e. the whole step, ~5 s on 16 cores), scaled to a full step
    (1 forward + 100 outputs) when n_snap is smaller."""
    import oracle

    t0 = time.perf_counter()
    F = oracle.state_spectrum(u0.astype(np.float64))
    t_fwd = time.perf_counter() - t0
    n_snap = len(times) if n_snap is None else n_snap
    pick = np.linspace(0, len(times) - 1, n_snap).round().astype(int)
    t1 = time.perf_counter()
    outs = []
    for j in pick:
        U = oracle.diffusion_spectrum(F, D, float(times[j]), lx, ly)
        outs.append(np.real(oracle.idft2(U)))
    t_snap = (time.perf_counter() - t1) / len(pick)
    step_s = t_fwd + len(times) * t_snap
    res = {
        "value": len(times) / step_s,
        "unit": "solves/s",
        "cores": os.cpu_count(),
        "kind": "oracle",
        "sample": (f"float64 direct-DFT oracle: the whole step, 1 forward 2D DFT + all {len(times)} output times"
                   if len(pick) == len(times) else
                   f"float64 direct-DFT oracle: 1 forward 2D DFT + {len(pick)} of the {len(times)} output "
                   f"times (t = {', '.join(f'{float(times[j]):.3f}' for j in pick)}), scaled to 1 forward + "
                   f"{len(times)} outputs"),
        "seconds": t_fwd + t_snap * len(pick),
    }
    if gpu_out is not None:
        errs = []
        for k, j in enumerate(pick):
            g = gpu_out[j].astype(np.float64)
            errs.append(float(np.linalg.norm(g - outs[k]) / np.linalg.norm(outs[k])))
        res["rel_l2_vs_oracle_max"] = max(errs)
    return res


# ----------------------------------------------------------------------------- ours
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of a
# workload's kernels from ncu captures (summaries under profiles/), valid only
# for the CUDA sources they were taken on: any change to the sources makes the
# reported traffic null until a new capture.
# (workload, kernel class) -> {"bytes": DRAM bytes per launch, "sources_sha256": digest of csrc/}
_SRC = "40b891cdd74796c97d907071010876e0d4d3a4b6bbe4f795d4a1a1a4b04eedd3"
TRAFFIC_CAPTURES = {
    # profiles/k_batch_diffusion_1024.md
    ("diffusion_1024", "batch"): {"bytes": 168_669_952 + 784_116_992, "sources_sha256": _SRC},
    # profiles/poisson_4096_pass_kernels.md
    ("poisson_4096", "row_r2c"): {"bytes": 67_155_200 + 20_592_640, "sources_sha256": _SRC},
    ("poisson_4096", "column"): {"bytes": 67_234_816 + 4_069_632, "sources_sha256": _SRC},
    ("poisson_4096", "row_c2r"): {"bytes": 67_198_720 + 13_627_648, "sources_sha256": _SRC},
    # profiles/wave_4096_snapshots_and_batch_mix_traffic.md
    ("wave_4096_snapshots", "column"): {"bytes": 67_242_240 + 8_427_520, "sources_sha256": _SRC},
    # both launches of the batch: the persistent one and the small problems' one
    ("batch_mix_512", "batch"): {"bytes": 4_151_266_816 + 4_488_077_568 + 13_422_592 + 57_344,
                                 "sources_sha256": _SRC},
}


def _csrc_digest():
    import glob
    import hashlib

    h = hashlib.sha256()
    root = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2412_12308_gb300", "csrc")
    for f in sorted(glob.glob(os.path.join(root, "*"))):
        if f.endswith((".cu", ".cuh", ".h")):
            h.update(os.path.basename(f).encode())
            with open(f, "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()


# ----------------------------------------------------------------------------- legs
# Further workloads of the same metric, reported beside the headline (each a
# configuration of the measured set): the one-shot 4096^2 Poisson solve with
# the plain per-solve comparator, the 4096^2 wave with 50 snapshots from one
# kept spectrum, and the 512-problem uneven batch (sharded across ranks).
LEGS = ("poisson_4096", "wave_4096_snapshots", "batch_mix_512", "factors_4096")


def _spec_bytes(n, esz=4):
    return (n // 2 + 1) * n * 2 * esz


def _events_ms(torch, fn, reps, flush):
    """Device time of `reps` calls of fn, L2 flushed (untimed) before each."""
    ms = []
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    return ms


def _kernel_us(fsolve, torch, fn, reps, flush):
    """Mean device time per launch of each pass class (library events on the
    launching stream) over `reps` calls of fn."""
    fsolve.fs_profile_enable(True)
    for _ in range(reps):
        flush.zero_()
        fn()
    torch.cuda.synchronize()
    prof = fsolve.fs_profile_report()
    fsolve.fs_profile_enable(False)
    return {k: (c, 1e3 * tot / c) for k, (c, tot) in prof.items() if c}


def _roof(algo_bytes, seconds, peak, peak_src, traffic=None, **extra):
    gbs = algo_bytes / seconds / 1e9 if seconds > 0 else 0.0
    out = {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s", "frac": round(gbs / peak, 4),
           "frac_of_8tbs": round(gbs / 8000.0, 4), "traffic": traffic, "peak_source": peak_src,
           "algorithmic_bytes_per_launch": int(algo_bytes)}
    out.update(extra)
    return out


def _capture_traffic(leg, kernel):
    """DRAM bytes per launch of `kernel` in `leg` from the ncu capture listed in
    TRAFFIC_CAPTURES, if it was taken on the current kernel sources."""
    cap = TRAFFIC_CAPTURES.get((leg, kernel))
    if cap and _csrc_digest() == cap["sources_sha256"]:
        return cap["bytes"]
    return None


def leg_poisson_4096(ctx):
    """One-shot Poisson solve on a 4096^2 FP32 grid (8-mode source, |k| <= 40,
    exact closed form), one solve per call, L2 flushed between calls; beside it
    the plain per-solve path: torch.fft.rfft2 -> multiply by -1/|k|^2 ->
    torch.fft.irfft2 (cuFFT, separate launches)."""
    torch, fsolve, dev, flush, reps = ctx["torch"], ctx["fsolve"], ctx["dev"], ctx["flush"], ctx["reps"]
    from paper_2412_12308_gb300 import workloads as wl

    n = 4096
    modes = wl.draw_modes(np.random.default_rng(12313), 8, 40)
    f = wl.mode_sum(modes, n, n, 1.0, 1.0).astype(np.float32)
    plan = fsolve.fs_plan_create(n, n, 1.0, 1.0, fsolve.FS_F32)
    fd = torch.tensor(f, device=dev)
    ud = torch.empty_like(fd)

    def solve():
        fsolve.fs_poisson_solve(plan, fd, ud)

    for _ in range(ctx["warmup"]):
        solve()
    torch.cuda.synchronize()
    l0 = fsolve.fs_kernel_launches()
    ms = _events_ms(torch, solve, reps, flush)
    launches = (fsolve.fs_kernel_launches() - l0) // reps
    kus = _kernel_us(fsolve, torch, solve, reps, flush)
    spec, real = _spec_bytes(n), n * n * 4
    ms_solve = statistics.mean(ms)
    passes = {"row_r2c": real + spec, "column": 2 * spec, "row_c2r": spec + real}
    per_pass = {k: {"us": round(kus[k][1], 3), "algorithmic_GBps": round(b / (kus[k][1] * 1e-6) / 1e9, 1),
                    "traffic": _capture_traffic("poisson_4096", k)} for k, b in passes.items() if k in kus}
    tr = [v["traffic"] for v in per_pass.values()]
    solve_traffic = sum(tr) if len(tr) == 3 and all(x is not None for x in tr) else None
    # plain path on the same GPU
    kx = 2 * math.pi * torch.fft.rfftfreq(n, d=1.0 / n, device=dev).double()
    ky = 2 * math.pi * torch.fft.fftfreq(n, d=1.0 / n, device=dev).double()
    w2 = ky[:, None] ** 2 + kx[None, :] ** 2
    w2[0, 0] = 1.0
    fac = (-1.0 / w2).float()
    fac[0, 0] = 0.0
    up = torch.empty_like(fd)

    def plain():
        up.copy_(torch.fft.irfft2(torch.fft.rfft2(fd) * fac, s=(n, n)))

    plain()
    ms_plain = statistics.mean(_events_ms(torch, plain, reps, flush))
    torch.cuda.synchronize()
    res = {
        "workload": "Poisson, periodic [0,1)^2, 4096x4096 FP32, 8-mode source |k|<=40, one solve per call",
        "value": round(1e3 / ms_solve, 2), "unit": "solves/s", "ms_per_solve": round(ms_solve, 5),
        "gpu_launches_per_solve": int(launches),
        "roofline": _roof(24 * n * n, ms_solve * 1e-3, ctx["peak"], ctx["peak_src"], solve_traffic,
                          what="24N^2 algorithmic bytes (3 passes) per solve / solve time", passes=per_pass),
        "plain_torch_fft": {"value": round(1e3 / ms_plain, 2), "unit": "solves/s", "ms_per_solve": round(ms_plain, 5),
                            "what": "torch.fft.rfft2 -> FP32 multiply by -1/|k|^2 -> irfft2 (cuFFT)"},
        "l2": "flushed between calls (256 MB write, untimed)",
    }
    ctx["checks"].append(("poisson_4096", "closed_form_poisson", modes, n, ud.cpu().numpy(), up.cpu().numpy()))
    fsolve.fs_plan_destroy(plan)
    return res


def leg_wave_4096_snapshots(ctx):
    """Wave u_tt = c^2 lap u on periodic [0,1)^2, 4096^2 FP32, c = 1: Gaussian
    pulse (width 0.02) + 0.01 N(0,1) noise, v0 = 0; one step = forward
    transform into the kept spectrum + 50 snapshots t = j/50 as one batch."""
    torch, fsolve, dev, flush, reps = ctx["torch"], ctx["fsolve"], ctx["dev"], ctx["flush"], ctx["reps"]
    from paper_2412_12308_gb300 import workloads as wl

    u0, (lx, ly), c, times, _ = wl.wave_pulse_4096()
    u0 = u0.astype(np.float32)
    n = u0.shape[0]
    plan = fsolve.fs_plan_create(n, n, lx, ly, fsolve.FS_F32)
    ud = torch.tensor(u0, device=dev)
    st = fsolve.fs_state_create(plan, ud)
    outs = torch.empty((len(times), n, n), dtype=torch.float32, device=dev)
    reqs = fsolve.fs_request_array([fsolve.fs_request(fsolve.FS_OP_WAVE_ADVANCE, state=st, out_u=outs[j], c=c,
                                                      t=float(t)) for j, t in enumerate(times)])

    def step():
        fsolve.fs_state_reset(st, ud)
        fsolve.fs_batch_submit(reqs)

    for _ in range(ctx["warmup"]):
        step()
    torch.cuda.synchronize()
    l0 = fsolve.fs_kernel_launches()
    ms = statistics.mean(_events_ms(torch, step, reps, flush))
    launches = (fsolve.fs_kernel_launches() - l0) // reps
    kus = _kernel_us(fsolve, torch, step, reps, flush)
    spec, real = _spec_bytes(n), n * n * 4
    dom = max(kus.items(), key=lambda kv: kv[1][0] * kv[1][1])
    # per step: the forward transform into the kept spectrum (16N^2) and 50
    # advances (16N^2 each: read the kept spectrum, write and read the work
    # spectrum, write u)
    step_bytes = (real + 3 * spec) * (len(times) + 1)
    res = {
        "workload": "wave, periodic [0,1)^2, 4096x4096 FP32, c=1, Gaussian pulse + white noise, v0=0, "
                    "1 forward + 50 snapshots t=j/50 per step",
        "value": round(len(times) / (ms / 1e3), 2), "unit": "snapshots/s", "ms_per_step": round(ms, 4),
        "gpu_launches_per_step": int(launches),
        "roofline": _roof(step_bytes, ms * 1e-3, ctx["peak"], ctx["peak_src"],
                          _capture_traffic("wave_4096_snapshots", dom[0]), kernel=dom[0],
                          what="algorithmic bytes per step (16N^2 per advance and for the forward transform) / "
                               "step time",
                          per_kernel_us={k: round(v[1], 3) for k, v in kus.items()}),
        "l2": "flushed between steps (256 MB write, untimed)",
    }
    j = len(times) - 1
    ctx["checks"].append(("wave_4096_snapshots", "oracle_wave", (u0, lx, ly, c, float(times[j])), n,
                          outs[j].cpu().numpy(), None))
    del outs
    fsolve.fs_state_destroy(st)
    fsolve.fs_plan_destroy(plan)
    return res


def leg_batch_mix_512(ctx):
    """512 independent problems (operator uniform over Poisson / diffusion /
    wave, N in {64, 80, ..., 2048}, 8-mode sources) in one persistent launch;
    with several ranks each runs its share (replicas.shard: LPT by grid
    points) and the time is the max over ranks."""
    torch, fsolve, dev, flush, reps = ctx["torch"], ctx["fsolve"], ctx["dev"], ctx["flush"], ctx["reps"]
    dist = ctx["dist"]
    from paper_2412_12308_gb300 import replicas, workloads as wl

    probs = wl.batch_mix()
    idx = replicas.my_share([replicas.problem_cost(p.n) for p in probs], dist.rank, dist.world)
    plans, ins, outs = {}, {}, {}
    for i in idx:
        p = probs[i]
        if p.n not in plans:
            plans[p.n] = fsolve.fs_plan_create(p.n, p.n, p.lx, p.ly, fsolve.FS_F32)
        ins[i] = torch.tensor(p.field(np.float32), device=dev)
        outs[i] = torch.empty_like(ins[i])
    arr, idx2 = replicas.batch_share_requests(probs, dist.rank, dist.world, plans, ins, outs)
    assert idx2 == idx

    def step():
        if arr is not None:
            fsolve.fs_batch_submit(arr)

    for _ in range(ctx["warmup"]):
        step()
    torch.cuda.synchronize()
    dist.barrier()
    l0 = fsolve.fs_kernel_launches()
    ms_local = statistics.mean(_events_ms(torch, step, reps, flush))
    launches = (fsolve.fs_kernel_launches() - l0) // reps
    ms = dist.max(ms_local)
    kus = _kernel_us(fsolve, torch, step, reps, flush)
    algo = sum(3 * (probs[i].n ** 2 * 4 + _spec_bytes(probs[i].n)) for i in idx)
    dom = max(kus.items(), key=lambda kv: kv[1][1]) if kus else ("batch", (0, 0.0))
    res = {
        "workload": "512 independent problems, op ~ U{Poisson, diffusion D~U[0.01,1], wave c~U[0.5,2]}, "
                    "N ~ U{64..2048: 2^k, 3*2^k, 5*2^k}, FP32, one persistent graph-captured launch per rank",
        "value": round(len(probs) / (ms / 1e3), 2), "unit": "solves/s", "ms_per_batch": round(ms, 4),
        "ranks": dist.world, "problems_this_rank": len(idx), "gpu_launches_per_batch": int(launches),
        "roofline": _roof(algo, dom[1][1] * 1e-6, ctx["peak"], ctx["peak_src"],
                          _capture_traffic("batch_mix_512", dom[0]), kernel=dom[0],
                          avg_launch_us=round(dom[1][1], 3),
                          what="sum over this rank's problems of 24N^2 (3-pass bytes) / batch launch time"),
        "scaling": "strong (the 512 problems are split across ranks)",
        "l2": "flushed between batches (256 MB write, untimed)",
    }
    sample = [i for i in idx if i % 8 == 0]
    ctx["checks"].append(("batch_mix_512", "closed_form_batch", [probs[i] for i in sample], None,
                          [outs[i].cpu().numpy() for i in sample], None))
    for h in plans.values():
        fsolve.fs_plan_destroy(h)
    return res


def leg_wave_advance_4096(ctx):
    """One wave advance per call from a kept 4096^2 FP32 spectrum (the pulse of
    the snapshot workload, t = 0.37): a column pass and a C2R pass per call.
    With FS_COLUMN_VARIANT=bf16x3 in the environment the column pass is the
    split-BF16 tensor-core variant."""
    torch, fsolve, dev, flush, reps = ctx["torch"], ctx["fsolve"], ctx["dev"], ctx["flush"], ctx["reps"]
    from paper_2412_12308_gb300 import workloads as wl

    u0, (lx, ly), c, _times, _ = wl.wave_pulse_4096()
    n = u0.shape[0]
    plan = fsolve.fs_plan_create(n, n, lx, ly, fsolve.FS_F32)
    ud = torch.tensor(u0.astype(np.float32), device=dev)
    st = fsolve.fs_state_create(plan, ud)
    out = torch.empty_like(ud)

    def adv():
        fsolve.fs_wave_advance(st, c, 0.37, out)

    for _ in range(ctx["warmup"]):
        adv()
    torch.cuda.synchronize()
    ms = statistics.mean(_events_ms(torch, adv, reps, flush))
    kus = _kernel_us(fsolve, torch, adv, reps, flush)
    res = {"workload": "wave advance from a kept 4096x4096 FP32 spectrum, one per call",
           "value": round(1e3 / ms, 2), "unit": "advances/s", "ms_per_advance": round(ms, 5),
           "column_variant": os.environ.get("FS_COLUMN_VARIANT", "fp32"),
           "roofline": _roof(16 * n * n, ms * 1e-3, ctx["peak"], ctx["peak_src"],
                             per_kernel_us={k: round(v[1], 3) for k, v in kus.items()})}
    fsolve.fs_state_destroy(st)
    fsolve.fs_plan_destroy(plan)
    return res


def leg_factors_4096(ctx):
    """Cost of the spectral factors on a 4096^2 half spectrum (8.4M elements):
    evaluated as the FP32 column pass does (two-float, hardware sine/cosine
    of the reduced phase) and in FP64 rounded once (fs_operator_factors, one
    float written per element, the same bytes both ways)."""
    torch, fsolve, dev, flush, reps = ctx["torch"], ctx["fsolve"], ctx["dev"], ctx["flush"], ctx["reps"]
    n = 4096
    plan = fsolve.fs_plan_create(n, n, 1.0, 1.0, fsolve.FS_F32)
    out = torch.empty((n // 2 + 1) * n, dtype=torch.float32, device=dev)
    res = {"workload": "operator factors of every half-spectrum element, 4096x4096 FP32 plan",
           "elements": (n // 2 + 1) * n}
    cases = (("poisson", fsolve.FS_OP_POISSON, {}), ("diffusion", fsolve.FS_OP_DIFFUSION, {"D": 0.1, "t": 0.5}),
             ("wave", fsolve.FS_OP_WAVE, {"c": 1.0, "t": 0.37}))
    for name, op, kw in cases:
        row = {}
        for fp64 in (False, True):
            def run():
                fsolve.fs_operator_factors(plan, op, out, fp64=fp64, **kw)
            run()
            row["fp64_us" if fp64 else "two_float_us"] = round(1e3 * statistics.mean(_events_ms(torch, run, reps, flush)), 3)
        res[name] = row
    fsolve.fs_plan_destroy(plan)
    return res


LEG_FNS = {"factors_4096": leg_factors_4096, "poisson_4096": leg_poisson_4096,
           "wave_4096_snapshots": leg_wave_4096_snapshots,
           "batch_mix_512": leg_batch_mix_512, "wave_advance_4096": leg_wave_advance_4096}


def leg_accuracy(checks):
    """rel-L2 of each leg's sampled outputs against the float64 oracle or the
    exact closed forms (part of the CPU-baseline leg: the only place here that
    runs oracle code)."""
    import oracle
    from oracle import closed_forms as cf

    out = {}
    for leg, kind, data, n, got, extra in checks:
        t0 = time.perf_counter()
        if kind == "closed_form_poisson":
            want = cf.poisson_modes(data, n, n, 1.0, 1.0)
            r = {"rel_l2_vs_closed_form": float(np.linalg.norm(got - want) / np.linalg.norm(want)),
                 "plain_torch_fft_rel_l2_vs_closed_form": float(np.linalg.norm(extra - want) / np.linalg.norm(want))}
        elif kind == "oracle_wave":
            u0, lx, ly, c, t = data
            U, _ = oracle.wave_spectrum(oracle.state_spectrum(u0.astype(np.float64)), None, c, t, lx, ly)
            want = np.real(oracle.idft2(U))
            r = {"rel_l2_vs_oracle": float(np.linalg.norm(got - want) / np.linalg.norm(want)), "t": t}
        else:  # batch mix sample
            worst = 0.0
            for p, g in zip(data, got):
                if p.op == "poisson":
                    want = cf.poisson_modes(p.modes, p.n, p.n, p.lx, p.ly)
                    den = np.linalg.norm(want)
                elif p.op == "diffusion":
                    want = cf.diffusion_modes(p.modes, p.D, p.t, p.n, p.n, p.lx, p.ly)
                    den = max(np.linalg.norm(want), np.linalg.norm(p.field(np.float32).astype(np.float64)))
                else:
                    want = cf.wave_modes(p.modes, p.c, p.t, p.n, p.n, p.lx, p.ly)
                    den = np.linalg.norm(want)
                worst = max(worst, float(np.linalg.norm(g - want) / den))
            r = {"rel_l2_vs_closed_form_max": worst, "problems_checked": len(data)}
        r["check_seconds"] = round(time.perf_counter() - t0, 2)
        out[leg] = r
    return out


def run_ours(args, dist):
    import torch

    from paper_2412_12308_gb300 import fsolve

    torch.cuda.set_device(dist.local)
    dist.init("nccl")
    fsolve.load()
    dev = torch.device("cuda", dist.local)
    peak, peak_src = peaks()
    ctx = {"torch": torch, "fsolve": fsolve, "dev": dev, "dist": dist, "reps": max(3, args.steps),
           "warmup": args.warmup, "peak": peak, "peak_src": peak_src, "checks": [],
           "flush": torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)}
    if args.leg:
        # one workload alone (profiling runs): its JSON only
        res = LEG_FNS[args.leg](ctx)
        if dist.rank == 0:
            print(json.dumps({"leg": args.leg, **res}), flush=True)
        dist.close()
        return
    u0, blobs, lx, ly, D, times = workload()
    plan = fsolve.fs_plan_create(N, N, lx, ly, fsolve.FS_F32)
    u0d = torch.tensor(u0, device=dev)
    out = torch.empty((len(times), N, N), dtype=torch.float32, device=dev)
    state = fsolve.fs_state_create(plan, u0d)
    flush = ctx["flush"]  # 256 MB > L2
    ts = [float(t) for t in times]
    reqs = fsolve.fs_request_array([fsolve.fs_request(fsolve.FS_OP_DIFFUSION_ADVANCE, state=state, out_u=out[j],
                                                      D=D, t=t) for j, t in enumerate(ts)])

    def step(src):
        # one forward transform into the kept spectrum, then all 100 advances
        # as one persistent batch launch
        fsolve.fs_state_reset(state, src)
        fsolve.fs_batch_submit(reqs)

    def step_percall(src):
        fsolve.fs_state_reset(state, src)
        for j, t in enumerate(ts):
            fsolve.fs_diffusion_advance(state, D, t, out[j])

    for _ in range(args.warmup):
        step(u0d)
    torch.cuda.synchronize()

    # ---- timed region: K steps, L2 flushed between steps (untimed)
    clocks = Clocks(dist.local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    l0 = fsolve.fs_kernel_launches()
    host_s = 0.0
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record()
        h0 = time.perf_counter()
        step(u0d)
        host_s += time.perf_counter() - h0
        ev[k][1].record()
    torch.cuda.synchronize()
    launches = (fsolve.fs_kernel_launches() - l0) // max(1, args.steps)
    clk = clocks.stop()
    dist.barrier()
    total_ms = sum(a.elapsed_time(b) for a, b in ev)
    total_ms = dist.max(total_ms)
    ms_per_step = total_ms / args.steps
    value = dist.world * len(ts) * args.steps / (total_ms / 1e3)

    # ---- per-kernel device time (library events on the launching stream), same steps
    fsolve.fs_profile_enable(True)
    for _ in range(args.steps):
        flush.zero_()
        step(u0d)
    torch.cuda.synchronize()
    prof = fsolve.fs_profile_report()
    fsolve.fs_profile_enable(False)
    dom = max(prof.items(), key=lambda kv: kv[1][1])
    name, (cnt, tot) = dom
    avg_s = tot / max(1, cnt) / 1e3
    M = N // 2
    spec_bytes = (M + 1) * N * 8
    # algorithmic bytes per launch (FP32): column advance reads the kept
    # spectrum and writes the work spectrum; C2R reads the work spectrum and
    # writes the real field; R2C reads the field and writes the spectrum.
    # the batch launch runs all 100 advances: per advance 16N^2 (read kept
    # spectrum, write + read the work spectrum, write u)
    algo = {"column": 2 * spec_bytes, "row_c2r": spec_bytes + N * N * 4, "row_r2c": N * N * 4 + spec_bytes,
            "factor": (M + 1 + N) * 16,
            "batch": len(ts) * (3 * spec_bytes + N * N * 4)}.get(name, 0)
    achieved = algo / avg_s / 1e9 if avg_s > 0 else 0.0
    traffic = _capture_traffic("diffusion_1024", name)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic, "kernel": name,
                "peak_source": peak_src, "avg_launch_us": round(avg_s * 1e6, 3),
                "algorithmic_bytes_per_launch": algo,
                "per_kernel_ms": {k: round(v[1] / max(1, v[0]), 5) for k, v in prof.items() if v[0]}}

    # ---- end to end through the C ABI with host buffers (pinned): each step
    # copies u0 host -> device, forms the kept spectrum, and the batch's C2R
    # units store the 100 outputs straight into the pinned host array (mapped
    # into the GPU's address space; the stores cross NVLink-C2C while the
    # batch computes).  Measured on GB300: the same step with the outputs in
    # device memory, copied back by the copy engine chunk by chunk (25
    # advances per batch) behind the compute, took 2.40 vs 2.34 ms: the host
    # link moves ~180 GB/s either way.
    h_u0 = torch.from_numpy(u0).pin_memory()
    h_out = torch.empty((len(ts), N, N), dtype=torch.float32).pin_memory()
    reqs_host = fsolve.fs_request_array([fsolve.fs_request(fsolve.FS_OP_DIFFUSION_ADVANCE, state=state,
                                                           out_u=h_out[j].data_ptr(), D=D, t=t)
                                         for j, t in enumerate(ts)])
    e2e_ms = []
    for k in range(max(3, args.steps // 2) + 2):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        u0d.copy_(h_u0, non_blocking=True)
        fsolve.fs_state_reset(state, u0d)
        fsolve.fs_batch_submit(reqs_host)
        b.record()
        torch.cuda.synchronize()
        if k >= 2:  # the first two build the host-output batch's graphs
            e2e_ms.append(a.elapsed_time(b))
    e2e_step = dist.max(statistics.median(e2e_ms))
    e2e = {"value": dist.world * len(ts) / (e2e_step / 1e3), "unit": "solves/s",
           "h2d_bytes_per_step": int(u0.nbytes), "d2h_bytes_per_step": int(len(ts) * N * N * 4),
           "d2h": "outputs stored by the kernels into pinned host memory"}

    # ---- comparators on the same GPU: this library one call per solve, and the
    # plain torch.fft path (rfft2 -> FP32 multiply -> irfft2, separate launches)
    def timed(fn, reps):
        ms = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return statistics.median(ms)

    step_percall(u0d)
    pc_ms = timed(lambda: step_percall(u0d), max(3, args.steps // 2))
    kx = 2 * math.pi * torch.fft.rfftfreq(N, d=lx / N, device=dev).double()
    ky = 2 * math.pi * torch.fft.fftfreq(N, d=ly / N, device=dev).double()
    w2 = (ky[:, None] ** 2 + kx[None, :] ** 2)
    facs = [torch.exp(-D * t * w2).float() for t in ts]

    def step_torch():
        for j in range(len(ts)):
            out[j] = torch.fft.irfft2(torch.fft.rfft2(u0d) * facs[j], s=(N, N))

    step_torch()
    tf_ms = timed(step_torch, max(3, args.steps // 2))
    comparators = {
        "library_one_call_per_solve": {"value": round(len(ts) / (pc_ms / 1e3), 2), "unit": "solves/s",
                                       "ms_per_step": round(pc_ms, 4)},
        "torch_fft_per_solve": {"value": round(len(ts) / (tf_ms / 1e3), 2), "unit": "solves/s",
                                "ms_per_step": round(tf_ms, 4),
                                "what": "torch.fft.rfft2 -> multiply by FP32 exp(-D|k|^2 t) -> irfft2 per output (cuFFT)"},
    }

    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "solves/s", "n_gpus": dist.world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded Gaussian blobs)",
        "config": {"workload": WORKLOAD, "grid": [N, N], "solves_per_step": len(ts),
                   "l2": "flushed between steps (256 MB write, untimed)",
                   "parallelism": f"replicas x{dist.world}"},
        "e2e": e2e, "roofline": roofline, "gpu_launches": int(launches), "clocks": clk,
        "host_us_per_step": round(1e6 * host_s / args.steps, 1),
        "comparators": comparators,
    }
    legs = [x for x in args.legs.split(",") if x]
    if legs:
        line["legs"] = {}
        for name in legs:
            line["legs"][name] = LEG_FNS[name](ctx)
    if not args.no_serving:
        # open-loop serving: 20,000 requests, N log-uniform in [128, 8192],
        # mixed operators with follow-ups, 150 GB budget, arrival rate 0.8 x
        # the plain per-call path's saturated throughput on the same mix
        from paper_2412_12308_gb300 import servebench

        line["serving"] = servebench.run(n_requests=args.serve_requests, load=0.8)
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        gpu_out = out.cpu().numpy()
        line["cpu_baseline"] = cpu_baseline(u0, lx, ly, D, times, gpu_out)
        line["rel_l2_vs_oracle_max"] = line["cpu_baseline"].pop("rel_l2_vs_oracle_max", None)
        for name, acc in leg_accuracy(ctx["checks"]).items():
            line["legs"][name]["accuracy"] = acc
    fsolve.fs_state_destroy(state)
    fsolve.fs_plan_destroy(plan)
    if dist.rank == 0:
        print(json.dumps(line), flush=True)
    dist.close()


# ----------------------------------------------------------------------------- reference
def run_reference(args, dist):
    if dist.rank != 0:
        return
    u0, blobs, lx, ly, D, times = workload()
    samples = []
    for k in range(args.warmup + args.steps):
        r = cpu_baseline(u0, lx, ly, D, times, None)
        if k >= args.warmup:
            samples.append(r)
    step_s = [len(times) / r["value"] for r in samples]
    ms = 1e3 * sum(step_s) / len(step_s)
    value = len(times) / (ms / 1e3)
    line = {
        "metric": METRIC, "value": round(value, 4), "unit": "solves/s", "n_gpus": dist.world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded Gaussian blobs)", "impl": "reference",
        "config": {"workload": WORKLOAD, "grid": [N, N], "solves_per_step": len(times),
                   "parallelism": "host cores"},
        "cpu_baseline": {"value": round(value, 4), "unit": "solves/s", "cores": os.cpu_count(),
                         "kind": "oracle", "sample": samples[0]["sample"]},
        "e2e": {"value": round(value, 4), "unit": "solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    dist = Dist()
    if args.impl == "reference":
        run_reference(args, dist)
    else:
        run_ours(args, dist)


if __name__ == "__main__":
    main()
