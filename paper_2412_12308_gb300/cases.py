"""Named solver workloads for timing and profiling (CUDA path only).

    python -m paper_2412_12308_gb300.cases poisson --n 4096 --iters 20
    python -m paper_2412_12308_gb300.cases wave_adv --n 4096 --iters 20
    python -m paper_2412_12308_gb300.cases diffusion_batch --n 1024 --iters 5
    python -m paper_2412_12308_gb300.cases batch_mix --iters 5
    python -m paper_2412_12308_gb300.cases wave_snapshots --n 4096 --iters 5
    python -m paper_2412_12308_gb300.cases wave_src_adv --n 4096 --iters 20

Each case runs `--warmup` untimed repetitions, then `--iters` timed ones
(CUDA events on the current stream) and prints one JSON line with the mean
time per repetition, the per-kernel averages from the library's event
profiler and the algorithmic HBM bytes per repetition.  Inputs are seeded
synthetic fields (workloads.py); no result is checked here (the tests do
that).  Used for ncu captures: pick kernels with `-k regex:...`.
"""

import argparse
import json

import numpy as np


def _setup(n, dtype, lx=1.0):
    import torch

    from . import fsolve, workloads

    fsolve.load()
    rng = np.random.default_rng(n)
    f = workloads.mode_sum(workloads.draw_modes(rng, 8, 16), n, n, lx, lx)
    tdt = torch.float32 if dtype == fsolve.FS_F32 else torch.float64
    fd = torch.tensor(f, dtype=tdt, device="cuda")
    plan = fsolve.fs_plan_create(n, n, lx, lx, dtype)
    return fsolve, plan, fd


def run(case, n, iters, warmup, dtype=0, profile=True):
    import torch

    from . import fsolve as fs

    fsolve, plan, fd = _setup(n, dtype)
    out = torch.empty_like(fd)
    esz = fd.element_size()
    spec = (n // 2 + 1) * n * 2 * esz
    real = n * n * esz
    state = None
    extra = {}
    if case == "poisson":
        def rep():
            fsolve.fs_poisson_solve(plan, fd, out)
        algo = 3 * (real + spec)  # three passes: R2C, column, C2R
    elif case == "poisson_c":
        # complex field, full spectrum: rows C2C, columns, inverse rows C2C
        fc = torch.complex(fd, torch.flip(fd, (0,))).contiguous()
        outc = torch.empty_like(fc)

        def rep():
            fsolve.fs_poisson_solve_c(plan, fc, outc)
        algo = 3 * 2 * n * n * 2 * esz
    elif case == "wave_solve":
        def rep():
            fsolve.fs_wave_solve(plan, fd, None, 1.0, 0.37, out)
        algo = 3 * (real + spec)
    elif case == "wave_solve_v0":
        # initial velocity: two row transforms, two-field column pass
        gd = torch.flip(fd, (1,)).contiguous()

        def rep():
            fsolve.fs_wave_solve(plan, fd, gd, 1.0, 0.37, out)
        algo = 2 * (real + spec) + 3 * spec + spec + real
    elif case == "wave_adv_v":
        # advance with the velocity output: two inverse column transforms, two C2R fields
        state = fsolve.fs_state_create(plan, fd)
        vout = torch.empty_like(out)

        def rep():
            fsolve.fs_wave_advance(state, 1.0, 0.37, out, vout)
        algo = spec + 2 * spec + 2 * (spec + real)
    elif case == "wave_adv":
        state = fsolve.fs_state_create(plan, fd)

        def rep():
            fsolve.fs_wave_advance(state, 1.0, 0.37, out)
        algo = 2 * spec + spec + real  # column (read kept, write work) + C2R
    elif case == "diffusion_adv":
        state = fsolve.fs_state_create(plan, fd)

        def rep():
            fsolve.fs_diffusion_advance(state, 0.1, 0.37, out)
        algo = 2 * spec + spec + real
    elif case in ("diffusion_src_adv", "wave_src_adv"):
        # advance with a constant source: the column pass also reads the kept
        # source spectrum
        state = fsolve.fs_state_create(plan, fd)
        fsolve.fs_state_set_source(state, fd)
        if case == "diffusion_src_adv":
            def rep():
                fsolve.fs_diffusion_advance(state, 0.1, 0.37, out)
        else:
            def rep():
                fsolve.fs_wave_advance(state, 1.0, 0.37, out)
        algo = 3 * spec + spec + real
    elif case == "wave_rk4":
        # RK4 with the orbiting source (A = 1, sigma = 0.1, Omega = 5, gamma = 10,
        # [-2, 2]^2, dt = h/4): one repetition = `rk4_steps` steps (one graph
        # replay); N = 256 with 640 steps is the paper's run to t = 2.5
        from .workloads import OrbitSource

        plan_rk = fs.fs_plan_create(n, n, 4.0, 4.0, dtype)
        rk = fs.fs_rk4_create(plan_rk, 1.0, OrbitSource())
        dt = 0.25 * 4.0 / n
        nst = 640 if n <= 256 else 20

        def rep():
            fsolve.fs_rk4_step(rk, dt, nst)
        chunks = -(-nst // 128)
        # per chunk: U, V read and written once, plus the 1D source tables
        algo = chunks * 4 * spec + (2 * nst + chunks) * (n // 2 + 1 + n) * 2 * esz
        extra["rk4_steps_per_rep"] = nst
        extra["modes"] = (n // 2 + 1) * n
        extra["dt"] = dt
        extra["_rk4"] = (rk, plan_rk)
    elif case == "batch_mix":
        # 512 uneven problems (N in {64..2048}, all three operators) in one
        # persistent launch per repetition
        probs = workloads_batch_mix()
        bplans, ins, outs_b = {}, [], []
        for pr in probs:
            if pr.n not in bplans:
                bplans[pr.n] = fs.fs_plan_create(pr.n, pr.n, pr.lx, pr.ly, fs.FS_F32)
            ins.append(torch.tensor(pr.field(np.float32), device="cuda"))
            outs_b.append(torch.empty_like(ins[-1]))
        ops = {"poisson": fs.FS_OP_POISSON, "diffusion": fs.FS_OP_DIFFUSION, "wave": fs.FS_OP_WAVE}
        reqs = [fs.fs_request(ops[pr.op], plan=bplans[pr.n], in_u=ins[i], out_u=outs_b[i], D=pr.D, c=pr.c, t=pr.t)
                for i, pr in enumerate(probs)]

        def rep():
            fsolve.fs_batch_submit(reqs)
        pts = sum(pr.n * pr.n for pr in probs)
        algo = sum(3 * (pr.n * pr.n * 4 + (pr.n // 2 + 1) * pr.n * 8) for pr in probs)
        extra["solves_per_rep"] = len(probs)
        extra["mean_points"] = pts / len(probs)
        extra["_cleanup"] = bplans
    elif case == "wave_snapshots":
        # 1 forward transform into the kept spectrum + 50 snapshots t = j/50
        nt = 50
        state = fsolve.fs_state_create(plan, fd)
        outs = torch.empty((nt, n, n), dtype=fd.dtype, device="cuda")
        reqs = [fs.fs_request(fs.FS_OP_WAVE_ADVANCE, state=state, out_u=outs[j], c=1.0, t=(j + 1) / nt)
                for j in range(nt)]

        def rep():
            fsolve.fs_state_reset(state, fd)
            fsolve.fs_batch_submit(reqs)
        algo = (real + 2 * spec) + nt * (3 * spec + real)
        extra["solves_per_rep"] = nt
    elif case == "diffusion_batch":
        nt = 100
        state = fsolve.fs_state_create(plan, fd)
        outs = torch.empty((nt, n, n), dtype=fd.dtype, device="cuda")
        reqs = [fs.fs_request(fs.FS_OP_DIFFUSION_ADVANCE, state=state, out_u=outs[j], D=0.1, t=j / (nt - 1))
                for j in range(nt)]

        def rep():
            fsolve.fs_state_reset(state, fd)
            fsolve.fs_batch_submit(reqs)
        algo = (real + 2 * spec) + nt * (3 * spec + real)
        extra["solves_per_rep"] = nt
    else:
        raise SystemExit(f"unknown case {case}")
    for _ in range(warmup):
        rep()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(iters):
        rep()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / iters
    res = {"case": case, "n": n, "dtype": dtype, "iters": iters, "ms_per_rep": round(ms, 5),
           "algorithmic_bytes": algo, "algorithmic_GBps": round(algo / (ms / 1e3) / 1e9, 1)}
    cleanup = extra.pop("_cleanup", None)
    rk4 = extra.pop("_rk4", None)
    res.update(extra)
    if rk4 is not None:
        res["us_per_rk4_step"] = round(1e3 * ms / extra["rk4_steps_per_rep"], 3)
        res["rk4_steps_per_s"] = round(extra["rk4_steps_per_rep"] / (ms / 1e3), 1)
        res["mode_steps_per_s"] = round(extra["modes"] * extra["rk4_steps_per_rep"] / (ms / 1e3), 1)
    if "solves_per_rep" in extra:
        res["solves_per_s"] = round(extra["solves_per_rep"] / (ms / 1e3), 1)
    if profile:
        fsolve.fs_profile_enable(True)
        for _ in range(iters):
            rep()
        torch.cuda.synchronize()
        prof = fsolve.fs_profile_report()
        fsolve.fs_profile_enable(False)
        res["per_kernel_us"] = {k: round(1e3 * v[1] / v[0], 3) for k, v in prof.items() if v[0]}
    if state is not None:
        fsolve.fs_state_destroy(state)
    if rk4 is not None:
        fsolve.fs_rk4_destroy(rk4[0])
        fsolve.fs_plan_destroy(rk4[1])
    for h in (cleanup or {}).values():
        fsolve.fs_plan_destroy(h)
    fsolve.fs_plan_destroy(plan)
    return res


def workloads_batch_mix():
    from . import workloads

    return workloads.batch_mix()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case")
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--iters", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--f64", action="store_true")
    ap.add_argument("--no-profile", action="store_true")
    ap.add_argument("--tune", action="store_true", help="autotune every grid of the case first (fs_tune)")
    a = ap.parse_args()
    if a.tune:
        from . import fsolve, workloads

        fsolve.load()
        if a.case == "batch_mix":  # the batch's own tuning, per grid of the mix
            for n in sorted({p.n for p in workloads.batch_mix()}):
                if n * n > 256 * 256:  # smaller grids run as single-CTA problems
                    fsolve.fs_tune_batch(n, n, 1.0, 1.0, 0, nprob=8, reps=3)
        else:
            fsolve.fs_tune(a.n, a.n, 1.0, 1.0, 1 if a.f64 else 0, reps=5)
    print(json.dumps(run(a.case, a.n, a.iters, a.warmup, 1 if a.f64 else 0, not a.no_profile)))


if __name__ == "__main__":
    main()
