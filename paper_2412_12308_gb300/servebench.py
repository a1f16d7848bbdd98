"""Open-loop serving measurement (CUDA path only).

Stream (workloads.serve_stream): N log-uniform in [128, 8192] snapped to a
supported size, operators uniform over {Poisson, diffusion, wave}; every
diffusion / wave request keeps its spectrum and is followed, after an
exponential delay (mean 10 ms), by one advance to a later time on that
spectrum.  Exponential inter-arrival gaps; the rate is `load` times the
saturated throughput of the plain path on the same mix (its capacity: the
requests divided by the sum of their per-call service times, measured with
CUDA events).

Plain path, run for real: one host thread takes the requests in arrival
order, waits for each arrival, runs it through the per-call entry points on
one stream (solve; or kept-state reset + advance; follow-up = advance) and
synchronises before taking the next.  One kept state per grid size stands in
for each parent's own (the same work per call).  Latency = arrival -> the
synchronise returning.

Served path: fs_serve_replay enqueues each request at its arrival time; the
server batches whatever is queued whenever one of its in-flight slots frees.
Latency = enqueue -> observed completion (fs_serve_latency).

`sweep` runs both paths at several loads (fractions of the plain capacity);
above 1.0 the plain path saturates and its throughput is its capacity.
"""

import time

import numpy as np


def _percentiles(x):
    x = np.asarray(x, dtype=np.float64)
    return {"p50_us": float(np.percentile(x, 50)), "p99_us": float(np.percentile(x, 99)),
            "mean_us": float(x.mean())}


def _items(base, service, load):
    """Initial requests and follow-ups with arrivals scaled so the offered load
    is `load` x the plain path's capacity; sorted by arrival.  Also returns
    the plain capacity (requests/s)."""
    items = []  # [arrival, kind, n, D, c, t, parent_key, key]
    for r in base:
        p = r.problem
        items.append([r.arrival_s, p.op, p.n, p.D, p.c, p.t, None, ("a", r.rid)])
        if r.followup_t >= 0:
            items.append([r.arrival_s + r.followup_delay_s, p.op + "_adv", p.n, p.D, p.c, r.followup_t,
                          ("a", r.rid), ("f", r.rid)])
    n_total = len(items)
    plain_rate = n_total / sum(service[(it[2], it[1])] for it in items)
    span = max(r.arrival_s for r in base)
    scale = (n_total / (load * plain_rate)) / span
    for it in items:
        it[0] *= scale
    items.sort(key=lambda it: it[0])
    return items, plain_rate


def _by_size(items, served, plain):
    out = {}
    sizes_arr = np.array([it[2] for it in items])
    s_arr, p_arr = np.asarray(served, dtype=np.float64), np.asarray(plain, dtype=np.float64)
    for lo, hi in ((0, 1024), (1025, 4096), (4097, 8192)):
        m = (sizes_arr >= lo) & (sizes_arr <= hi)
        if m.any():
            out[f"N{lo}-{hi}"] = {"count": int(m.sum()), "served": _percentiles(s_arr[m]),
                                  "plain": _percentiles(p_arr[m])}
    return out


def run(n_requests=20000, load=0.8, seed=12312, budget_bytes=150 << 30, slots=3, max_batch=32,
        nmin=128, nmax=8192, pool=3, verbose=False, sweep=(0.5, 1.0, 1.2), sweep_requests=6000):
    """The served and the plain path at `load` on `n_requests` initial
    requests, and (unless `sweep` is empty) at each load of `sweep` on
    `sweep_requests` initial requests of the same stream."""
    import torch

    from . import fsolve as fs
    from . import workloads as wl

    fs.load()
    base = wl.serve_stream(1.0, seed=seed, count=n_requests, nmin=nmin, nmax=nmax)
    sizes = sorted({r.problem.n for r in base})
    plans, inputs, outs, states = {}, {}, {}, {}
    rng = np.random.default_rng(seed)
    for n in sizes:
        plans[n] = fs.fs_plan_create(n, n, 1.0, 1.0, fs.FS_F32)
        f = wl.mode_sum(wl.draw_modes(rng, 8, min(16, n // 2 - 1)), n, n, 1.0, 1.0).astype(np.float32)
        inputs[n] = torch.tensor(f, device="cuda")
        outs[n] = [torch.empty_like(inputs[n]) for _ in range(pool)]
        states[n] = fs.fs_state_create(plans[n], inputs[n])
    ops = {"poisson": fs.FS_OP_POISSON, "diffusion": fs.FS_OP_DIFFUSION, "wave": fs.FS_OP_WAVE}

    # ---- plain path: the per-call entry points, one request at a time
    def plain_call(n, kind, out, t=0.3):
        if kind == "poisson":
            fs.fs_poisson_solve(plans[n], inputs[n], out)
        elif kind in ("diffusion", "wave"):  # first request: forward into the kept state + advance
            fs.fs_state_reset(states[n], inputs[n])
            if kind == "diffusion":
                fs.fs_diffusion_advance(states[n], 0.1, t, out)
            else:
                fs.fs_wave_advance(states[n], 1.0, t, out)
        elif kind == "diffusion_adv":
            fs.fs_diffusion_advance(states[n], 0.1, t, out)
        else:
            fs.fs_wave_advance(states[n], 1.0, t, out)

    service = {}
    for n in sizes:
        for kind in ("poisson", "diffusion", "wave", "diffusion_adv", "wave_adv"):
            for _ in range(2):
                plain_call(n, kind, outs[n][0])
            torch.cuda.synchronize()
            reps = 5 if n >= 4096 else 10
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps):
                plain_call(n, kind, outs[n][0])
            b.record()
            torch.cuda.synchronize()
            service[(n, kind)] = a.elapsed_time(b) / reps / 1e3  # seconds

    def plain_run(items):
        """Open loop, one request at a time: wait for the arrival, run, synchronise."""
        lat = []
        counters = {n: 0 for n in sizes}
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for it in items:
            arrival, kind, n, D, c, t = it[:6]
            due = t0 + arrival
            while time.perf_counter() < due:
                pass
            out = outs[n][counters[n] % pool]
            counters[n] += 1
            plain_call(n, kind, out, t)
            torch.cuda.synchronize()
            lat.append((time.perf_counter() - due) * 1e6)
        return lat, time.perf_counter() - (t0 + items[0][0])

    def served_run(items):
        index = {it[7]: i for i, it in enumerate(items)}
        reqs = []
        counters = {n: 0 for n in sizes}
        for it in items:
            arrival, kind, n, D, c, t, parent, key = it
            out = outs[n][counters[n] % pool]
            counters[n] += 1
            if kind.endswith("_adv"):
                op = fs.FS_OP_DIFFUSION_ADVANCE if kind.startswith("diffusion") else fs.FS_OP_WAVE_ADVANCE
                reqs.append(fs.fs_request(op, out_u=out, D=D, c=c, t=t, parent=index[parent] + 1))
            else:
                keep = 0 if kind == "poisson" else 1
                reqs.append(fs.fs_request(ops[kind], plan=plans[n], in_u=inputs[n], out_u=out, D=D, c=c, t=t,
                                          keep=keep))
        arrivals = [it[0] for it in items]
        fs.fs_serve_start(budget_bytes, slots=slots, max_batch=max_batch)
        try:
            t0 = time.perf_counter()
            tickets = fs.fs_serve_replay(reqs, arrivals)
            pending = set(tickets)
            while pending:
                for tk in fs.fs_serve_poll(8192, 200_000):
                    pending.discard(tk)
                if time.perf_counter() - t0 > 600:
                    raise RuntimeError(f"serving: {len(pending)} requests unfinished after 600 s")
            makespan = time.perf_counter() - t0 - arrivals[0]
            lat = [fs.fs_serve_latency(tk) for tk in tickets]
            stats = fs.fs_serve_stats()
        finally:
            fs.fs_serve_stop()
        return lat, makespan, stats

    def one(base_k, ld):
        items, plain_rate = _items(base_k, service, ld)
        s_lat, s_span, stats = served_run(items)
        p_lat, p_span = plain_run(items)
        n_total = len(items)
        return items, {
            "load": ld, "requests": n_total, "initial_requests": len(base_k),
            "rate_per_s": n_total / (items[-1][0] - items[0][0]),
            "served": {"solves_per_s": n_total / s_span, **_percentiles(s_lat), "batches": stats["batches"],
                       "max_in_flight": stats["max_in_flight"], "peak_hbm_bytes": stats["peak_bytes"]},
            "plain_path": {"capacity_solves_per_s": plain_rate, "solves_per_s": n_total / p_span,
                           **_percentiles(p_lat)},
        }, s_lat, p_lat

    try:
        items, res, s_lat, p_lat = one(base, load)
        res["by_size"] = _by_size(items, s_lat, p_lat)
        res["plain_path"]["what"] = ("open loop, one request at a time through the per-call entry points, "
                                     "synchronised after each")
        res.update({"budget_bytes": budget_bytes, "slots": slots, "max_batch": max_batch,
                    "sizes": [int(n) for n in sizes]})
        if sweep:
            res["sweep"] = []
            for ld in sweep:
                _, r, _, _ = one(base[:sweep_requests], ld)
                res["sweep"].append(r)
    finally:
        for n in sizes:
            fs.fs_state_destroy(states[n])
            fs.fs_plan_destroy(plans[n])
    if verbose:
        print(res)
    return res


if __name__ == "__main__":
    import argparse
    import json

    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=20000)
    ap.add_argument("--load", type=float, default=0.8)
    ap.add_argument("--budget-gb", type=float, default=150.0)
    ap.add_argument("--slots", type=int, default=3)
    ap.add_argument("--max-batch", type=int, default=32)
    a = ap.parse_args()
    print(json.dumps(run(a.requests, a.load, budget_bytes=int(a.budget_gb * (1 << 30)), slots=a.slots,
                         max_batch=a.max_batch)))
