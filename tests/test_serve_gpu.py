"""Serving loop on the GPU: continuous batching, kept spectra, admission.

* every request's result is the same alone and in an overlapping open-loop
  mix (bit for bit: a request's units do not depend on the batch around it);
* follow-up requests advance the spectrum kept by their parent;
* results match the float64 oracle;
* a tight HBM budget admits requests as memory frees up (no deadlock) and
  never exceeds the budget; batches overlap on the device;
* requests that can never fit, or that name a spectrum nobody keeps, are
  rejected on the host.
"""

import numpy as np
import pytest
import torch

import oracle
from paper_2412_12308_gb300 import fsolve, workloads as wl

pytestmark = pytest.mark.gpu

OPS = {"poisson": fsolve.FS_OP_POISSON, "diffusion": fsolve.FS_OP_DIFFUSION, "wave": fsolve.FS_OP_WAVE}


class Stream:
    """Seeded request stream with device buffers (each request its own output)."""

    def __init__(self, count, sizes, seed, explicit=False):
        rng = np.random.default_rng(seed)
        self.plans, self.items = {}, []
        for i in range(count):
            n = int(sizes[i % len(sizes)]) if explicit else int(sizes[int(rng.integers(0, len(sizes)))])
            op = ("poisson", "diffusion", "wave")[int(rng.integers(0, 3))]
            p = wl.Problem(op=op, n=n, modes=wl.draw_modes(rng, 8, min(16, n // 2 - 1)))
            if op == "diffusion":
                p.D, p.t = float(rng.uniform(0.001, 0.05)), float(rng.uniform(0.0, 1.0))
            elif op == "wave":
                p.c, p.t = float(rng.uniform(0.5, 2.0)), float(rng.uniform(0.0, 1.0))
            if n not in self.plans:
                self.plans[n] = fsolve.fs_plan_create(n, n, 1.0, 1.0, fsolve.FS_F32)
            f = torch.tensor(p.field(np.float32), device="cuda")
            item = {"p": p, "f": f, "out": torch.empty_like(f), "follow": None}
            if op != "poisson":
                item["t2"] = p.t + float(rng.uniform(0.0, 0.5))
                item["follow"] = torch.empty_like(f)
            self.items.append(item)

    def requests(self):
        """Requests in order; a follow-up right after its parent (parent = index + 1)."""
        reqs, where = [], []
        for it in self.items:
            p = it["p"]
            keep = 1 if it["follow"] is not None else 0
            reqs.append(fsolve.fs_request(OPS[p.op], plan=self.plans[p.n], in_u=it["f"], out_u=it["out"], D=p.D,
                                          c=p.c, t=p.t, keep=keep))
            where.append((it, "out"))
            if keep:
                op = fsolve.FS_OP_DIFFUSION_ADVANCE if p.op == "diffusion" else fsolve.FS_OP_WAVE_ADVANCE
                reqs.append(fsolve.fs_request(op, out_u=it["follow"], D=p.D, c=p.c, t=it["t2"],
                                              parent=len(reqs)))  # parent index + 1
                where.append((it, "follow"))
        return reqs, where

    def close(self):
        for h in self.plans.values():
            fsolve.fs_plan_destroy(h)


def _drain(tickets, timeout_s=60.0):
    import time

    pending = set(tickets)
    t0 = time.time()
    while pending:
        for t in fsolve.fs_serve_poll(4096, 100_000):
            pending.discard(t)
        assert time.time() - t0 < timeout_s, f"{len(pending)} requests did not finish"


def _snapshot(items):
    return [(it["out"].clone(), None if it["follow"] is None else it["follow"].clone()) for it in items]


def _alone_vs_mix(S, budget, slots, max_batch, window_s):
    """Each request alone on an idle server, then all of them in an open-loop
    mix arriving within `window_s`: identical results bit for bit."""
    reqs, where = S.requests()
    fsolve.fs_serve_start(budget, slots=slots, max_batch=max_batch)
    try:
        i = 0
        while i < len(reqs):
            k = 2 if (i + 1 < len(reqs) and reqs[i + 1].parent) else 1
            tk = fsolve.fs_serve_replay(reqs[i:i + k], [0.0] * k) if k == 1 else \
                fsolve.fs_serve_replay([reqs[i], _reparent(reqs[i + 1], 1)], [0.0, 0.0])
            _drain(tk)
            i += k
        alone = _snapshot(S.items)
        for it in S.items:
            it["out"].fill_(float("nan"))
            if it["follow"] is not None:
                it["follow"].fill_(float("nan"))
        arrivals = np.sort(np.random.default_rng(1).uniform(0.0, window_s, len(reqs)))
        tk = fsolve.fs_serve_replay(reqs, list(arrivals))
        _drain(tk, timeout_s=120.0)
        stats = fsolve.fs_serve_stats()
        for t in tk:
            assert fsolve.fs_serve_latency(t) > 0.0
        mixed = _snapshot(S.items)
        for (a_out, a_fol), (m_out, m_fol) in zip(alone, mixed):
            assert torch.equal(a_out, m_out)
            if a_fol is not None:
                assert torch.equal(a_fol, m_fol)
        return stats, tk
    finally:
        fsolve.fs_serve_stop()


def test_alone_vs_mix_large_grids(gpu_lib):
    """Grids of 2048^2 and more run as standalone passes inside their slot;
    they too give the same bits alone and next to small requests that share
    the persistent launch."""
    S = Stream(9, (2048, 256, 4096, 512, 1024, 2048, 128, 4096, 640), seed=17, explicit=True)
    stats, _ = _alone_vs_mix(S, 8 << 30, 3, 8, 0.003)
    assert stats["max_in_flight"] >= 2, stats
    for it in S.items:
        assert torch.isfinite(it["out"]).all()
    # the large grids against their closed forms (mode sums: exact on the grid)
    from oracle import closed_forms as cf

    for it in S.items:
        p = it["p"]
        if p.n < 2048:
            continue
        if p.op == "poisson":
            want = cf.poisson_modes(p.modes, p.n, p.n, 1.0, 1.0)
            den = np.linalg.norm(want)
        elif p.op == "diffusion":
            want = cf.diffusion_modes(p.modes, p.D, p.t, p.n, p.n, 1.0, 1.0)
            den = max(np.linalg.norm(want), np.linalg.norm(it["f"].double().cpu().numpy()))
        else:
            want = cf.wave_modes(p.modes, p.c, p.t, p.n, p.n, 1.0, 1.0)
            den = np.linalg.norm(want)
        got = it["out"].double().cpu().numpy()
        assert np.linalg.norm(got - want) / den <= 1e-5, (p.op, p.n)
    S.close()


def test_alone_vs_mix_and_oracle(gpu_lib):
    S = Stream(40, (128, 160, 256, 320, 512, 640, 1024), seed=3)
    # the mix: all requests arrive within ~2 ms
    stats, tk = _alone_vs_mix(S, 4 << 30, 3, 16, 0.002)
    assert stats["max_in_flight"] >= 2, stats
    # oracle on a sample (first output and follow-up of every fourth item)
    for it in S.items[::4]:
        p = it["p"]
        f = it["f"].double().cpu().numpy()
        if p.op == "poisson":
            want = oracle.poisson(f, 1.0, 1.0)
        elif p.op == "diffusion":
            want = oracle.diffusion(f, p.D, p.t, 1.0, 1.0)
        else:
            want = oracle.wave(f, None, p.c, p.t, 1.0, 1.0)
        got = it["out"].double().cpu().numpy()
        den = max(np.linalg.norm(want), np.linalg.norm(f) if p.op == "diffusion" else 0.0)
        assert np.linalg.norm(got - want) / den <= 1e-5, (p.op, p.n)
        if it["follow"] is not None:
            if p.op == "diffusion":
                want2 = oracle.diffusion(f, p.D, it["t2"], 1.0, 1.0)
            else:
                want2 = oracle.wave(f, None, p.c, it["t2"], 1.0, 1.0)
            got2 = it["follow"].double().cpu().numpy()
            den2 = max(np.linalg.norm(want2), np.linalg.norm(f) if p.op == "diffusion" else 0.0)
            assert np.linalg.norm(got2 - want2) / den2 <= 1e-5, (p.op, p.n, "follow-up")
    S.close()


def _reparent(req, parent_plus_one):
    r = fsolve.FsRequest()
    ctypes_copy(r, req)
    r.parent = parent_plus_one
    return r


def ctypes_copy(dst, src):
    import ctypes

    ctypes.memmove(ctypes.addressof(dst), ctypes.addressof(src), ctypes.sizeof(src))


def test_tight_budget_admits_as_memory_frees(gpu_lib):
    S = Stream(24, (512, 1024), seed=9)
    reqs, where = S.requests()
    one = (1024 // 2 + 1) * 1024 * 8  # one 1024^2 half spectrum
    budget = 4 * one + (1 << 20)
    fsolve.fs_serve_start(budget, slots=2, max_batch=8)
    try:
        tk = fsolve.fs_serve_replay(reqs, [0.0] * len(reqs))
        _drain(tk)
        st = fsolve.fs_serve_stats()
        assert st["completed"] >= len(reqs)
        assert st["peak_bytes"] <= budget
        assert st["kept"] == 0 and st["bytes_used"] == 0
    finally:
        fsolve.fs_serve_stop()
    for it in S.items:
        assert torch.isfinite(it["out"]).all()
    S.close()


def test_rejections(gpu_lib):
    S = Stream(2, (1024,), seed=4)
    fsolve.fs_serve_start(2 << 20, slots=2, max_batch=4)  # 2 MiB: nothing of 1024^2 fits
    try:
        it = S.items[0]
        r = fsolve.fs_request(OPS[it["p"].op], plan=S.plans[1024], in_u=it["f"], out_u=it["out"], D=0.1, c=1.0,
                              t=0.1)
        with pytest.raises(fsolve.FsError) as ei:
            fsolve.fs_serve_enqueue(r)
        assert ei.value.status == -4  # FS_ERR_BUDGET
        adv = fsolve.fs_request(fsolve.FS_OP_DIFFUSION_ADVANCE, out_u=it["out"], D=0.1, t=0.2, parent=987654)
        with pytest.raises(fsolve.FsError):
            fsolve.fs_serve_enqueue(adv)
    finally:
        fsolve.fs_serve_stop()
    S.close()


def test_followups_beyond_keep_are_rejected(gpu_lib):
    """A kept spectrum serves exactly `keep` follow-ups: the one after them is
    rejected at enqueue (it would otherwise read a released spectrum or wait
    forever), and the server still drains and stops."""
    S = Stream(1, (256,), seed=21)
    it = S.items[0]
    f = it["f"]
    out = [torch.empty_like(f) for _ in range(3)]
    fsolve.fs_serve_start(1 << 30, slots=2, max_batch=4)
    try:
        parent = fsolve.fs_serve_enqueue(fsolve.fs_request(fsolve.FS_OP_DIFFUSION, plan=S.plans[256], in_u=f,
                                                           out_u=out[0], D=0.01, t=0.2, keep=2))
        tk = [parent]
        for j in (1, 2):
            tk.append(fsolve.fs_serve_enqueue(fsolve.fs_request(fsolve.FS_OP_DIFFUSION_ADVANCE, out_u=out[j],
                                                                D=0.01, t=0.2 + 0.1 * j, parent=parent)))
        with pytest.raises(fsolve.FsError) as ei:
            fsolve.fs_serve_enqueue(fsolve.fs_request(fsolve.FS_OP_DIFFUSION_ADVANCE, out_u=out[1], D=0.01, t=0.9,
                                                      parent=parent))
        assert ei.value.status == -1
        _drain(tk)
        # every declared follow-up done: the spectrum is released, later ones are refused
        with pytest.raises(fsolve.FsError):
            fsolve.fs_serve_enqueue(fsolve.fs_request(fsolve.FS_OP_DIFFUSION_ADVANCE, out_u=out[1], D=0.01, t=0.9,
                                                      parent=parent))
        st = fsolve.fs_serve_stats()
        assert st["kept"] == 0 and st["bytes_used"] == 0 and st["failed"] == 0
    finally:
        fsolve.fs_serve_stop()  # returns: nothing is left waiting in the queue
    fh = f.double().cpu().numpy()
    for j, t in ((1, 0.3), (2, 0.4)):
        # normwise bar of strongly decaying diffusion: ||u - u_ref|| <= 1e-5 max(||u_ref||, ||f||)
        want = oracle.diffusion(fh, 0.01, t, 1.0, 1.0)
        den = max(np.linalg.norm(want), np.linalg.norm(fh))
        assert np.linalg.norm(out[j].double().cpu().numpy() - want) / den <= 1e-5
    S.close()
