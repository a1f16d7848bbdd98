"""The seeded input generators follow their stated recipe (CPU).

Every timed or tested workload is synthetic.  These checks pin what the
generators promise: fixed seeds give fixed inputs, parameters stay in their
stated ranges and distributions, mode sums have zero mean, periodic Gaussians
are periodic with the stated mass, and the serving stream's arrivals,
sizes and follow-ups have the stated statistics.
"""

import math

import numpy as np

from paper_2412_12308_gb300 import workloads as wl


def test_poisson_modes_recipe():
    f, modes, (lx, ly) = wl.poisson_modes_64()
    g, modes2, _ = wl.poisson_modes_64()
    assert np.array_equal(f, g) and modes == modes2  # seeded
    assert f.shape == (64, 64) and (lx, ly) == (1.0, 1.0)
    assert len(modes) == 8
    for kx, ky, amp, phi in modes:
        assert -16 <= kx <= 16 and -16 <= ky <= 16 and (kx, ky) != (0, 0)
        assert 0.0 <= phi < 2 * math.pi
    assert abs(f.mean()) <= 1e-12 * np.abs(f).max()  # zero mean by construction


def test_mode_sum_is_the_stated_cosine_sum():
    modes = [(3, -2, 0.7, 0.4), (0, 5, -1.1, 2.0)]
    nx, ny = 24, 20
    f = wl.mode_sum(modes, nx, ny, 2.0, 3.0)
    x = np.arange(nx) * 2.0 / nx
    y = np.arange(ny) * 3.0 / ny
    want = sum(a * np.cos(2 * np.pi * (kx * x[None, :] / 2.0 + ky * y[:, None] / 3.0) + p)
               for kx, ky, a, p in modes)
    assert np.allclose(f, want, atol=1e-12)


def test_periodic_gaussian_is_periodic_with_the_stated_mass():
    lx = ly = 2 * math.pi
    n = 256
    blob = (0.05, 6.2, 0.3, 1.5)  # centre next to the domain edges: images matter
    g = wl.periodic_gaussians([blob], n, n, lx, ly)
    # mass of A exp(-r^2/w^2) over the plane: A pi w^2 (the grid sum is exact
    # to roundoff for a smooth periodic function)
    mass = g.sum() * (lx / n) * (ly / n)
    assert abs(mass - 1.5 * math.pi * 0.3 ** 2) <= 1e-10
    # periodicity: shifting the centre by a period leaves the field unchanged
    g2 = wl.periodic_gaussians([(0.05 + lx, 6.2 - ly, 0.3, 1.5)], n, n, lx, ly)
    assert np.allclose(g, g2, atol=1e-12)


def test_diffusion_blobs_recipe():
    u0, blobs, (lx, ly), D, times = wl.diffusion_blobs_1024(n=128)
    u1, blobs1, _, _, _ = wl.diffusion_blobs_1024(n=128)
    assert np.array_equal(u0, u1) and blobs == blobs1
    assert u0.shape == (128, 128) and lx == ly == 2 * math.pi and D == 0.1
    assert len(blobs) == 16
    for cx, cy, w, amp in blobs:
        assert 0.0 <= cx < lx and 0.0 <= cy < ly and 0.05 <= w <= 0.3
    assert len(times) == 100 and times[0] == 0.0 and times[-1] == 1.0
    assert np.allclose(np.diff(times), 1.0 / 99)


def test_wave_pulse_recipe():
    n = 256
    u0, (lx, ly), c, times, (cx, cy) = wl.wave_pulse_4096(n=n)
    assert u0.shape == (n, n) and (lx, ly) == (1.0, 1.0) and c == 1.0
    assert 0.0 <= cx < 1.0 and 0.0 <= cy < 1.0
    assert len(times) == 50 and np.allclose(times, np.arange(1, 51) / 50)
    noise = u0 - wl.periodic_gaussians([(cx, cy, 0.02, 1.0)], n, n, 1.0, 1.0, images=1)
    assert abs(noise.std() - 0.01) <= 0.001 and abs(noise.mean()) <= 0.001


def test_batch_mix_recipe():
    probs = wl.batch_mix()
    again = wl.batch_mix()
    assert len(probs) == 512
    assert [(p.op, p.n, p.D, p.c, p.t) for p in probs] == [(p.op, p.n, p.D, p.c, p.t) for p in again]
    sizes = {p.n for p in probs}
    assert sizes <= set(wl.BATCH_SIZES) and len(sizes) == len(wl.BATCH_SIZES)
    assert all(wl.is_supported_size(n) for n in wl.BATCH_SIZES)
    counts = {op: sum(p.op == op for p in probs) for op in wl.OPS}
    assert all(abs(c - 512 / 3) < 4 * math.sqrt(512 * (1 / 3) * (2 / 3)) for c in counts.values()), counts
    for p in probs:
        assert len(p.modes) == 8
        if p.op == "diffusion":
            assert 0.01 <= p.D <= 1.0 and 0.0 <= p.t <= 1.0
        elif p.op == "wave":
            assert 0.5 <= p.c <= 2.0 and 0.0 <= p.t <= 1.0
        # every mode below the Nyquist frequency of its grid
        assert all(max(abs(kx), abs(ky)) < p.n // 2 for kx, ky, _, _ in p.modes)


def test_serve_stream_recipe():
    rate = 2000.0
    reqs = wl.serve_stream(rate, count=4000)
    assert len(reqs) == 4000
    gaps = np.diff([0.0] + [r.arrival_s for r in reqs])
    assert (gaps > 0).all()
    assert abs(gaps.mean() * rate - 1.0) <= 0.06  # exponential gaps of mean 1/rate
    assert abs(gaps.std() / gaps.mean() - 1.0) <= 0.08  # coefficient of variation 1
    ns = np.array([r.problem.n for r in reqs])
    assert ns.min() >= 128 and ns.max() <= 8192 and all(wl.is_supported_size(int(n)) for n in set(ns))
    # log-uniform sizes: about half the requests below the geometric middle (1024)
    assert 0.4 <= (ns < 1024).mean() <= 0.6
    delays = []
    for r in reqs:
        if r.problem.op == "poisson":
            assert r.followup_t < 0
        else:
            assert r.followup_t > r.problem.t
            delays.append(r.followup_delay_s)
    assert abs(np.mean(delays) / 0.010 - 1.0) <= 0.1
