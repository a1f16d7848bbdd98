"""Seeded synthetic inputs for the 2D Fourier-space solves.

This module holds input synthesis only -- random draws and the evaluation of
the initial fields -- and none of the solver's arithmetic.  The same
generators feed the CUDA path, the float64 oracle and the benchmark, so that
both sides of every parity check see identical inputs.

The paper's examples (Sec. III) use Gaussian sources and pulses A exp(-r^2/s^2)
on periodic squares; the workloads below keep those shapes and widen them to
the sizes the solver is measured on.  Seeds default to 12308 + workload index.
"""

from dataclasses import dataclass, field
import math

import numpy as np

__all__ = [
    "SUPPORTED_SIZES",
    "is_supported_size",
    "grid",
    "draw_modes",
    "mode_sum",
    "periodic_gaussians",
    "poisson_modes_64",
    "diffusion_blobs_1024",
    "wave_pulse_4096",
    "Problem",
    "batch_mix",
    "ServeRequest",
    "serve_stream",
    "OrbitSource",
]


def is_supported_size(n):
    """Even n = 2^a * {1, 3, 5} with 8 <= n <= 8192 (the solver's size set)."""
    if n < 8 or n > 8192 or n % 2:
        return False
    m = n
    while m % 2 == 0:
        m //= 2
    return m in (1, 3, 5)


SUPPORTED_SIZES = tuple(n for n in range(8, 8193, 2) if is_supported_size(n))


def grid(nx, ny, lx, ly, x0=0.0, y0=0.0):
    """Sample coordinates x_j = x0 + j Lx/Nx, y_k = y0 + k Ly/Ny (right end excluded)."""
    x = x0 + (lx / nx) * np.arange(nx, dtype=np.float64)
    y = y0 + (ly / ny) * np.arange(ny, dtype=np.float64)
    return x, y


def draw_modes(rng, n_modes=8, kmax=16):
    """n_modes (kx, ky, A, phi): integer wavenumbers uniform in [-kmax, kmax]^2
    (redrawn if (0, 0), so the field has zero mean), A ~ N(0, 1), phi ~ U[0, 2 pi)."""
    modes = []
    while len(modes) < n_modes:
        kx, ky = (int(v) for v in rng.integers(-kmax, kmax + 1, size=2))
        if kx == 0 and ky == 0:
            continue
        amp = float(rng.standard_normal())
        phi = float(rng.uniform(0.0, 2.0 * math.pi))
        modes.append((kx, ky, amp, phi))
    return modes


def mode_sum(modes, nx, ny, lx, ly):
    """Evaluate sum_m A_m cos(2 pi (kx x/Lx + ky y/Ly) + phi_m) on the grid (origin 0)."""
    j = np.arange(nx, dtype=np.int64)
    k = np.arange(ny, dtype=np.int64)
    out = np.zeros((ny, nx), dtype=np.float64)
    for kx, ky, amp, phi in modes:
        ang = 2.0 * np.pi * (((kx * j) % nx)[None, :] / nx + ((ky * k) % ny)[:, None] / ny) + phi
        out += amp * np.cos(ang)
    return out


def periodic_gaussians(blobs, nx, ny, lx, ly, images=2):
    """Sum over blobs (cx, cy, w, A) of A exp(-r^2/w^2), summed over periodic images."""
    x, y = grid(nx, ny, lx, ly)
    out = np.zeros((ny, nx), dtype=np.float64)
    for cx, cy, w, amp in blobs:
        for ix in range(-images, images + 1):
            ex = np.exp(-((x - cx - ix * lx) ** 2) / w**2)[None, :]
            for iy in range(-images, images + 1):
                out += amp * ex * np.exp(-((y - cy - iy * ly) ** 2) / w**2)[:, None]
    return out


# --------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------

def poisson_modes_64(seed=12308, n=64):
    """Poisson source on [0,1)^2, n x n (64 by default): 8 random Fourier modes.

    Returns (f, modes, (lx, ly)); f is float64 with zero mean by construction.
    """
    rng = np.random.default_rng(seed)
    kmax = min(16, n // 2 - 1)
    modes = draw_modes(rng, 8, kmax)
    lx = ly = 1.0
    return mode_sum(modes, n, n, lx, ly), modes, (lx, ly)


def diffusion_blobs_1024(seed=12309, n=1024, n_blobs=16, n_times=100):
    """Diffusion initial field on [0, 2 pi)^2: 16 periodic Gaussian blobs.

    Centres uniform in the domain, widths uniform in [0.05, 0.3], amplitudes
    N(0, 1); D = 0.1; output times evenly spaced in [0, 1] (n_times of them,
    both ends included).  Returns (u0, blobs, (lx, ly), D, times).
    """
    rng = np.random.default_rng(seed)
    lx = ly = 2.0 * math.pi
    blobs = []
    for _ in range(n_blobs):
        cx, cy = (float(v) for v in rng.uniform(0.0, lx, size=2))
        w = float(rng.uniform(0.05, 0.3))
        amp = float(rng.standard_normal())
        blobs.append((cx, cy, w, amp))
    u0 = periodic_gaussians(blobs, n, n, lx, ly)
    times = np.linspace(0.0, 1.0, n_times)
    return u0, blobs, (lx, ly), 0.1, times


def wave_pulse_4096(seed=12310, n=4096, n_snap=50, width=0.02, noise=0.01):
    """Wave initial data on [0,1)^2: a Gaussian pulse of width 0.02 at a seeded
    centre plus 0.01 * N(0,1) white noise; v0 = 0; c = 1; snapshot times
    t_j = j / n_snap, j = 1..n_snap.  Returns (u0, (lx, ly), c, times, centre).
    """
    rng = np.random.default_rng(seed)
    lx = ly = 1.0
    cx, cy = (float(v) for v in rng.uniform(0.0, 1.0, size=2))
    u0 = periodic_gaussians([(cx, cy, width, 1.0)], n, n, lx, ly, images=1)
    u0 += noise * rng.standard_normal((n, n))
    times = np.arange(1, n_snap + 1, dtype=np.float64) / n_snap
    return u0, (lx, ly), 1.0, times, (cx, cy)


OPS = ("poisson", "diffusion", "wave")
BATCH_SIZES = (64, 80, 96, 128, 160, 192, 256, 320, 384, 512, 640, 768, 1024, 1280, 1536, 2048)


@dataclass
class Problem:
    """One independent solve of a batch: operator, size, parameters and its source modes."""

    op: str
    n: int
    lx: float = 1.0
    ly: float = 1.0
    D: float = 0.0
    c: float = 0.0
    t: float = 0.0
    modes: list = field(default_factory=list)

    def field(self, dtype=np.float64):
        return mode_sum(self.modes, self.n, self.n, self.lx, self.ly).astype(dtype)


def batch_mix(seed=12311, count=512, sizes=BATCH_SIZES):
    """Uneven batch: operator uniform over {Poisson, diffusion D~U[0.01,1],
    wave c~U[0.5,2]} (t ~ U[0,1] for the time-dependent ones), square size
    uniform over ``sizes``, an 8-mode source on [0,1)^2."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        op = OPS[int(rng.integers(0, 3))]
        n = int(sizes[int(rng.integers(0, len(sizes)))])
        p = Problem(op=op, n=n)
        if op == "diffusion":
            p.D = float(rng.uniform(0.01, 1.0))
            p.t = float(rng.uniform(0.0, 1.0))
        elif op == "wave":
            p.c = float(rng.uniform(0.5, 2.0))
            p.t = float(rng.uniform(0.0, 1.0))
        p.modes = draw_modes(rng, 8, min(16, n // 2 - 1))
        out.append(p)
    return out


@dataclass
class ServeRequest:
    """One request of the open-loop serving stream."""

    rid: int
    arrival_s: float
    problem: Problem
    followup_t: float = -1.0   # >= 0: a second time requested on the same state
    followup_delay_s: float = 0.0


def _snap_log(n_real, sizes):
    ln = math.log(n_real)
    return min(sizes, key=lambda s: abs(math.log(s) - ln))


def serve_stream(rate_per_s, seed=12312, count=20000, nmin=128, nmax=8192, followup_mean_s=0.010):
    """Open-loop request stream: exponential inter-arrival gaps at ``rate_per_s``,
    size log-uniform in [nmin, nmax] snapped (in log distance) to a supported
    size, operator mixed as in ``batch_mix``; diffusion and wave requests carry
    a follow-up time t2 > t1 on the same state after an Exp(mean 10 ms) delay."""
    rng = np.random.default_rng(seed)
    sizes = [s for s in SUPPORTED_SIZES if nmin <= s <= nmax]
    t = 0.0
    out = []
    for rid in range(count):
        t += float(rng.exponential(1.0 / rate_per_s))
        n = _snap_log(math.exp(rng.uniform(math.log(nmin), math.log(nmax))), sizes)
        op = OPS[int(rng.integers(0, 3))]
        p = Problem(op=op, n=n)
        req = ServeRequest(rid=rid, arrival_s=t, problem=p)
        if op == "diffusion":
            p.D = float(rng.uniform(0.01, 1.0))
            p.t = float(rng.uniform(0.0, 1.0))
        elif op == "wave":
            p.c = float(rng.uniform(0.5, 2.0))
            p.t = float(rng.uniform(0.0, 1.0))
        p.modes = draw_modes(rng, 8, min(16, n // 2 - 1))
        if op != "poisson":
            req.followup_t = p.t + float(rng.uniform(0.0, 1.0))
            req.followup_delay_s = float(rng.exponential(followup_mean_s))
        out.append(req)
    return out


# --------------------------------------------------------------------------
# Time-dependent source of the wave example (Sec. III.C, example with source)
# --------------------------------------------------------------------------

@dataclass
class OrbitSource:
    """s(t, x, y) = A exp(-|x - x0(t)|^2 / sigma^2) cos(gamma t), with the
    centre on a circle: x0(t) = radius (cos(Omega t), sin(Omega t)).

    The paper's parameters: A = 1, sigma = 0.1, Omega = 5, gamma = 10 on
    [-2, 2]^2.  The orbit radius is not stated; radius = 1 is our reading.
    The distance is the minimum image on the periodic domain (images beyond
    it contribute below e^-100 for these widths).  Grid x_j = x_min + j Lx/Nx.
    """

    A: float = 1.0
    sigma: float = 0.1
    radius: float = 1.0
    Omega: float = 5.0
    gamma: float = 10.0
    x_min: float = -2.0
    y_min: float = -2.0

    def centre(self, t):
        return self.radius * math.cos(self.Omega * t), self.radius * math.sin(self.Omega * t)

    def field(self, t, nx, ny, lx, ly):
        """The source sampled on the [ny][nx] grid at time t (float64)."""
        cx, cy = self.centre(t)
        x, y = grid(nx, ny, lx, ly, self.x_min, self.y_min)
        dx = x - cx
        dx -= lx * np.round(dx / lx)
        dy = y - cy
        dy -= ly * np.round(dy / ly)
        r2 = dy[:, None] ** 2 + dx[None, :] ** 2
        return self.A * math.cos(self.gamma * t) * np.exp(-r2 / self.sigma**2)

