"""Pins for the float64 oracle: checks against what the paper and the mathematics fix.

Each ``pin_*`` function returns the worst relative error it observed; the
tests assert a bound on it, and the mutation tests assert that a planted
mistake in the oracle drives at least one pin over its bound.  None of these
re-types the oracle's formula: they use brute-force sums, numpy.fft (a library
routine), exact closed forms, finite differences and invariants.
"""

import cmath
import math

import numpy as np

import oracle
from oracle import closed_forms as cf
from paper_2412_12308_gb300 import workloads as wl


def rel(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    den = float(np.linalg.norm(b.ravel()))
    return float(np.linalg.norm((a - b).ravel())) / (den if den > 0 else 1.0)


# ----------------------------------------------------------------- transforms
def brute_dft2(p):
    """O(N^4) direct 2D sum with one combined exponential (Eq. 2D_DFT, sign -1)."""
    ny, nx = p.shape
    out = np.zeros((ny, nx), dtype=np.complex128)
    for b in range(ny):
        for a in range(nx):
            s = 0j
            for k in range(ny):
                for j in range(nx):
                    s += complex(p[k, j]) * cmath.exp(-2j * math.pi * (a * j / nx + b * k / ny))
            out[b, a] = s
    return out


def pin_bruteforce(shapes=((1, 1), (2, 3), (4, 4), (5, 7), (8, 6), (3, 16), (12, 10))):
    rng = np.random.default_rng(1)
    worst = 0.0
    for ny, nx in shapes:
        p = rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))
        worst = max(worst, rel(oracle.dft2(p), brute_dft2(p)))
    return worst


def pin_numpy_fft(shapes=((64, 64), (96, 80), (160, 128), (256, 320), (30, 42))):
    rng = np.random.default_rng(2)
    worst = 0.0
    for ny, nx in shapes:
        p = rng.standard_normal((ny, nx))
        worst = max(worst, rel(oracle.dft2(p), np.fft.fft2(p)))
        P = rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))
        worst = max(worst, rel(oracle.idft2(P), np.fft.ifft2(P)))
    return worst


def pin_roundtrip(shapes=((64, 64), (48, 40), (128, 96))):
    rng = np.random.default_rng(3)
    worst = 0.0
    for ny, nx in shapes:
        p = rng.standard_normal((ny, nx))
        worst = max(worst, rel(oracle.idft2(oracle.dft2(p)), p))
    return worst


def pin_parseval(shapes=((64, 64), (40, 96))):
    rng = np.random.default_rng(4)
    worst = 0.0
    for ny, nx in shapes:
        p = rng.standard_normal((ny, nx))
        lhs = float(np.sum(p * p))
        rhs = float(np.sum(np.abs(oracle.dft2(p)) ** 2)) / (nx * ny)
        worst = max(worst, abs(lhs - rhs) / lhs)
    return worst


def pin_single_mode(n=24):
    """x_j = exp(+2 pi i a0 j / N) transforms (sign -1) to N at index a0 only."""
    worst = 0.0
    for a0 in (0, 1, 5, n // 2, n - 1):
        x = np.exp(2j * np.pi * a0 * np.arange(n) / n)
        want = np.zeros(n, dtype=np.complex128)
        want[a0] = n
        worst = max(worst, rel(oracle.dft1(x, sign=-1), want))
    return worst


# ----------------------------------------------------------------- Poisson
def pin_poisson_modes(seed=12308, n=64):
    f, modes, (lx, ly) = wl.poisson_modes_64(seed, n)
    u = oracle.poisson(f, lx, ly)
    return rel(u, cf.poisson_modes(modes, n, n, lx, ly))


def pin_poisson_sinsin(n=32):
    """f = sin(2 pi x) sin(2 pi y) on [0,1)^2 has lap u = f for u = -f / (8 pi^2)."""
    x = np.arange(n) / n
    f = np.sin(2 * np.pi * x)[None, :] * np.sin(2 * np.pi * x)[:, None]
    return rel(oracle.poisson(f, 1.0, 1.0), -f / (8.0 * np.pi**2))


def pin_poisson_rect(nx=48, ny=20, lx=3.0, ly=0.5):
    """Non-square grid and domain: f = cos(2 pi (2x/Lx + 3y/Ly)), u = -f/|w|^2."""
    x = lx * np.arange(nx) / nx
    y = ly * np.arange(ny) / ny
    f = np.cos(2 * np.pi * (2 * x[None, :] / lx + 3 * y[:, None] / ly))
    w2 = (2 * np.pi * 2 / lx) ** 2 + (2 * np.pi * 3 / ly) ** 2
    return rel(oracle.poisson(f, lx, ly), -f / w2)


def pin_poisson_nyquist(n=16, length=2.0):
    """The Nyquist mode (-1)^j along x is kept with |omega| = pi N / L."""
    f = np.tile(((-1.0) ** np.arange(n))[None, :], (n, 1))
    w2 = (np.pi * n / length) ** 2
    return rel(oracle.poisson(f, length, length), -f / w2)


def pin_poisson_fd(n=128, length=4.0, sigma=0.1):
    """Gaussian source of Sec. III.A on [-2,2]^2: an 8th-order finite-difference
    Laplacian of u must reproduce f - mean(f)."""
    h = length / n
    x = -length / 2 + h * np.arange(n)
    r2 = x[None, :] ** 2 + x[:, None] ** 2
    f = np.exp(-r2 / sigma**2)
    u = oracle.poisson(f, length, length)
    c = [-205.0 / 72, 8.0 / 5, -1.0 / 5, 8.0 / 315, -1.0 / 560]
    lap = 2 * c[0] * u
    for m in range(1, 5):
        lap = lap + c[m] * (np.roll(u, m, 0) + np.roll(u, -m, 0) + np.roll(u, m, 1) + np.roll(u, -m, 1))
    lap /= h * h
    return rel(lap, f - f.mean())


def pin_poisson_invariants(seed=7, n=40):
    rng = np.random.default_rng(seed)
    f = rng.standard_normal((n, n))
    u = oracle.poisson(f, 1.0, 1.0)
    u2 = oracle.poisson(f + 3.25, 1.0, 1.0)
    mean_err = abs(float(u.mean())) / float(np.abs(u).max())
    return max(mean_err, rel(u2, u))


# ----------------------------------------------------------------- diffusion
def pin_diffusion_mode(n=32, D=0.01, t=0.7):
    modes = [(3, -2, 1.0, 0.4), (0, 5, -0.5, 1.1)]
    u0 = wl.mode_sum(modes, n, n, 1.0, 1.0)
    got = oracle.diffusion(u0, D, t, 1.0, 1.0)
    want = np.zeros_like(u0)
    for kx, ky, amp, phi in modes:
        w2 = (2 * np.pi) ** 2 * (kx * kx + ky * ky)
        want += math.exp(-D * w2 * t) * wl.mode_sum([(kx, ky, amp, phi)], n, n, 1.0, 1.0)
    return rel(got, want)


def pin_diffusion_gaussian(n=256, D=0.1, t=1.0, seed=5):
    """Heat-kernel evolution of periodic Gaussians on [0, 2 pi)^2."""
    rng = np.random.default_rng(seed)
    lx = 2 * math.pi
    blobs = [(float(rng.uniform(0, lx)), float(rng.uniform(0, lx)), float(rng.uniform(0.15, 0.3)),
              float(rng.standard_normal())) for _ in range(4)]
    u0 = wl.periodic_gaussians(blobs, n, n, lx, lx)
    got = oracle.diffusion(u0, D, t, lx, lx)
    return rel(got, cf.gaussian_heat(blobs, D, t, n, n, lx, lx))


def pin_diffusion_invariants(n=48, D=0.05, seed=8):
    rng = np.random.default_rng(seed)
    u0 = rng.standard_normal((n, n)) + 0.7
    worst = rel(oracle.diffusion(u0, D, 0.0, 1.0, 1.0), u0)  # t = 0 is the identity
    for t in (0.1, 1.0, 10.0):
        u = oracle.diffusion(u0, D, t, 1.0, 1.0)
        worst = max(worst, abs(u.mean() / u0.mean() - 1.0))  # mean conserved
    u1 = oracle.diffusion(u0, D, 0.3, 1.0, 1.0)
    worst = max(worst, rel(oracle.diffusion(u1, D, 0.4, 1.0, 1.0), oracle.diffusion(u0, D, 0.7, 1.0, 1.0)))
    return worst


def pin_diffusion_fd_time(n=32, D=0.2, t=0.05, dt=1e-5, seed=9):
    """du/dt = D lap u: the central time difference of u, Poisson-inverted and
    divided by D, gives u - mean(u) (O(dt^2) accurate)."""
    rng = np.random.default_rng(seed)
    u0 = wl.mode_sum(wl.draw_modes(rng, 6, 5), n, n, 1.0, 1.0)
    up = oracle.diffusion(u0, D, t + dt, 1.0, 1.0)
    um = oracle.diffusion(u0, D, t - dt, 1.0, 1.0)
    u = oracle.diffusion(u0, D, t, 1.0, 1.0)
    dudt = (up - um) / (2 * dt)
    return rel(oracle.poisson(dudt / D, 1.0, 1.0), u - u.mean())


# ----------------------------------------------------------------- wave
def pin_wave_mode(n=32, c=1.3, t=0.37):
    modes = [(2, 1, 0.8, 0.2), (-3, 4, 0.3, 2.0)]
    u0 = wl.mode_sum(modes, n, n, 1.0, 1.0)
    u, v = oracle.wave(u0, None, c, t, 1.0, 1.0, want_v=True)
    wu = np.zeros_like(u0)
    wv = np.zeros_like(u0)
    for kx, ky, amp, phi in modes:
        w = 2 * np.pi * math.sqrt(kx * kx + ky * ky)
        m = wl.mode_sum([(kx, ky, amp, phi)], n, n, 1.0, 1.0)
        wu += math.cos(c * w * t) * m
        wv += -c * w * math.sin(c * w * t) * m
    return max(rel(u, wu), rel(v, wv))


def pin_wave_velocity_fd(n=32, c=0.8, t=0.3, dt=1e-5, seed=10):
    """v returned by the oracle equals the central time difference of u; the
    initial velocity g is honoured (checked by a difference at t = 0)."""
    rng = np.random.default_rng(seed)
    u0 = wl.mode_sum(wl.draw_modes(rng, 5, 6), n, n, 1.0, 1.0) + 0.2
    g0 = wl.mode_sum(wl.draw_modes(rng, 5, 6), n, n, 1.0, 1.0) - 0.1
    up = oracle.wave(u0, g0, c, t + dt, 1.0, 1.0)
    um = oracle.wave(u0, g0, c, t - dt, 1.0, 1.0)
    _u, v = oracle.wave(u0, g0, c, t, 1.0, 1.0, want_v=True)
    e1 = rel((up - um) / (2 * dt), v)
    vp = oracle.wave(u0, g0, c, dt, 1.0, 1.0)
    vm = oracle.wave(u0, g0, c, -dt, 1.0, 1.0)
    e2 = rel((vp - vm) / (2 * dt), g0)
    return max(e1, e2)


def pin_wave_invariants(n=40, c=1.0, seed=11):
    rng = np.random.default_rng(seed)
    u0 = rng.standard_normal((n, n)) + 0.3
    g0 = 0.5 * rng.standard_normal((n, n)) - 0.05
    worst = 0.0
    # mean conserved for g = 0; grows as mean(g) t otherwise (Eq. OmegaZero)
    for t in (0.25, 1.0, 2.0):
        u = oracle.wave(u0, None, c, t, 1.0, 1.0)
        worst = max(worst, abs(u.mean() / u0.mean() - 1.0))
        u = oracle.wave(u0, g0, c, t, 1.0, 1.0)
        worst = max(worst, abs(u.mean() - (u0.mean() + g0.mean() * t)) / abs(u0.mean()))
    # energy: sum v^2 + c^2 |grad u|^2, with the gradient energy from a 2D FFT (numpy)
    def energy(u, v):
        U = np.fft.fft2(u)
        k = 2 * np.pi * np.fft.fftfreq(n, 1.0 / n)
        kk = k[None, :] ** 2 + k[:, None] ** 2
        return float(np.sum(v * v)) + c * c * float(np.sum(kk * np.abs(U) ** 2)) / (n * n)
    e0 = energy(u0, g0)
    u, v = oracle.wave(u0, g0, c, 0.77, 1.0, 1.0, want_v=True)
    worst = max(worst, abs(energy(u, v) / e0 - 1.0))
    # time reversal: evolve (u, v) back by -t
    ub, vb = oracle.wave(u, v, c, -0.77, 1.0, 1.0, want_v=True)
    worst = max(worst, rel(ub, u0), rel(vb, g0))
    # period return of a single mode
    w = 2 * np.pi * math.sqrt(2 * 2 + 1 * 1)
    m = wl.mode_sum([(2, 1, 1.0, 0.3)], n, n, 1.0, 1.0)
    worst = max(worst, rel(oracle.wave(m, None, c, 2 * np.pi / (c * w), 1.0, 1.0), m))
    return worst


def pin_sign_independence(n=24, seed=12):
    rng = np.random.default_rng(seed)
    f = rng.standard_normal((n, n + 8))
    a = oracle.poisson(f, 1.0, 1.3, sign=-1)
    b = oracle.poisson(f, 1.0, 1.3, sign=+1)
    worst = rel(a, b)
    a = oracle.wave(f, f * 0.5, 1.1, 0.4, 1.0, 1.3, sign=-1)
    b = oracle.wave(f, f * 0.5, 1.1, 0.4, 1.0, 1.3, sign=+1)
    worst = max(worst, rel(a, b))
    a = oracle.diffusion(f, 0.01, 0.4, 1.0, 1.3, sign=-1)
    b = oracle.diffusion(f, 0.01, 0.4, 1.0, 1.3, sign=+1)
    return max(worst, rel(a, b))


# ----------------------------------------------------------------- constant sources
def _nrm(x):
    return float(np.linalg.norm(x))


def _lap_fft(u, L=1.0):
    n = u.shape[0]
    k = 2 * np.pi * np.fft.fftfreq(n, L / n)
    kk = k[None, :] ** 2 + k[:, None] ** 2
    return np.real(np.fft.ifft2(-kk * np.fft.fft2(u)))


def pin_diffusion_source_pde(n=32, D=0.2, t=0.07, dt=1e-5, seed=13):
    """u_t - D lap u = s (time central difference; Laplacian from numpy.fft) and u(0) = f."""
    rng = np.random.default_rng(seed)
    f = wl.mode_sum(wl.draw_modes(rng, 6, 5), n, n, 1.0, 1.0) + 0.3
    src = wl.mode_sum(wl.draw_modes(rng, 6, 5), n, n, 1.0, 1.0) + 0.7
    F, S = oracle.state_spectrum(f), oracle.state_spectrum(src)

    def u(tt):
        return np.real(oracle.idft2(oracle.diffusion_source_spectrum(F, S, D, tt, 1.0, 1.0)))
    res = (u(t + dt) - u(t - dt)) / (2 * dt) - D * _lap_fft(u(t)) - src
    return max(_nrm(res) / _nrm(src), rel(u(0.0), f))


def pin_wave_source_pde(n=32, c=0.9, t=0.21, dt=2e-4, seed=14):
    """u_tt - c^2 lap u = s, u(0) = f, u_t(0) = g, and v = u_t.

    u_tt is the Richardson combination of central second differences at dt
    and dt/2 (truncation O(dt^4)).
    """
    rng = np.random.default_rng(seed)
    f = wl.mode_sum(wl.draw_modes(rng, 6, 3), n, n, 1.0, 1.0) + 0.2
    g = wl.mode_sum(wl.draw_modes(rng, 6, 3), n, n, 1.0, 1.0) - 0.1
    src = wl.mode_sum(wl.draw_modes(rng, 6, 3), n, n, 1.0, 1.0) + 0.4
    F, G, S = (oracle.state_spectrum(x) for x in (f, g, src))

    def uv(tt):
        U, V = oracle.wave_source_spectrum(F, G, S, c, tt, 1.0, 1.0)
        return np.real(oracle.idft2(U)), np.real(oracle.idft2(V))
    u0, v0 = uv(t)

    def d2(h):
        return (uv(t + h)[0] - 2 * u0 + uv(t - h)[0]) / h**2
    utt = (4 * d2(dt / 2) - d2(dt)) / 3
    res = utt - c * c * _lap_fft(u0) - src
    e1 = _nrm(res) / _nrm(src)
    ut = (8 * (uv(t + dt / 2)[0] - uv(t - dt / 2)[0]) - (uv(t + dt)[0] - uv(t - dt)[0])) / (6 * dt)
    e2 = rel(ut, v0)
    a, b = uv(0.0)
    return max(e1, e2, rel(a, f), rel(b, g))


# ------------------------------------------------------------ complex fields
def pin_complex_plane_wave(nx=24, ny=20, lx=1.7, ly=0.8, kx=3, ky=-5, D=0.001, c=1.1, t=0.4):
    """exp(i (wx x + wy y)) is an eigenfunction: Poisson -> -mode/|w|^2,
    diffusion -> mode exp(-D|w|^2 t), wave (v0 = 0) -> mode cos(c|w|t); the
    negative ky checks that a complex field uses the full spectrum."""
    x = (lx / nx) * np.arange(nx)
    y = (ly / ny) * np.arange(ny)
    wx, wy = 2 * np.pi * kx / lx, 2 * np.pi * ky / ly
    mode = np.exp(1j * (wy * y[:, None] + wx * x[None, :]))
    w2 = wx * wx + wy * wy
    e1 = rel(oracle.poisson_complex(mode, lx, ly), -mode / w2)
    e2 = rel(oracle.diffusion_complex(mode, D, t, lx, ly), mode * math.exp(-D * w2 * t))
    e3 = rel(oracle.wave_complex(mode, None, c, t, lx, ly), mode * math.cos(c * math.sqrt(w2) * t))
    return max(e1, e2, e3)


def pin_complex_linearity(n=32, seed=17):
    """The operators are real multipliers: solve(a + i b) = solve(a) + i solve(b)
    with the real solves (pinned above) on a and b."""
    rng = np.random.default_rng(seed)
    a, b, g = rng.standard_normal((n, n)), rng.standard_normal((n, n)), rng.standard_normal((n, n))
    e1 = rel(oracle.poisson_complex(a + 1j * b, 1.0, 1.3), oracle.poisson(a, 1.0, 1.3) + 1j * oracle.poisson(b, 1.0, 1.3))
    e2 = rel(oracle.diffusion_complex(a + 1j * b, 0.02, 0.3, 1.0, 1.3),
             oracle.diffusion(a, 0.02, 0.3, 1.0, 1.3) + 1j * oracle.diffusion(b, 0.02, 0.3, 1.0, 1.3))
    e3 = rel(oracle.wave_complex(a + 1j * b, g + 0j, 0.9, 0.37, 1.0, 1.3),
             oracle.wave(a, g, 0.9, 0.37, 1.0, 1.3) + 1j * oracle.wave(b, None, 0.9, 0.37, 1.0, 1.3))
    return max(e1, e2, e3)


# ----------------------------------------------------------------------- RK4
def pin_rk4_propagator(nx=8, ny=6, lx=1.3, ly=0.9, c=1.1, dt=0.06, seed=15):
    """One RK4 step of the free oscillator is the degree-4 Taylor polynomial of
    exp(dt A), A = [[0, 1], [-w^2, 0]]; with A^2 = -w^2 I it is
    a I + b A, a = 1 - z^2/2 + z^4/24, b = dt (1 - z^2/6), z = dt w."""
    rng = np.random.default_rng(seed)
    F = rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))
    G = rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))
    U, V = oracle.wave_rk4_spectrum(F, G, None, c, 0.0, dt, 1, lx, ly)
    w2 = c * c * oracle.omega2(nx, ny, lx, ly)
    z2 = dt * dt * w2
    a = 1.0 - z2 / 2.0 + z2 * z2 / 24.0
    b = dt * (1.0 - z2 / 6.0)
    return max(rel(U, a * F + b * G), rel(V, a * G - w2 * b * F))


def _const_gauss(n, L):
    src = wl.OrbitSource(A=1.0, sigma=0.5, radius=0.3, Omega=0.0, gamma=0.0)
    return src.field(0.0, n, n, L, L)


def pin_rk4_constant_source_order(n=16, L=4.0, c=1.0, T=0.5, seed=16):
    """Constant source: RK4 converges to solve.wave_source_spectrum with
    order 4 (errors at dt = 0.01 and 0.005 in ratio ~16) and is within
    1.5e-6 of it at dt = 0.005."""
    rng = np.random.default_rng(seed)
    F = oracle.state_spectrum(rng.standard_normal((n, n)))
    G = oracle.state_spectrum(rng.standard_normal((n, n)))
    s = _const_gauss(n, L)
    Ue, _ = oracle.wave_source_spectrum(F, G, oracle.state_spectrum(s), c, T, L, L)
    errs = []
    for steps in (50, 100):
        U, _ = oracle.wave_rk4_spectrum(F, G, lambda t: s, c, 0.0, T / steps, steps, L, L)
        errs.append(rel(U, Ue))
    order = math.log2(errs[0] / errs[1])
    return max(abs(order - 4.0), errs[1] / 1e-5)


def _orbit_mean(n, dt, T, L=4.0):
    src = wl.OrbitSource()
    steps = int(round(T / dt))
    U, _ = oracle.wave_rk4_spectrum(np.zeros((n, n)), None, lambda t: src.field(t, n, n, L, L), 1.0, 0.0, dt,
                                    steps, L, L)
    return U[0, 0].real / (n * n)


def pin_rk4_orbit_self_convergence(n=64, T=1.0):
    """The paper's example with an orbiting source (A = 1, sigma = 0.1, Omega = 5,
    gamma = 10 on [-2, 2]^2, dt = h/4 for N = 64, 128, 256): the means u1, u2,
    u3 at dt, dt/2, dt/4 self-converge with (u2 - u1)/(u3 - u2) ~ 2^4
    (tests/golden/paper_facts.txt); also the mean mode u'' = mean(s) has the
    exact solution A pi sigma^2/L^2 (1 - cos(gamma t))/gamma^2 (the grid sum
    of the Gaussian equals pi sigma^2/h^2 to ~1e-11 at N = 64), and u3 is
    within twice the Richardson estimate |u3 - u2|/15 of it."""
    from tests.golden import load_facts

    dts = [0.25 * 4.0 / N for N in (64, 128, 256)]
    u1, u2, u3 = (_orbit_mean(n, dt, T) for dt in dts)
    factor = (u2 - u1) / (u3 - u2)
    want = load_facts()["rk4_self_convergence_factor"]
    src = wl.OrbitSource()
    exact = src.A * math.pi * src.sigma**2 / 16.0 * (1.0 - math.cos(src.gamma * T)) / src.gamma**2
    richardson = abs(u3 - u2) / 15.0
    return max(abs(factor - want) / want, 0.1 * abs(u3 - exact) / (2.0 * richardson))


# name -> (function, bound)
PINS = {
    "bruteforce": (pin_bruteforce, 1e-13),
    "numpy_fft": (pin_numpy_fft, 1e-13),
    "roundtrip": (pin_roundtrip, 1e-14),
    "parseval": (pin_parseval, 1e-13),
    "single_mode": (pin_single_mode, 1e-13),
    "poisson_modes": (pin_poisson_modes, 1e-12),
    "poisson_sinsin": (pin_poisson_sinsin, 1e-13),
    "poisson_rect": (pin_poisson_rect, 1e-13),
    "poisson_nyquist": (pin_poisson_nyquist, 1e-13),
    "poisson_fd": (pin_poisson_fd, 2e-3),
    "poisson_invariants": (pin_poisson_invariants, 1e-12),
    "diffusion_mode": (pin_diffusion_mode, 1e-12),
    "diffusion_gaussian": (pin_diffusion_gaussian, 1e-11),
    "diffusion_invariants": (pin_diffusion_invariants, 1e-12),
    "diffusion_fd_time": (pin_diffusion_fd_time, 1e-6),
    "wave_mode": (pin_wave_mode, 1e-12),
    "wave_velocity_fd": (pin_wave_velocity_fd, 1e-6),
    "wave_invariants": (pin_wave_invariants, 1e-11),
    "sign_independence": (pin_sign_independence, 1e-13),
    "diffusion_source_pde": (pin_diffusion_source_pde, 1e-6),
    "wave_source_pde": (pin_wave_source_pde, 1e-5),
    "complex_plane_wave": (pin_complex_plane_wave, 1e-13),
    "complex_linearity": (pin_complex_linearity, 1e-13),
    "rk4_propagator": (pin_rk4_propagator, 1e-13),
    "rk4_constant_source_order": (pin_rk4_constant_source_order, 0.15),
    "rk4_orbit_self_convergence": (pin_rk4_orbit_self_convergence, 0.1),
}
