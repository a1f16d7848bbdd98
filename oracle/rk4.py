"""RK4 time integration of the wave equation in Fourier space (test infrastructure only).

Sec. III.C: in Fourier space the wave equation u_tt = c^2 lap u + s is, for
every mode, a forced oscillator (Eq. WaveEquationFourierSpace); written as the
first-order system of Eq. SystemOfODEsForWaveEquation,
    dU/dt = V,   dV/dt = -c^2 |omega|^2 U + S(t),
it is integrated with the classical fourth-order Runge-Kutta method (Kutta's
1901 scheme: slopes at the start, twice at the midpoint, at the end, weights
1/6, 2/6, 2/6, 1/6), as the paper's example with an orbiting source does.
The wave speed c rescales time as in the source-free case (c = 1 there).

S(t) is the forward 2D DFT (oracle.dft2, full spectrum) of the source sampled
on the grid at the stage time; the caller passes the sampler.  Step k runs
from t_k = t0 + k dt and evaluates the source at t_k, t_k + dt/2 and
t_k + dt.  Everything is float64 / complex128.

Pinned by: the one-step RK4 propagator of the free oscillator in closed form,
fourth-order convergence to the constant-source closed form
(solve.wave_source_spectrum), the mean mode against the exact solution for
the orbiting source, and the paper's self-convergence factor ~16.
"""

import numpy as np

from .dft import dft2
from .solve import omega2

__all__ = ["wave_rk4_spectrum"]


def wave_rk4_spectrum(F, G, source, c, t0, dt, nsteps, lx, ly, sign=-1):
    """(U, V) after `nsteps` RK4 steps of size dt from (F, G) at time t0.

    F, G: full spectra [Ny][Nx] of u and u_t at t0 (G may be None: zero).
    source(t): the real source field [Ny][Nx] at time t (None: s = 0).
    """
    F = np.asarray(F, dtype=np.complex128)
    ny, nx = F.shape
    w2 = float(c) ** 2 * omega2(nx, ny, lx, ly)
    U = F.copy()
    V = np.zeros_like(U) if G is None else np.asarray(G, dtype=np.complex128).copy()

    def S(t):
        if source is None:
            return np.zeros_like(U)
        return dft2(np.asarray(source(t), dtype=np.float64), sign=sign)

    def slope(u, v, s):
        return v, -w2 * u + s

    s_start = S(float(t0))
    for k in range(int(nsteps)):
        t = float(t0) + k * float(dt)
        s_mid = S(t + 0.5 * dt)
        s_end = S(t + dt)
        k1u, k1v = slope(U, V, s_start)
        k2u, k2v = slope(U + 0.5 * dt * k1u, V + 0.5 * dt * k1v, s_mid)
        k3u, k3v = slope(U + 0.5 * dt * k2u, V + 0.5 * dt * k2v, s_mid)
        k4u, k4v = slope(U + dt * k3u, V + dt * k3v, s_end)
        U = U + (dt / 6.0) * (k1u + 2.0 * k2u + 2.0 * k3u + k4u)
        V = V + (dt / 6.0) * (k1v + 2.0 * k2v + 2.0 * k3v + k4v)
        s_start = s_end
    return U, V
