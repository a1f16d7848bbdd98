"""Fourier-space solves of Sec. III in float64 (test infrastructure only).

Every solve is: forward 2D DFT (Sec. II.D), a pointwise operator on the FULL
complex spectrum (no Hermitian half-spectrum shortcut, so the CUDA path's real
to half-complex packing is checked independently), and the inverse 2D DFT.

Wavenumbers (Sec. II.D, frequency grid k_a = a / (N dx); Sec. II.B, the index
shift for a > N/2):  the DFT index a maps to the signed index a' = a for
a <= N/2 and a - N for a > N/2, and the angular wavenumber is
omega = 2 pi a' / L (L = N dx).  The angular (2 pi) form follows from the
differentiation property of Sec. III.A, F{d^k u/dx^k} = (-i omega)^k F{u},
with the 2 pi in the exponent of Eq. FT.  The Nyquist index a = N/2 is kept
(|omega| = pi N / L); every multiplier below is even in omega, so its sign
never matters.

Operators (all multipliers real and even in (omega_x, omega_y)):
  Poisson   (Eq. PoissonFourier, Eq. Poisson2, Eq. SolutionPoisson):
            U = -F / |omega|^2 and U(0,0) = 0, i.e. the zero-mean solution of
            lap u = f - mean(f).
  Diffusion (Eq. DiffusionIVPFS with s = 0, Eq. solCalorFourier, with a
            diffusivity D by rescaling time as done for c in Sec. III.C):
            U(t) = F exp(-D |omega|^2 t); the omega = 0 mode keeps F.
  Wave      (Eq. WaveEquationFourierSpace with s = 0; Eq. OmegaZero,
            Eq. OmegaNonZero with t -> c t):
            U(t) = F cos(c|omega|t) + G sin(c|omega|t) / (c|omega|),
            U(t) = F + G t at omega = 0;
            the velocity V = dU/dt of the first-order system
            (Eq. SystemOfODEsForWaveEquation):
            V(t) = -c|omega| F sin(c|omega|t) + G cos(c|omega|t).
"""

import numpy as np

from .dft import dft2, idft2

__all__ = [
    "poisson_complex",
    "diffusion_complex",
    "wave_complex",
    "diffusion_source_spectrum",
    "wave_source_spectrum",
    "omega_axis",
    "omega2",
    "state_spectrum",
    "poisson_spectrum",
    "diffusion_spectrum",
    "wave_spectrum",
    "poisson",
    "diffusion",
    "wave",
]


def omega_axis(n, length):
    """Angular wavenumbers 2 pi a' / L for DFT indices a = 0..n-1.

    a' = a for a <= n/2, a - n for a > n/2 (the frequency shift of Sec. II.B);
    for even n the Nyquist index a = n/2 is kept with a' = +n/2.
    """
    a = np.arange(n, dtype=np.int64)
    ap = np.where(2 * a <= n, a, a - n)
    return (2.0 * np.pi / float(length)) * ap.astype(np.float64)


def omega2(nx, ny, lx, ly):
    """|omega|^2 on the [Ny][Nx] spectrum grid: omega_x(a)^2 + omega_y(b)^2."""
    wx = omega_axis(nx, lx)
    wy = omega_axis(ny, ly)
    return wy[:, None] ** 2 + wx[None, :] ** 2


def _real_part(z, what):
    """Take the real part of an inverse transform, checking it is real.

    For real input and real, even multipliers the exact result is real; the
    imaginary part is pure round-off.  A large imaginary part means an
    operator broke the Hermitian symmetry -- a bug in the oracle.
    """
    re = z.real
    scale = max(1.0, float(np.max(np.abs(re))) if re.size else 1.0)
    im = float(np.max(np.abs(z.imag))) if z.size else 0.0
    if im > 1e-9 * scale:
        raise AssertionError(f"{what}: imaginary residue {im:.3e} (scale {scale:.3e})")
    return re


def state_spectrum(field, sign=-1):
    """Forward 2D DFT of a real field: the kept spectrum of an initial state."""
    return dft2(np.asarray(field, dtype=np.float64), sign=sign)


def poisson_spectrum(F, lx, ly):
    """U = -F / |omega|^2 with the zero mode set to 0 (Eq. SolutionPoisson)."""
    ny, nx = F.shape
    w2 = omega2(nx, ny, lx, ly)
    U = np.zeros_like(F)
    nz = w2 > 0.0
    U[nz] = -F[nz] / w2[nz]
    U[0, 0] = 0.0  # Eq. Poisson2: the mean of the source is removed
    return U


def diffusion_spectrum(F, D, t, lx, ly):
    """U(t) = F exp(-D |omega|^2 t); omega = 0 keeps F (Eq. solCalorFourier)."""
    ny, nx = F.shape
    w2 = omega2(nx, ny, lx, ly)
    fac = np.exp(-float(D) * float(t) * w2)
    fac[w2 == 0.0] = 1.0
    return F * fac


def wave_spectrum(F, G, c, t, lx, ly):
    """(U(t), V(t)) of the free wave equation per mode (Eq. OmegaZero, Eq. OmegaNonZero).

    ``G`` may be None (zero initial velocity).
    """
    ny, nx = F.shape
    w = np.sqrt(omega2(nx, ny, lx, ly))
    cw = float(c) * w
    th = cw * float(t)
    cos = np.cos(th)
    sin = np.sin(th)
    U = F * cos
    V = -cw * sin * F
    if G is not None:
        nz = cw > 0.0
        sinc_t = np.empty_like(th)
        sinc_t[nz] = sin[nz] / cw[nz]
        sinc_t[~nz] = float(t)  # Eq. OmegaZero: u = f + g t at omega = 0
        U = U + G * sinc_t
        V = V + G * cos
    return U, V


def poisson(f, lx, ly, sign=-1):
    """Zero-mean solution u of lap u = f - mean(f) on the periodic [Ny][Nx] grid."""
    F = dft2(np.asarray(f, dtype=np.float64), sign=sign)
    U = poisson_spectrum(F, lx, ly)
    return _real_part(idft2(U, sign=-sign), "poisson")


def diffusion(u0, D, t, lx, ly, sign=-1):
    """u(t) of u_t = D lap u from u(0) = u0 (Eq. solCalorFourier)."""
    F = dft2(np.asarray(u0, dtype=np.float64), sign=sign)
    U = diffusion_spectrum(F, D, t, lx, ly)
    return _real_part(idft2(U, sign=-sign), "diffusion")


def wave(u0, v0, c, t, lx, ly, sign=-1, want_v=False):
    """u(t) (and optionally v = u_t(t)) of u_tt = c^2 lap u from (u0, v0).

    ``v0`` may be None (zero initial velocity).
    """
    F = dft2(np.asarray(u0, dtype=np.float64), sign=sign)
    G = None if v0 is None else dft2(np.asarray(v0, dtype=np.float64), sign=sign)
    U, V = wave_spectrum(F, G, c, t, lx, ly)
    u = _real_part(idft2(U, sign=-sign), "wave u")
    if not want_v:
        return u
    v = _real_part(idft2(V, sign=-sign), "wave v")
    return u, v


# ---------------------------------------------------------------- complex fields
# Sec. II.B lets the samples p_jk be complex; the solves are the same
# spectral operators on the full spectrum, returned as complex fields.
def poisson_complex(f, lx, ly, sign=-1):
    """Zero-mean solution of lap u = f - mean(f) for a complex field f."""
    F = dft2(np.asarray(f, dtype=np.complex128), sign=sign)
    return idft2(poisson_spectrum(F, lx, ly), sign=-sign)


def diffusion_complex(u0, D, t, lx, ly, sign=-1):
    F = dft2(np.asarray(u0, dtype=np.complex128), sign=sign)
    return idft2(diffusion_spectrum(F, D, t, lx, ly), sign=-sign)


def wave_complex(u0, v0, c, t, lx, ly, sign=-1):
    F = dft2(np.asarray(u0, dtype=np.complex128), sign=sign)
    G = None if v0 is None else dft2(np.asarray(v0, dtype=np.complex128), sign=sign)
    U, _ = wave_spectrum(F, G, c, t, lx, ly)
    return idft2(U, sign=-sign)


# ---------------------------------------------------------------- constant sources
# Eq. DiffusionIVPFS and Eq. WaveEquationFourierSpace with a time-independent
# source s.  Each mode is a linear ODE with constant forcing:
#   diffusion  dU/dt = -D w^2 U + S      ->  U = F E + S (1 - E) / (D w^2),
#              E = exp(-D w^2 t);  w = 0: U = F + S t
#   wave       U'' + c^2 w^2 U = S       ->  U = S/(c w)^2 + (F - S/(c w)^2) cos(c w t)
#                                                + G sin(c w t) / (c w);
#              w = 0: U = F + G t + S t^2 / 2  (Eq. OmegaZero)
# The printed Eq. OmegaNonZero omits the particular term S/w^2 added outside the
# cosine; the form above satisfies the ODE and the initial conditions.
def diffusion_source_spectrum(F, S, D, t, lx, ly):
    ny, nx = F.shape
    w2 = omega2(nx, ny, lx, ly)
    lam = float(D) * w2
    E = np.exp(-lam * float(t))
    gain = np.empty_like(w2)
    nz = lam > 0.0
    gain[nz] = -np.expm1(-lam[nz] * float(t)) / lam[nz]
    gain[~nz] = float(t)
    return F * E + S * gain


def wave_source_spectrum(F, G, S, c, t, lx, ly):
    """(U(t), V(t)) with initial velocity spectrum G (or None) and source S."""
    U, V = wave_spectrum(F, G, c, t, lx, ly)
    ny, nx = F.shape
    cw = float(c) * np.sqrt(omega2(nx, ny, lx, ly))
    th = cw * float(t)
    pu = np.empty_like(cw)
    pv = np.empty_like(cw)
    nz = cw > 0.0
    pu[nz] = 2.0 * np.sin(0.5 * th[nz]) ** 2 / cw[nz] ** 2  # (1 - cos th) / (c w)^2
    pv[nz] = np.sin(th[nz]) / cw[nz]
    pu[~nz] = 0.5 * float(t) ** 2
    pv[~nz] = float(t)
    return U + S * pu, V + S * pv
