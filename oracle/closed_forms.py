"""Closed-form solutions used to pin the oracle and to check large grids.

Test infrastructure only.  These are exact solutions of the continuous
problems of Sec. III for inputs whose spectrum the grid represents exactly:

* a sum of Fourier modes  f = sum_m A_m cos(2 pi (kx_m x / Lx + ky_m y / Ly) + phi_m)
  with integer (kx, ky), |kx| <= Nx/2, |ky| <= Ny/2.  Each mode is an
  eigenfunction of the Laplacian with eigenvalue -|omega_m|^2,
  omega_m = 2 pi (kx/Lx, ky/Ly) (the differentiation property of Sec. III.A):
    Poisson   u = sum -A_m / |omega_m|^2 * mode_m            (modes with omega != 0)
    Diffusion u(t) = sum A_m exp(-D |omega_m|^2 t) * mode_m  (Eq. solCalorFourier)
    Wave      u(t) = sum A_m cos(c |omega_m| t) * mode_m     (Eq. OmegaNonZero, g = 0)
              v(t) = sum -A_m c|omega_m| sin(c|omega_m| t) * mode_m
* a periodic Gaussian  A exp(-r^2 / w^2)  (width convention of the examples in
  Sec. III), whose heat-equation evolution is the heat kernel:
    u(t) = A w^2 / (w^2 + 4 D t) * exp(-r^2 / (w^2 + 4 D t)),
  summed over the periodic images.

All evaluation is float64 on the sample points x_j = x0 + j Lx / Nx,
y_k = y0 + k Ly / Ny (right end excluded, as in Eq. discrete_temporal_domain).
"""

import numpy as np

__all__ = [
    "mode_field",
    "poisson_modes",
    "diffusion_modes",
    "wave_modes",
    "gaussian_heat",
]


def _grid(nx, ny, lx, ly, x0=0.0, y0=0.0):
    x = x0 + (lx / nx) * np.arange(nx, dtype=np.float64)
    y = y0 + (ly / ny) * np.arange(ny, dtype=np.float64)
    return x[None, :], y[:, None]


def _mode(kx, ky, phi, nx, ny, lx, ly):
    # Phase reduced with exact integer arithmetic on the index: for x_j = j Lx/Nx
    # the phase 2 pi kx x_j / Lx = 2 pi (kx j mod Nx) / Nx.
    j = np.arange(nx, dtype=np.int64)
    k = np.arange(ny, dtype=np.int64)
    mx = (int(kx) * j) % nx
    my = (int(ky) * k) % ny
    ang = 2.0 * np.pi * (mx[None, :] / nx + my[:, None] / ny) + float(phi)
    return np.cos(ang)


def _omega2_mode(kx, ky, lx, ly):
    return (2.0 * np.pi * kx / lx) ** 2 + (2.0 * np.pi * ky / ly) ** 2


def mode_field(modes, nx, ny, lx, ly, weights=None):
    """sum_m w_m A_m cos(2 pi (kx x/Lx + ky y/Ly) + phi) on the grid with origin 0.

    ``modes`` is a sequence of (kx, ky, A, phi).  ``weights`` (per mode) default to 1.
    """
    out = np.zeros((ny, nx), dtype=np.float64)
    for i, (kx, ky, amp, phi) in enumerate(modes):
        w = 1.0 if weights is None else float(weights[i])
        out += (w * float(amp)) * _mode(kx, ky, phi, nx, ny, lx, ly)
    return out


def poisson_modes(modes, nx, ny, lx, ly):
    """Exact zero-mean Poisson solution for a mode-sum source."""
    weights = []
    for kx, ky, _amp, _phi in modes:
        w2 = _omega2_mode(kx, ky, lx, ly)
        weights.append(0.0 if w2 == 0.0 else -1.0 / w2)
    return mode_field(modes, nx, ny, lx, ly, weights)


def diffusion_modes(modes, D, t, nx, ny, lx, ly):
    """Exact heat-equation solution at time t for a mode-sum initial field."""
    weights = [np.exp(-D * t * _omega2_mode(kx, ky, lx, ly)) for kx, ky, _a, _p in modes]
    return mode_field(modes, nx, ny, lx, ly, weights)


def wave_modes(modes, c, t, nx, ny, lx, ly, want_v=False):
    """Exact standing-wave solution (zero initial velocity) for a mode-sum u0."""
    wu, wv = [], []
    for kx, ky, _a, _p in modes:
        cw = c * np.sqrt(_omega2_mode(kx, ky, lx, ly))
        wu.append(np.cos(cw * t))
        wv.append(-cw * np.sin(cw * t))
    u = mode_field(modes, nx, ny, lx, ly, wu)
    if not want_v:
        return u
    return u, mode_field(modes, nx, ny, lx, ly, wv)


def gaussian_heat(blobs, D, t, nx, ny, lx, ly, x0=0.0, y0=0.0, images=2):
    """Heat-kernel evolution of a sum of periodic Gaussians A exp(-r^2/w^2).

    ``blobs`` is a sequence of (cx, cy, w, A).  The periodic field is the sum
    over images n in [-images, images]^2; at t = 0 this is the initial field.
    """
    x, y = _grid(nx, ny, lx, ly, x0, y0)
    # exp(-r^2/s2) = exp(-dx^2/s2) exp(-dy^2/s2), and the sum over the image
    # lattice factors the same way, so each blob is the outer product of its
    # x and y image sums: u = sum_blob pref * Y_blob X_blob^T
    xs = np.zeros((len(blobs), nx), dtype=np.float64)
    ys = np.zeros((ny, len(blobs)), dtype=np.float64)
    for i, (cx, cy, w, amp) in enumerate(blobs):
        s2 = float(w) ** 2 + 4.0 * float(D) * float(t)
        pref = float(amp) * float(w) ** 2 / s2
        for ix in range(-images, images + 1):
            xs[i] += np.exp(-((x[0] - cx - ix * lx) ** 2) / s2)
        for iy in range(-images, images + 1):
            ys[:, i] += np.exp(-((y[:, 0] - cy - iy * ly) ** 2) / s2)
        xs[i] *= pref
    return ys @ xs
