"""Direct discrete Fourier transforms in float64 (test infrastructure only).

Sec. II.B defines the length-N DFT as a plain sum over samples (Eq. DFT), i.e.
a product with the N x N matrix W of powers of omega_N (Eq. DFT2), and the
inverse as the conjugate sum divided by N (the W^{-1} = W^dagger / N property
stated after Eq. DFT2).  Sec. II.D computes the 2D transform as N_y length-N_x
transforms along x followed by N_x length-N_y transforms along y.

Sign convention: the paper writes the exponent as +2 pi i in Eq. FT, Eq. DFT and
Eq. 2D_DFT but as -2 pi i in the separable form of Sec. II.D.  Every spectral
multiplier used by the solves is even in omega, so the solutions do not depend
on the choice; the oracle takes ``sign=-1`` (the separable form) as forward and
``sign=+1`` as inverse, and both choices are exercised by the tests.

Implementation: W[a, j] = exp(sign * 2 pi i * ((a*j) mod N) / N).  The product
a*j is reduced modulo N in exact integer arithmetic before the angle is formed,
so every entry is cos/sin of 2 pi m / N with 0 <= m < N -- no phase growth for
large N.  The matrix product itself is a library matmul (numpy / BLAS), which
is a plain step of the definition.
"""

import numpy as np

__all__ = ["dft_matrix", "dft1", "dft2", "idft2"]

_W_CACHE = {}


def dft_matrix(n, sign=-1):
    """The N x N matrix W of Eq. DFT2 with entries omega^(a*j), omega = e^{sign*2 pi i/N}.

    Built from the exact integer table (a*j) mod N (see module docstring).
    """
    if n < 1:
        raise ValueError("DFT length must be >= 1")
    if sign not in (-1, 1):
        raise ValueError("sign must be -1 or +1")
    key = (n, sign)
    w = _W_CACHE.get(key)
    if w is None:
        idx = np.arange(n, dtype=np.int64)
        m = np.outer(idx, idx) % n  # exact phase index, 0 <= m < n
        ang = (2.0 * np.pi / n) * np.arange(n, dtype=np.float64)
        c = np.cos(ang)
        s = np.sin(ang)
        w = c[m] + (sign * 1j) * s[m]
        if n <= 4096:
            _W_CACHE[key] = w
    return w


def dft1(x, axis=-1, sign=-1):
    """Unnormalised 1D DFT along ``axis``: X_a = sum_j x_j omega_N^{a j} (Eq. DFT)."""
    x = np.asarray(x)
    n = x.shape[axis]
    w = dft_matrix(n, sign)
    xm = np.moveaxis(x.astype(np.complex128, copy=False), axis, -1)
    out = xm @ w.T  # out[..., a] = sum_j x[..., j] * W[a, j]
    return np.moveaxis(out, -1, axis)


def dft2(p, sign=-1):
    """2D DFT of a field p[k, j] = p(x_j, y_k) (layout [Ny][Nx], x fastest).

    Rows first (length-Nx transforms along x for every y index, the bracketed
    sum of Sec. II.D), then columns (length-Ny transforms along y).
    """
    p = np.asarray(p)
    if p.ndim != 2:
        raise ValueError("dft2 expects a 2D array [Ny, Nx]")
    px = dft1(p, axis=1, sign=sign)  # P^x_{a k}
    return dft1(px, axis=0, sign=sign)  # P_{a b}, stored [b, a]


def idft2(P, sign=+1):
    """Inverse 2D DFT: conjugate-sign sums along x then y, times 1/(Nx Ny).

    Follows the inverse formula after Eq. DFT2 applied per axis.
    """
    P = np.asarray(P)
    ny, nx = P.shape
    q = dft1(P, axis=1, sign=sign)
    q = dft1(q, axis=0, sign=sign)
    return q / float(nx * ny)
