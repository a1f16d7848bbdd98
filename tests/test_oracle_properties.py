"""Property-based checks of the oracle on random tiny grids (CPU).

The fixed pins of test_oracle.py are complemented here by randomly drawn
shapes (odd and even, nx != ny), domains and parameters, each checked against
something other than the oracle itself: the brute-force 2D sum of Eq. 2D_DFT,
numpy's FFT (a library routine), and identities the mathematics fixes
(the spectral Laplacian of a Poisson solution is the zero-mean source; the
diffusion semigroup; wave time reversal).
"""

import math

import numpy as np
import pytest

import oracle

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")
given, settings = hyp.given, hyp.settings

SET = settings(max_examples=40, deadline=None, derandomize=True)
dims = st.integers(min_value=1, max_value=9)
seeds = st.integers(min_value=0, max_value=2**31 - 1)
lengths = st.floats(min_value=0.5, max_value=7.0)


def _field(seed, ny, nx, complex_=True):
    rng = np.random.default_rng(seed)
    z = rng.standard_normal((ny, nx))
    return z + 1j * rng.standard_normal((ny, nx)) if complex_ else z


def _brute_dft2(p, sign):
    ny, nx = p.shape
    out = np.zeros((ny, nx), complex)
    for b in range(ny):
        for a in range(nx):
            s = 0j
            for k in range(ny):
                for j in range(nx):
                    s += p[k, j] * np.exp(sign * 2j * math.pi * (a * j / nx + b * k / ny))
            out[b, a] = s
    return out


@SET
@given(ny=dims, nx=dims, seed=seeds, sign=st.sampled_from([-1, 1]))
def test_dft2_equals_the_brute_force_sum(ny, nx, seed, sign):
    p = _field(seed, ny, nx)
    got = oracle.dft2(p, sign=sign)
    want = _brute_dft2(p, sign)
    assert np.allclose(got, want, rtol=0, atol=1e-11 * max(1.0, np.abs(want).max()))


@SET
@given(ny=st.integers(1, 40), nx=st.integers(1, 40), seed=seeds)
def test_dft2_equals_numpy_fft_and_round_trips(ny, nx, seed):
    p = _field(seed, ny, nx)
    P = oracle.dft2(p)
    assert np.allclose(P, np.fft.fft2(p), rtol=0, atol=1e-11 * max(1.0, np.abs(P).max()))
    assert np.allclose(oracle.idft2(P), p, rtol=0, atol=1e-12 * max(1.0, np.abs(p).max()))


def _spectral_laplacian(u, lx, ly):
    ny, nx = u.shape
    kx = 2 * math.pi * np.fft.fftfreq(nx, d=lx / nx)
    ky = 2 * math.pi * np.fft.fftfreq(ny, d=ly / ny)
    return np.real(np.fft.ifft2(-(kx[None, :] ** 2 + ky[:, None] ** 2) * np.fft.fft2(u)))


@SET
@given(n=st.sampled_from([2, 4, 6, 8, 10, 12, 16]), m=st.sampled_from([2, 4, 6, 8, 12]), seed=seeds,
       lx=lengths, ly=lengths)
def test_poisson_solution_satisfies_the_equation(n, m, seed, lx, ly):
    """Even sizes with the Nyquist modes removed from the source (their
    derivative is not defined by a real spectral Laplacian), so the check is
    exact: lap u = f - mean(f), and u has zero mean."""
    rng = np.random.default_rng(seed)
    F = np.fft.fft2(rng.standard_normal((m, n)))
    F[m // 2, :] = 0.0
    F[:, n // 2] = 0.0
    f = np.real(np.fft.ifft2(F))
    u = oracle.poisson(f, lx, ly)
    assert abs(u.mean()) <= 1e-12 * max(1.0, np.abs(u).max())
    lap = _spectral_laplacian(u, lx, ly)
    assert np.allclose(lap, f - f.mean(), rtol=0, atol=1e-10 * max(1.0, np.abs(f).max()))


@SET
@given(ny=st.integers(2, 12), nx=st.integers(2, 12), seed=seeds, lx=lengths, ly=lengths,
       D=st.floats(0.001, 0.5), t1=st.floats(0.0, 1.0), t2=st.floats(0.0, 1.0))
def test_diffusion_semigroup(ny, nx, seed, lx, ly, D, t1, t2):
    u0 = _field(seed, ny, nx, complex_=False)
    a = oracle.diffusion(oracle.diffusion(u0, D, t1, lx, ly), D, t2, lx, ly)
    b = oracle.diffusion(u0, D, t1 + t2, lx, ly)
    assert np.allclose(a, b, rtol=0, atol=1e-11 * max(1.0, np.abs(u0).max()))


@SET
@given(ny=st.integers(2, 12), nx=st.integers(2, 12), seed=seeds, lx=lengths, ly=lengths,
       c=st.floats(0.3, 2.0), t=st.floats(0.0, 2.0))
def test_wave_time_reversal(ny, nx, seed, lx, ly, c, t):
    rng = np.random.default_rng(seed)
    u0, v0 = rng.standard_normal((ny, nx)), rng.standard_normal((ny, nx))
    u1, v1 = oracle.wave(u0, v0, c, t, lx, ly, want_v=True)
    u2, v2 = oracle.wave(u1, v1, c, -t, lx, ly, want_v=True)
    scale = max(1.0, np.abs(u0).max(), np.abs(v0).max())
    assert np.allclose(u2, u0, rtol=0, atol=1e-10 * scale)
    assert np.allclose(v2, v0, rtol=0, atol=1e-10 * scale)
