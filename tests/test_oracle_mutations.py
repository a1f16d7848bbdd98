"""Planted mistakes in the oracle must trip at least one pin (no GPU).

Each mutant replaces one oracle function with a plausibly wrong version (a
dropped term, a wrong sign or index, a transposed operand) for the duration of
the test only, on the CPU, and the pins are re-run.  A mutant that no pin
catches would mean the pins do not constrain that part of the oracle.
"""

import numpy as np
import pytest

import oracle
import oracle.dft as odft
import oracle.solve as osolve
from tests import oracle_pins as pins


def _no_shift_axis(n, length):
    return (2.0 * np.pi / float(length)) * np.arange(n, dtype=np.float64)


def _no_two_pi_axis(n, length):
    a = np.arange(n)
    ap = np.where(2 * a <= n, a, a - n)
    return ap.astype(np.float64) / float(length)


def _nyquist_negative_dropped_axis(n, length):
    # maps the Nyquist index to 0 (a common off-by-one: a < n/2 kept, else shifted by n)
    a = np.arange(n)
    ap = np.where(2 * a < n, a, a - n)
    ap = np.where(2 * a == n, 0, ap)
    return (2.0 * np.pi / float(length)) * ap.astype(np.float64)


def _poisson_sign(F, lx, ly):
    ny, nx = F.shape
    w2 = osolve.omega2(nx, ny, lx, ly)
    U = np.zeros_like(F)
    nz = w2 > 0
    U[nz] = F[nz] / w2[nz]
    return U


def _poisson_keep_mean(F, lx, ly):
    ny, nx = F.shape
    w2 = osolve.omega2(nx, ny, lx, ly)
    U = F.copy()
    nz = w2 > 0
    U[nz] = -F[nz] / w2[nz]
    return U


def _diffusion_omega_not_squared(F, D, t, lx, ly):
    ny, nx = F.shape
    w = np.sqrt(osolve.omega2(nx, ny, lx, ly))
    return F * np.exp(-D * t * w)


def _wave_g_times_omega(F, G, c, t, lx, ly):
    ny, nx = F.shape
    cw = c * np.sqrt(osolve.omega2(nx, ny, lx, ly))
    U = F * np.cos(cw * t)
    V = -cw * np.sin(cw * t) * F
    if G is not None:
        U = U + G * np.sin(cw * t) * cw
        V = V + G * np.cos(cw * t)
    return U, V


def _wave_v_sign(F, G, c, t, lx, ly):
    U, V = _ORIG_WAVE(F, G, c, t, lx, ly)
    return U, -V


def _idft2_unnormalised(P, sign=+1):
    q = odft.dft1(P, axis=1, sign=sign)
    return odft.dft1(q, axis=0, sign=sign)


def _dft2_transposed(p, sign=-1):
    px = odft.dft1(np.asarray(p), axis=0, sign=sign)
    return odft.dft1(px, axis=1, sign=sign).T.copy() if p.shape[0] == p.shape[1] else \
        odft.dft1(px, axis=1, sign=sign)[::-1].copy()


def _dft1_sign_ignored(x, axis=-1, sign=-1):
    return _ORIG_DFT1(x, axis=axis, sign=+1)


def _diffusion_source_gain_sign(F, S, D, t, lx, ly):
    ny, nx = F.shape
    lam = D * osolve.omega2(nx, ny, lx, ly)
    gain = np.where(lam > 0, np.expm1(-lam * t) / np.where(lam > 0, lam, 1.0), t)
    return F * np.exp(-lam * t) + S * gain


def _wave_source_printed(F, G, S, c, t, lx, ly):
    # the particular term subtracted inside the cosine but not added back
    U, V = osolve.wave_spectrum(F, G, c, t, lx, ly)
    ny, nx = F.shape
    cw = c * np.sqrt(osolve.omega2(nx, ny, lx, ly))
    cw2 = np.where(cw > 0, cw * cw, 1.0)
    pu = np.where(cw > 0, -np.cos(cw * t) / cw2, 0.5 * t * t)
    pv = np.where(cw > 0, np.sin(cw * t) / np.where(cw > 0, cw, 1.0), t)
    return U + S * pu, V + S * pv


def _rk4_variant(weights=(1, 2, 2, 1), src_stage=("start", "mid", "mid", "end"), k2_step=0.5):
    import oracle.rk4 as ork

    def fn(F, G, source, c, t0, dt, nsteps, lx, ly, sign=-1):
        F = np.asarray(F, dtype=np.complex128)
        ny, nx = F.shape
        w2 = float(c) ** 2 * osolve.omega2(nx, ny, lx, ly)
        U = F.copy()
        V = np.zeros_like(U) if G is None else np.asarray(G, dtype=np.complex128).copy()

        def S(t):
            return np.zeros_like(U) if source is None else ork.dft2(np.asarray(source(t), float), sign=sign)
        for k in range(int(nsteps)):
            t = t0 + k * dt
            at = {"start": S(t), "mid": S(t + dt / 2), "end": S(t + dt)}
            s1, s2, s3, s4 = (at[x] for x in src_stage)
            k1u, k1v = V, -w2 * U + s1
            k2u, k2v = V + k2_step * dt * k1v, -w2 * (U + k2_step * dt * k1u) + s2
            k3u, k3v = V + 0.5 * dt * k2v, -w2 * (U + 0.5 * dt * k2u) + s3
            k4u, k4v = V + dt * k3v, -w2 * (U + dt * k3u) + s4
            a, b, cc, d = weights
            U = U + dt / 6 * (a * k1u + b * k2u + cc * k3u + d * k4u)
            V = V + dt / 6 * (a * k1v + b * k2v + cc * k3v + d * k4v)
        return U, V
    return fn


def _poisson_complex_real_only(f, lx, ly, sign=-1):
    # drops the imaginary part of the input (a real-only solve)
    F = odft.dft2(np.real(np.asarray(f)).astype(np.complex128), sign=sign)
    return odft.idft2(osolve.poisson_spectrum(F, lx, ly), sign=-sign)


def _diffusion_complex_half_spectrum(u0, D, t, lx, ly, sign=-1):
    # treats negative x frequencies as positive-index frequencies (no shift)
    F = odft.dft2(np.asarray(u0, dtype=np.complex128), sign=sign)
    ny, nx = F.shape
    w2 = (2 * np.pi * np.arange(nx) / lx)[None, :] ** 2 + osolve.omega_axis(ny, ly)[:, None] ** 2
    return odft.idft2(F * np.exp(-D * t * w2), sign=-sign)


_ORIG_DFT1 = odft.dft1
_ORIG_WAVE = osolve.wave_spectrum

MUTANTS = {
    "omega_no_shift": [(osolve, "omega_axis", _no_shift_axis)],
    "omega_no_2pi": [(osolve, "omega_axis", _no_two_pi_axis)],
    "omega_nyquist_zero": [(osolve, "omega_axis", _nyquist_negative_dropped_axis)],
    "poisson_sign": [(osolve, "poisson_spectrum", _poisson_sign)],
    "poisson_keep_mean": [(osolve, "poisson_spectrum", _poisson_keep_mean)],
    "diffusion_omega_not_squared": [(osolve, "diffusion_spectrum", _diffusion_omega_not_squared)],
    "wave_g_times_omega": [(osolve, "wave_spectrum", _wave_g_times_omega)],
    "wave_v_sign": [(osolve, "wave_spectrum", _wave_v_sign)],
    "idft2_unnormalised": [(osolve, "idft2", _idft2_unnormalised), (oracle, "idft2", _idft2_unnormalised)],
    "dft2_transposed": [(osolve, "dft2", _dft2_transposed), (oracle, "dft2", _dft2_transposed)],
    "dft1_sign_ignored": [(odft, "dft1", _dft1_sign_ignored), (oracle, "dft1", _dft1_sign_ignored)],
    "diffusion_source_gain_sign": [(oracle, "diffusion_source_spectrum", _diffusion_source_gain_sign)],
    "wave_source_printed_form": [(oracle, "wave_source_spectrum", _wave_source_printed)],
    "complex_real_only": [(oracle, "poisson_complex", _poisson_complex_real_only)],
    "complex_no_shift": [(oracle, "diffusion_complex", _diffusion_complex_half_spectrum)],
    "rk4_weights": [(oracle, "wave_rk4_spectrum", _rk4_variant(weights=(1, 1, 2, 2)))],
    "rk4_source_at_step_start": [(oracle, "wave_rk4_spectrum",
                                  _rk4_variant(src_stage=("start", "start", "start", "start")))],
    "rk4_k2_full_step": [(oracle, "wave_rk4_spectrum", _rk4_variant(k2_step=1.0))],
}


def _failing_pins():
    failed = []
    for name, (fn, bound) in pins.PINS.items():
        try:
            err = fn()
        except Exception:  # a crash counts as caught
            failed.append(name)
            continue
        if not (err <= bound):
            failed.append(name)
    return failed


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_mutant_is_caught(mutant, monkeypatch):
    for mod, attr, repl in MUTANTS[mutant]:
        monkeypatch.setattr(mod, attr, repl)
    failed = _failing_pins()
    assert failed, f"mutant {mutant} passed every pin"
