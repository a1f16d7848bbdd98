"""FP64 CPU oracle for the 2D Fourier-space PDE solves (arXiv:2412.12308).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
reference that the CUDA path is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py`` (its ``cpu_baseline`` leg and
``--impl reference``) may import it; the product package never does, and the
oracle imports nothing from the product.

Every transform here is the direct O(N^2)-per-axis sum of the paper's DFT
definition (Sec. II.B, Eq. DFT and its matrix form Eq. DFT2), evaluated with an
exact integer phase table so that no phase error accumulates; the 2D transform
is the row-then-column order of Sec. II.D.  The solves follow Sec. III: the
Poisson division by -|omega|^2 with the zero mode removed (Eq. Poisson2,
Eq. SolutionPoisson), the diffusion decay (Eq. solCalorFourier) and the wave
closed forms (Eq. OmegaZero, Eq. OmegaNonZero).  All arithmetic is float64 /
complex128.

Pinning status (what fixes each function independently of itself):
  dft.dft1/dft2/idft2      brute-force 2D sum, numpy.fft, round trip, Parseval,
                           single-mode delta                        -> pinned
  solve.omega_axis/omega2  sin*sin manufactured Poisson solution (angular
                           wavenumber), Nyquist-mode closed form    -> pinned
  solve.poisson            mode-sum closed form, zero mean, constant shift
                                                                    -> pinned
  solve.diffusion          single-mode decay, periodic-Gaussian heat kernel,
                           mean conservation, semigroup             -> pinned
  solve.wave               standing-wave closed form, energy, mean,
                           time reversal, period return             -> pinned
  closed_forms.*           cross-checked against each other via the solves
                           above and by finite differences of the PDE -> pinned
  solve.*_source_spectrum  constant-source forms: the PDE residual by time
                           finite differences and a spectral Laplacian from
                           numpy.fft, initial conditions, zero-mode
                           polynomials                               -> pinned
  solve.*_complex          complex fields: a complex plane wave's closed
                           form per operator, and linearity against the
                           (pinned) real solves on re and im parts   -> pinned
  rk4.wave_rk4_spectrum    RK4 of Eq. SystemOfODEsForWaveEquation: the
                           closed-form one-step propagator, 4th-order
                           convergence to the constant-source closed form,
                           the orbiting source's mean mode, the paper's
                           self-convergence factor ~16               -> pinned
"""

from .dft import dft1, dft2, idft2, dft_matrix  # noqa: F401
from .solve import (  # noqa: F401
    omega_axis,
    omega2,
    poisson,
    poisson_spectrum,
    diffusion,
    diffusion_spectrum,
    wave,
    wave_spectrum,
    state_spectrum,
    diffusion_source_spectrum,
    wave_source_spectrum,
    poisson_complex,
    diffusion_complex,
    wave_complex,
)
from .rk4 import wave_rk4_spectrum  # noqa: F401
from . import closed_forms  # noqa: F401
