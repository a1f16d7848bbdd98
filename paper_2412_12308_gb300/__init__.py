"""GB300-native 2D Fourier-space PDE solves (arXiv:2412.12308).

The compute path is the C-ABI library ``libfsolve.so`` (hand-written CUDA for
sm_103a); ``fsolve`` is its thin ctypes binding.  Importing this package does
not load the library; the first call through ``fsolve`` does, and fails loudly
if it has not been built.
"""

__all__ = ["fsolve", "workloads"]
