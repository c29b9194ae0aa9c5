"""GB300 (sm_103a) library for the fast Fourier transform on SO(3).

The forward transform (FSOFT) and its inverse (iFSOFT) of Kostelec and
Rockmore, as reviewed and parallelised in Lux, Wuelker, Chirikjian,
"Parallelization of the FFT on SO(3)" (arXiv:1808.00896): a 2-D FFT of every
beta slice and the discrete Wigner transform per order pair (m, m'), both
in hand-written CUDA kernels (cuFFT covers the FFT sizes that are not powers
of two) that generate the Wigner-d functions on the fly.

Importing this package does not load the CUDA library; the first plan does,
and fails loudly if it has not been built.
"""

__all__ = ["Plan", "num_coeffs", "soft_forward", "soft_inverse", "batched_inverse", "batched_forward",
           "batched_correlate"]


def __getattr__(name):
    if name in __all__:
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
