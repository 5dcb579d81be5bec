"""GB300-native batched complex FFT library (sm_103a).

Implements the DFT problem dft(N, V, I, O) of Johnson & Frigo, "Implementing
FFTs in Practice" (sec. 4.1) with Cooley-Tukey Stockham passes built from
generated radix codelets, Bluestein for large primes and a measuring planner.
The compute path is the CUDA library ``libgbfft.so`` behind the C ABI in
``include/gbfft.h``; ``gbfft`` is its ctypes binding.
"""
from . import gbfft  # noqa: F401
from .gbfft import Plan  # noqa: F401

__all__ = ["gbfft", "Plan"]
