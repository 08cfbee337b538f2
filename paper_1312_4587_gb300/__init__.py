"""GB300-native FFTPL objective-gradient library.

The CUDA kernels live in ``csrc/`` and are built into ``libfftpl.so`` (C ABI
in ``include/fftpl.h``).  ``fftpl`` is the thin ctypes binding with the C
names; ``autograd`` wraps the density energy as a torch.autograd.Function;
``serve`` runs streams of placement jobs.
"""
from . import fftpl  # noqa: F401

__all__ = ["fftpl"]
