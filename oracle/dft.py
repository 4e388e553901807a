"""Discrete Fourier transforms of the oracle (TEST INFRASTRUCTURE ONLY).

The one place where the oracle calls a library routine for a DFT: scipy.fft
(pocketfft).  Same definition and signatures as numpy.fft: forward sign -1,
unnormalised; the inverse divides by the number of points; rfftn/irfftn keep
the half spectrum of the last axis.  The thread count is a setting (default 1,
or the environment variable ORACLE_FFT_WORKERS, or set_workers): it only
divides the independent one-dimensional transforms among threads, so every
result is the same for any count.
"""
from __future__ import annotations

import os

import scipy.fft as _sf

_workers = max(1, int(os.environ.get("ORACLE_FFT_WORKERS", "1")))


def set_workers(n: int) -> None:
    """Threads the transforms may use (n >= 1)."""
    global _workers
    _workers = max(1, int(n))


def workers() -> int:
    return _workers


def rfftn(x, s=None, axes=None):
    return _sf.rfftn(x, s=s, axes=axes, workers=_workers)


def irfftn(x, s=None, axes=None):
    return _sf.irfftn(x, s=s, axes=axes, workers=_workers)


def fft2(x):
    return _sf.fft2(x, workers=_workers)
