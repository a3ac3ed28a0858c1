"""Discrete Fourier transforms for the dynamic Fourier method (oracle).

Sec. II G switches the wavepacket between the position and the momentum
representation with fast Fourier transforms.  The paper does not fix a sign
or normalisation; this oracle uses the forward transform
X_k = sum_j x_j exp(-2 pi i j k / N) and the inverse x_j = (1/N) sum_k X_k
exp(+2 pi i j k / N).  The kinetic operator T(p) is even in p, so results of
the propagation do not depend on that choice.

``fft_axis`` is a textbook iterative radix-2 (decimation in time, bit-reversed
input) transform along one axis of an N-d array; ``dft_axis`` is the direct
O(N^2) sum used to pin it on small sizes.
"""
from __future__ import annotations

import numpy as np


def _bit_reverse(N: int) -> np.ndarray:
    bits = N.bit_length() - 1
    idx = np.arange(N)
    rev = np.zeros(N, dtype=np.int64)
    for b in range(bits):
        rev |= ((idx >> b) & 1) << (bits - 1 - b)
    return rev


def fft_axis(x: np.ndarray, axis: int, inverse: bool = False) -> np.ndarray:
    """Radix-2 FFT of ``x`` along ``axis`` (length a power of two).  The
    inverse includes the 1/N factor."""
    x = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, -1)
    N = x.shape[-1]
    if N & (N - 1):
        raise ValueError("radix-2 FFT needs a power-of-two length")
    y = x[..., _bit_reverse(N)].copy()
    sign = 1.0 if inverse else -1.0
    size = 2
    while size <= N:
        half = size // 2
        w = np.exp(sign * 2j * np.pi * np.arange(half) / size)
        y = y.reshape(y.shape[:-1] + (N // size, size))
        top = y[..., :half].copy()
        bot = y[..., half:] * w
        y[..., :half] = top + bot
        y[..., half:] = top - bot
        y = y.reshape(y.shape[:-2] + (N,))
        size *= 2
    if inverse:
        y = y / N
    return np.moveaxis(y, -1, axis)


def dft_axis(x: np.ndarray, axis: int, inverse: bool = False) -> np.ndarray:
    """Direct DFT along ``axis`` by the defining sum (small N only)."""
    x = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, -1)
    N = x.shape[-1]
    sign = 1.0 if inverse else -1.0
    j = np.arange(N)
    F = np.exp(sign * 2j * np.pi * np.outer(j, j) / N)
    y = x @ F.T
    if inverse:
        y = y / N
    return np.moveaxis(y, -1, axis)


def fftn_grid(psi: np.ndarray, inverse: bool = False, dft: bool = False) -> np.ndarray:
    """Transform every surface of psi[s, i0, ..., i_{D-1}] over all grid axes."""
    f = dft_axis if dft else fft_axis
    out = psi
    for axis in range(1, psi.ndim):
        out = f(out, axis, inverse)
    return out
