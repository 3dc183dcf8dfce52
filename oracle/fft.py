"""The oracle's own discrete Fourier transform (Sec. 2.3, Eq. dft).

Forward:  F_k = sum_n f_n exp(-2 pi i k n / N)           (unnormalised)
Inverse:  f_n = (1/N) sum_k F_k exp(+2 pi i k n / N)

Implemented as a textbook recursive radix-2 decimation-in-time split
(Cooley-Tukey): F_k = E_k + w^k O_k, F_{k+N/2} = E_k - w^k O_k with E/O the
transforms of the even/odd samples and w = exp(-2 pi i / N).  When the length
is odd the recursion stops and the DFT sum is evaluated directly, so lengths of
the form m * 2^k (m odd) are supported.  Multi-dimensional transforms are
successive 1D transforms along each axis (Sec. 2.3, the pencil procedure).

Pinned in tests/test_oracle_transforms.py against the O(N^2) definition,
numpy.fft, Parseval's identity and inverse(forward(x)) = x.
"""
from __future__ import annotations

import numpy as np


def _direct_dft_last(x: np.ndarray, sign: int) -> np.ndarray:
    n = x.shape[-1]
    j = np.arange(n)
    w = np.exp(sign * 2j * np.pi * np.outer(j, j) / n)
    return x @ w


def _fft_last(x: np.ndarray, sign: int) -> np.ndarray:
    n = x.shape[-1]
    if n == 1:
        return x.astype(np.complex128, copy=True)
    if n % 2 == 1:
        return _direct_dft_last(x.astype(np.complex128), sign)
    even = _fft_last(x[..., 0::2], sign)
    odd = _fft_last(x[..., 1::2], sign)
    k = np.arange(n // 2)
    tw = np.exp(sign * 2j * np.pi * k / n)
    t = tw * odd
    return np.concatenate([even + t, even - t], axis=-1)


def dft(x: np.ndarray, axis: int = -1) -> np.ndarray:
    """Unnormalised forward DFT along one axis."""
    xm = np.moveaxis(np.asarray(x), axis, -1)
    return np.moveaxis(_fft_last(xm, -1), -1, axis)


def idft(x: np.ndarray, axis: int = -1) -> np.ndarray:
    """Inverse DFT along one axis, including the 1/N factor."""
    xm = np.moveaxis(np.asarray(x), axis, -1)
    n = xm.shape[-1]
    return np.moveaxis(_fft_last(xm, +1) / n, -1, axis)


def dftn(x: np.ndarray, axes) -> np.ndarray:
    out = np.asarray(x, dtype=np.complex128)
    for ax in axes:
        out = dft(out, ax)
    return out


def idftn(x: np.ndarray, axes) -> np.ndarray:
    out = np.asarray(x, dtype=np.complex128)
    for ax in reversed(list(axes)):
        out = idft(out, ax)
    return out
