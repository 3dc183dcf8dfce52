"""Spectral differential operators (Sec. 2.4.3, Eq. ft_sd).

A derivative along a Fourier axis is a multiplication of the transformed field
by i*kappa, kappa = 2 pi m / P the angular wavenumber of the periodic length P
(P = L for periodic axes, P = 2L for the doubled unbounded axes) and m the
signed mode index.  The Nyquist mode m = M/2 of an even-length axis has no
well defined odd derivative; it is set to zero (reading of the paper, which is
silent on this).  The Laplacian operator NABLA keeps the Nyquist mode: it
multiplies by -(kappa_x^2 + ...) with kappa = 2 pi min(m, M-m)/P.

Operators act on the solution psi after the convolution (Sec. 4.3, Eq.
poisscurl):
  GRAD  (1 -> dim):  d_a psi
  DIV   (dim -> 1):  sum_a d_a psi_a
  CURL  3D (3 -> 3): d x psi;   2D (1 -> 2): (d_y psi, -d_x psi)
  NABLA (c -> c):    -|kappa|^2 psi_c

Pinned in tests/test_oracle_ops.py against the closed-form Fourier
differentiation matrix (Trefethen, "Spectral Methods in MATLAB", ch. 3),
analytic derivatives and div(curl) = 0.
"""
from __future__ import annotations

import numpy as np


def signed_modes(M: int) -> np.ndarray:
    m = np.arange(M)
    return np.where(m <= M // 2, m, m - M).astype(np.float64)


def deriv_multiplier(M: int, period: float) -> np.ndarray:
    """i*kappa for an axis of M points, Nyquist zeroed."""
    m = signed_modes(M)
    if M % 2 == 0:
        m[M // 2] = 0.0
    return 1j * 2.0 * np.pi * m / period


def laplace_multiplier_1d(M: int, period: float) -> np.ndarray:
    m = np.arange(M)
    mm = np.minimum(m, M - m).astype(np.float64)
    return -(2.0 * np.pi * mm / period) ** 2


def _bcast(v: np.ndarray, dim: int, ax: int) -> np.ndarray:
    """Reshape a 1D per-axis vector for arrays laid out [z][y][x] (x = axis 0)."""
    shape = [1] * dim
    shape[dim - 1 - ax] = -1
    return v.reshape(shape)


def apply_op(op: str, dim: int, psi_hat: np.ndarray, mults) -> np.ndarray:
    """psi_hat: [ncomp][...spectral...]; mults[a]: 1D i*kappa vector of axis a."""
    d = [_bcast(mults[a], dim, a) for a in range(dim)]
    if op == "GRAD":
        return np.stack([d[a] * psi_hat[0] for a in range(dim)])
    if op == "DIV":
        return (sum(d[a] * psi_hat[a] for a in range(dim)))[None]
    if op == "CURL":
        if dim == 3:
            px, py, pz = psi_hat
            return np.stack([d[1] * pz - d[2] * py, d[2] * px - d[0] * pz, d[0] * py - d[1] * px])
        return np.stack([d[1] * psi_hat[0], -d[0] * psi_hat[0]])
    raise ValueError(op)


def apply_op_transpose(op: str, dim: int, g_hat: np.ndarray, mults, ncomp: int) -> np.ndarray:
    """Plain (non-conjugate) transpose of apply_op's per-mode matrix.

    Used by the adjoint, which transforms with the inverse DFT first; see adjoint.py.
    """
    d = [_bcast(mults[a], dim, a) for a in range(dim)]
    if op == "GRAD":
        return (sum(d[a] * g_hat[a] for a in range(dim)))[None]
    if op == "DIV":
        return np.stack([d[a] * g_hat[0] for a in range(dim)])
    if op == "CURL":
        if dim == 3:
            gx, gy, gz = g_hat
            # transpose of [[0,-d2,d1],[d2,0,-d0],[-d1,d0,0]]
            return np.stack([d[2] * gy - d[1] * gz, d[0] * gz - d[2] * gx, d[1] * gx - d[0] * gy])
        return (d[1] * g_hat[0] - d[0] * g_hat[1])[None]
    raise ValueError(op)
