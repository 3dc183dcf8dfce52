"""Unbounded solve by Hockney-Eastwood domain doubling (Sec. 2.6, Fig. unbounded).

Steps, in the paper's order:
  1. tabulate the Green's function on the doubled grid (2N per axis), mirrored
     about the index N: offset m along an axis is the distance
     min(m, 2N - m) * h (Sec. 2.6: "doubled ... and mirrored");
  2. transform it once: G_hat = DFT(G_table) (real, since the table is even);
  3. zero-pad the source into the doubled domain and transform it;
  4. multiply: psi_hat = -rhs_scale * h^d * G_hat * f_hat;
  5. optional spectral operator with the doubled grid's wavenumbers
     (Sec. 4.3: the derivative is taken after the convolution);
  6. inverse transform and keep the first N points per axis.

On a staggered grid the result equals the aperiodic discrete convolution
psi_i = -rhs_scale h^d sum_j G(x_i - x_j) f_j exactly: offsets only span
-(N-1)..(N-1), so the wrap index N is never used.  Only staggered grids are
handled (a regular grid would need 2N_c+1 points; not in this build).

Pinned in tests/test_oracle_unbounded.py by brute-force direct summation and
the closed-form potential of a Gaussian blob.
"""
from __future__ import annotations

import numpy as np

from . import fft, ops
from .desc import Desc
from .green import green


def green_table(desc: Desc) -> np.ndarray:
    """G on the doubled grid, [2Nz][2Ny][2Nx] (or [2Ny][2Nx])."""
    r2 = 0.0
    for ax in range(desc.dim):
        M = 2 * desc.n[ax]
        m = np.arange(M)
        d = np.minimum(m, M - m) * desc.h(ax)
        r2 = r2 + ops._bcast(d * d, desc.dim, ax)
    return green(desc.dim, np.sqrt(r2), desc.sigma)


def green_hat(desc: Desc) -> np.ndarray:
    axes = [1 + (desc.dim - 1 - ax) for ax in range(desc.dim)]
    g = green_table(desc)[None]
    return fft.dftn(g, axes)[0].real


def _check(desc: Desc):
    if not all(b == "U" for b in desc.bc[: desc.dim]):
        raise NotImplementedError("all axes must be unbounded")
    if not desc.staggered:
        raise NotImplementedError("unbounded solves use the staggered grid")
    if desc.sigma <= 0:
        raise ValueError("sigma must be positive")


def multipliers(desc: Desc):
    mults, laps = [], []
    for ax in range(desc.dim):
        M = 2 * desc.n[ax]
        period = M * desc.h(ax)
        mults.append(ops.deriv_multiplier(M, period))
        laps.append(ops.laplace_multiplier_1d(M, period))
    return mults, laps


def solve_unbounded(desc: Desc, f: np.ndarray, g_hat: np.ndarray = None):
    """Return (psi [ncomp][N...], op_out [nop][N...] or None)."""
    _check(desc)
    f = np.asarray(f, dtype=np.float64)
    if f.ndim == desc.dim:
        f = f[None]
    ncomp = f.shape[0]
    dim = desc.dim
    axes = [1 + (dim - 1 - ax) for ax in range(dim)]
    padded = tuple(2 * desc.n[ax] for ax in reversed(range(dim)))
    fp = np.zeros((ncomp,) + padded)
    fp[(slice(None),) + tuple(slice(0, n) for n in f.shape[1:])] = f
    if g_hat is None:
        g_hat = green_hat(desc)
    hd = 1.0
    for ax in range(dim):
        hd *= desc.h(ax)
    psi_hat = (-desc.rhs_scale * hd) * g_hat[None] * fft.dftn(fp, axes)
    op_hat = None
    if desc.op != "NONE":
        mults, laps = multipliers(desc)
        if desc.op == "NABLA":
            lap = sum(ops._bcast(laps[a], dim, a) for a in range(dim))
            op_hat = lap[None] * psi_hat
        else:
            op_hat = ops.apply_op(desc.op, dim, psi_hat, mults)
    keep = (slice(None),) + tuple(slice(0, n) for n in f.shape[1:])
    psi = fft.idftn(psi_hat, axes).real[keep]
    op_out = None if op_hat is None else fft.idftn(op_hat, axes).real[keep]
    return psi, op_out
