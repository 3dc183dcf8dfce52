"""Semi-unbounded solve: one unbounded axis, the other axes periodic.

The paper names semi-unbounded domains as the next step beyond uniform
boundaries (Sec. 2.6 and Sec. 6) without giving their kernels; this is our
reading, from first principles.  Along the periodic axes the solve is
spectral (Sec. 2.4): every periodic mode k separates, and with
kappa^2 = -(sum of the periodic axes' eigenvalues, Table 1, PS or FD2) the
unbounded axis carries the one-dimensional problem
    psi_k'' - kappa^2 psi_k = rhs_scale f_k,   psi_k bounded as |z| -> infinity,
whose free-space kernel (of -(d^2/dz^2 - kappa^2)) is
    G_kappa(z) = exp(-kappa |z|) / (2 kappa)   (kappa > 0),
    G_0(z)     = -|z| / 2                      (kappa = 0, the 1D free-space kernel),
so psi_k(z_i) = -rhs_scale h_z sum_j G_kappa(z_i - z_j) f_k(z_j): a point-sampled
(trapezoidal) discretisation of the convolution; these kernels are
continuous, so no regularisation is needed.  The aperiodic sum is evaluated
by Hockney-Eastwood doubling of the unbounded axis only (Sec. 2.6): the
kernel row is sampled on the doubled axis with mirrored distances, both rows
are transformed, multiplied and transformed back, and the first N points are
kept.  Operators use ik with the periodic axes' wavenumbers and the doubled
axis's wavenumbers (Nyquist zeroed for first derivatives), after the
convolution, as for unbounded domains.

Steps, in order:
  1. DFT of f along every periodic axis (oracle's own FFT);
  2. per periodic mode, kappa and the kernel row on the doubled axis;
  3. zero-pad f along the unbounded axis, DFT along it, DFT of the kernel rows;
  4. multiply: psi_hat = -rhs_scale h_z K_hat f_hat;
  5. optional operator;
  6. inverse DFT along the unbounded axis, keep the first N, inverse DFTs along
     the periodic axes, real part.

Pinned in tests/test_oracle_semi.py by a direct O(N^2) sum along the
unbounded axis per mode, and by second-order convergence to the continuous
solution of a Gaussian source (closed forms with erfc).
"""
from __future__ import annotations

import numpy as np

from . import eigen, fft, ops
from .desc import Desc
from .unbounded import padded_length


def is_semi(desc: Desc) -> bool:
    bcs = list(desc.bc[: desc.dim])
    return desc.dim >= 2 and bcs.count("U") == 1 and bcs.count("P") == desc.dim - 1


def unbounded_axis(desc: Desc) -> int:
    return list(desc.bc[: desc.dim]).index("U")


def _check(desc: Desc):
    if not is_semi(desc):
        raise NotImplementedError("semi-unbounded solves: exactly one unbounded axis, the others periodic")


def kappa2(desc: Desc) -> np.ndarray:
    """kappa^2 of every periodic mode, broadcast over the [z][y][x] array (size 1 along the unbounded axis)."""
    dim = desc.dim
    ua = unbounded_axis(desc)
    k2 = 0.0
    for a in range(dim):
        if a == ua:
            continue
        lam = eigen.eigenvalues("P", True, desc.eig, desc.n[a], desc.length(a), desc.h(a))
        k2 = k2 + ops._bcast(-lam, dim, a)
    return np.asarray(k2, dtype=np.float64)


def kernel_rows(desc: Desc) -> np.ndarray:
    """G_kappa on the doubled unbounded axis (mirrored distances) for every periodic mode."""
    dim = desc.dim
    ua = unbounded_axis(desc)
    M = padded_length(desc, ua)
    m = np.arange(M)
    dist = ops._bcast(np.minimum(m, M - m) * desc.h(ua), dim, ua)
    k = np.sqrt(kappa2(desc))
    safe = np.where(k > 0.0, k, 1.0)
    return np.where(k > 0.0, np.exp(-safe * dist) / (2.0 * safe), -0.5 * dist)


def multipliers(desc: Desc):
    """Derivative and Laplacian multipliers per axis (periodic: own length; unbounded: doubled)."""
    ua = unbounded_axis(desc)
    mults, laps = [], []
    for a in range(desc.dim):
        if a == ua:
            M = padded_length(desc, a)
            period = M * desc.h(a)
        else:
            M = desc.n[a]
            period = desc.length(a)
        mults.append(ops.deriv_multiplier(M, period))
        laps.append(ops.laplace_multiplier_1d(M, period))
    return mults, laps


def solve_semi(desc: Desc, f: np.ndarray):
    """Return (psi [ncomp][...], op_out [nop][...] or None)."""
    _check(desc)
    dim = desc.dim
    f = np.asarray(f, dtype=np.float64)
    if f.ndim == dim:
        f = f[None]
    ncomp = f.shape[0]
    ua = unbounded_axis(desc)
    uax = 1 + (dim - 1 - ua)  # numpy axis of the unbounded axis in [c][z][y][x]
    pax = [1 + (dim - 1 - a) for a in range(dim) if a != ua]
    M = padded_length(desc, ua)
    Nu = desc.nodes(ua)
    # 1. periodic transforms
    F = fft.dftn(f, pax)
    # 3. zero-pad along the unbounded axis and transform along it
    shape = list(F.shape)
    shape[uax] = M
    Fp = np.zeros(shape, dtype=np.complex128)
    sl = [slice(None)] * len(shape)
    sl[uax] = slice(0, Nu)
    Fp[tuple(sl)] = F
    Fh = fft.dft(Fp, uax)
    # 2. + 3. kernel rows and their transform along the unbounded axis
    K = kernel_rows(desc)
    Kh = fft.dft(K, uax - 1)
    # 4. multiply
    psi_hat = (-desc.rhs_scale * desc.h(ua)) * Kh[None] * Fh
    # 5. operator
    op_hat = None
    if desc.op != "NONE":
        mults, laps = multipliers(desc)
        if desc.op == "NABLA":
            lap = sum(ops._bcast(laps[a], dim, a) for a in range(dim))
            op_hat = lap[None] * psi_hat
        else:
            op_hat = ops.apply_op(desc.op, dim, psi_hat, mults)

    # 6. back: inverse along the unbounded axis, crop, inverse along the periodic axes
    def back(h):
        x = fft.idft(h, uax)[tuple(sl)]
        return fft.idftn(x, pax).real

    psi = back(psi_hat)
    op_out = None if op_hat is None else back(op_hat)
    return psi, op_out
