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
-(N-1)..(N-1), so the wrap index N is never used.  A regular grid carries
N_c + 1 nodes per axis, so offsets span -N_c..N_c and the padded length must
be at least 2 N_c + 1 (Sec. 4.3 notes the grid type is otherwise immaterial);
our reading takes the smallest length of the form 2^p or 3 * 2^p that is at
least that (the same rule fixes the wavenumbers of the spectral operators).
With "2N" below read as that padded length M per axis.

Pinned in tests/test_oracle_unbounded.py by brute-force direct summation and
the closed-form potential of a Gaussian blob.
"""
from __future__ import annotations

import numpy as np

from . import fft, ops
from .desc import Desc
from .green import green


def spectral_cutoff(desc: Desc) -> float:
    """Cut-off wavenumber of the spectral kernel: the largest wavenumber every axis resolves, pi / max h."""
    return float(np.pi / max(desc.h(a) for a in range(desc.dim)))


def padded_length(desc: Desc, ax: int) -> int:
    """Length M of the doubled axis: 2 N_c (staggered), else the smallest 2^p or 3 * 2^p >= 2 N_c + 1."""
    n = desc.n[ax]
    if desc.staggered:
        return 2 * n
    need = max(2 * n + 1, 4)
    best = None
    for base in (1, 3):
        m = base
        while m < need:
            m *= 2
        best = m if best is None else min(best, m)
    return best


def green_table(desc: Desc) -> np.ndarray:
    """G on the doubled grid, [2Nz][2Ny][2Nx] (or [2Ny][2Nx])."""
    r2 = 0.0
    for ax in range(desc.dim):
        M = padded_length(desc, ax)
        m = np.arange(M)
        d = np.minimum(m, M - m) * desc.h(ax)
        r2 = r2 + ops._bcast(d * d, desc.dim, ax)
    return green(desc.dim, np.sqrt(r2), desc.sigma, desc.kernel, spectral_cutoff(desc))


def green_hat(desc: Desc) -> np.ndarray:
    axes = [1 + (desc.dim - 1 - ax) for ax in range(desc.dim)]
    g = green_table(desc)[None]
    return fft.dftn(g, axes)[0].real


def _check(desc: Desc):
    if not all(b == "U" for b in desc.bc[: desc.dim]):
        raise NotImplementedError("all axes must be unbounded")
    if desc.sigma <= 0 and desc.kernel != "SPECT":
        raise ValueError("sigma must be positive")


def multipliers(desc: Desc):
    mults, laps = [], []
    for ax in range(desc.dim):
        M = padded_length(desc, ax)
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
    padded = tuple(padded_length(desc, ax) for ax in reversed(range(dim)))
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


# ---------------------------------------------------------------------------
# one output point at a time (for grids too large for the full oracle)
# ---------------------------------------------------------------------------
# The doubled-domain solve equals psi_i = -s h^d sum_j G(x_i - x_j) f_j.  An
# operator applied after the convolution acts on the 2N-periodic solution, so
# d_a psi = -s h^d sum_j K_a(i - j) f_j with K_a = (spectral derivative along a
# of the periodic G table).  K_a is odd in its own offset and even in the
# others, so it is tabulated on [0, N] x [0, 2N) x [0, N] (own axis full) with
# the oracle's DFT along that axis; each requested point is then a direct sum.

def derivative_tables(desc: Desc):
    """K_a on the half-octant, list over axes a; entry [a] has axis a of length 2N."""
    _check(desc)
    dim = desc.dim
    tabs = []
    for a in range(dim):
        r2 = 0.0
        for ax in range(dim):
            M = padded_length(desc, ax)
            if ax == a:
                m = np.arange(M)
                d = np.minimum(m, M - m) * desc.h(ax)
            else:
                d = np.arange(desc.n[ax] + 1) * desc.h(ax)
            r2 = r2 + ops._bcast(d * d, dim, ax)
        g = green(dim, np.sqrt(r2), desc.sigma, desc.kernel, spectral_cutoff(desc))
        nax = dim - 1 - a
        M = padded_length(desc, a)
        mult = ops.deriv_multiplier(M, M * desc.h(a))
        shape = [1] * dim
        shape[nax] = -1
        k = fft.idft(mult.reshape(shape) * fft.dft(g, nax), nax).real
        tabs.append(k)
    return tabs


def _gather(tab, dim, offs, a):
    """tab at signed offsets offs[ax] (arrays broadcasting over sources)."""
    idx = []
    for ax in reversed(range(dim)):
        o = offs[ax]
        if ax == a:
            M = tab.shape[dim - 1 - ax]
            idx.append(np.mod(o, M))
        else:
            idx.append(np.abs(o))
    return tab[tuple(idx)]


def sample_points(desc: Desc, f: np.ndarray, points, tables=None):
    """psi and op_out at the given output points (list of (x, y[, z]) indices).

    Returns (psi [npts][ncomp], op [npts][nop] or None).
    """
    _check(desc)
    dim = desc.dim
    f = np.asarray(f, dtype=np.float64)
    if f.ndim == dim:
        f = f[None]
    ncomp = f.shape[0]
    hd = 1.0
    for ax in range(dim):
        hd *= desc.h(ax)
    scale = -desc.rhs_scale * hd
    src = [np.arange(desc.nodes(ax)) for ax in range(dim)]
    if desc.op not in ("NONE",) and desc.op != "NABLA" and tables is None:
        tables = derivative_tables(desc)
    psi_out, op_out = [], []
    for p in points:
        offs = []
        r2 = 0.0
        for ax in range(dim):
            o = p[ax] - src[ax]
            o = ops._bcast(o, dim, ax)
            offs.append(o)
            r2 = r2 + (o * desc.h(ax)) ** 2
        g = green(dim, np.sqrt(r2), desc.sigma, desc.kernel, spectral_cutoff(desc))
        psi_out.append([scale * np.sum(g * f[c]) for c in range(ncomp)])
        if desc.op in ("GRAD", "DIV", "CURL"):
            K = [_gather(tables[a], dim, offs, a) for a in range(dim)]
            dpsi = [[scale * np.sum(K[a] * f[c]) for a in range(dim)] for c in range(ncomp)]  # d_a psi_c
            if desc.op == "GRAD":
                op_out.append([dpsi[0][a] for a in range(dim)])
            elif desc.op == "DIV":
                op_out.append([sum(dpsi[a][a] for a in range(dim))])
            elif dim == 3:
                op_out.append([dpsi[2][1] - dpsi[1][2], dpsi[0][2] - dpsi[2][0], dpsi[1][0] - dpsi[0][1]])
            else:
                op_out.append([dpsi[0][1], -dpsi[0][0]])
    psi_arr = np.array(psi_out)
    op_arr = np.array(op_out) if op_out else None
    return psi_arr, op_arr


# ---------------------------------------------------------------------------
# whole lines (3D): direct sums across, exact aperiodic convolution along
# ---------------------------------------------------------------------------
# For a line parallel to axis L through (i_P, i_Q) on the other two axes,
#   psi(i_L) = s sum_{j_P, j_Q} sum_{j_L} G(i - j) f(j),  s = -rhs_scale h^d.
# The inner sum over j_L is an aperiodic 1D convolution, evaluated as the
# circular convolution of length M (the doubled axis) of the zero-padded source
# row with the kernel row of the doubled grid (mirrored distances, exactly the
# row the full solve uses), i.e. as a product of DFTs of the two rows; the
# sums over j_P, j_Q are direct.  The derivative along L is the doubled
# grid's i kappa applied to the line's DFT (the full solve applies it to the
# whole padded solution, whose rows along L are these circular convolutions).
# A derivative across, along a in {P, Q}, uses the kernel
# K_a = IDFT_a(i kappa_a DFT_a(G)) of the doubled grid along a (the same
# definition as derivative_tables), whose rows along L only enter at offsets
# |j_L - i_L| < N_L.  The transforms of this sampler are numpy.fft calls (a
# library FFT as one step); it is pinned against the full doubled-domain
# solve, which uses the oracle's own transform.


def sample_lines(desc: Desc, f: np.ndarray, axis: int, positions):
    """psi and op_out along whole lines parallel to `axis` (3D; op NONE, GRAD, DIV or CURL).

    positions: (i_P, i_Q) index pairs on the two other axes P < Q.
    Returns (psi [nlines][ncomp][N_axis], op [nlines][nop][N_axis] or None).
    """
    _check(desc)
    if desc.dim != 3:
        raise ValueError("sample_lines is for 3D problems")
    if desc.op == "NABLA":
        raise ValueError("NABLA is not sampled by lines")
    f = np.asarray(f, dtype=np.float64)
    if f.ndim == 3:
        f = f[None]
    ncomp = f.shape[0]
    L = axis
    P, Q = [a for a in range(3) if a != L]
    ML, MP, MQ = padded_length(desc, L), padded_length(desc, P), padded_length(desc, Q)
    NL, NP, NQ = desc.nodes(L), desc.nodes(P), desc.nodes(Q)
    hL, hP, hQ = desc.h(L), desc.h(P), desc.h(Q)
    s = -desc.rhs_scale * hL * hP * hQ
    kc = spectral_cutoff(desc)

    def mirrored(M, h):
        m = np.arange(M)
        return np.minimum(m, M - m) * h

    # sources as [c][j_P][j_Q][j_L], zero-padded to M along L, transformed along L
    perm = (0,) + tuple(1 + (2 - a) for a in (P, Q, L))
    fr = np.zeros((ncomp, NP, NQ, ML))
    fr[..., :NL] = np.transpose(f, perm)
    F = np.fft.fft(fr, axis=-1)
    del fr
    # G rows along L (full mirrored row of the doubled grid) for offsets |o_P| < N_P, |o_Q| < N_Q
    dL = mirrored(ML, hL)
    r = np.sqrt((np.arange(NP) * hP)[:, None, None] ** 2 + (np.arange(NQ) * hQ)[None, :, None] ** 2 +
                dL[None, None, :] ** 2)
    Ghat = np.fft.fft(green(3, r, desc.sigma, desc.kernel, kc), axis=-1).real
    del r
    need_op = desc.op in ("GRAD", "DIV", "CURL")
    if need_op:
        m = np.arange(ML)
        inside = (m < NL) | (m > ML - NL)
        oL = np.where(inside, np.minimum(m, ML - m), 0)

        def cross_rows(Ma, ha, No, ho):
            # K_a on [own axis a, doubled (M_a)][other cross axis (N_o)][|o_L| < N_L],
            # then rows along L (zero outside |o_L| < N_L), transformed along L
            ra = mirrored(Ma, ha)
            rr = np.sqrt(ra[:, None, None] ** 2 + (np.arange(No) * ho)[None, :, None] ** 2 +
                         (np.arange(NL) * hL)[None, None, :] ** 2)
            g = green(3, rr, desc.sigma, desc.kernel, kc)
            mult = ops.deriv_multiplier(Ma, Ma * ha)
            k = np.fft.ifft(mult[:, None, None] * np.fft.fft(g, axis=0), axis=0).real
            rows = k[:, :, oL] * inside[None, None, :]
            return np.fft.fft(rows, axis=-1).real
        KP = cross_rows(MP, hP, NQ, hQ)  # [M_P][N_Q][M_L]
        KQ = cross_rows(MQ, hQ, NP, hP)  # [M_Q][N_P][M_L]
        dmult = ops.deriv_multiplier(ML, ML * hL)
    psi_out, op_out = [], []
    jP = np.arange(NP)
    jQ = np.arange(NQ)
    for iP, iQ in positions:
        aP = np.abs(iP - jP)
        aQ = np.abs(iQ - jQ)
        Gl = Ghat[aP[:, None], aQ[None, :], :]
        ph = [s * np.einsum("pqk,pqk->k", Gl, F[c]) for c in range(ncomp)]
        psi_out.append([np.fft.ifft(h_)[:NL].real for h_ in ph])
        if need_op:
            KPl = KP[np.mod(iP - jP, MP)[:, None], aQ[None, :], :]
            KQl = KQ[np.mod(iQ - jQ, MQ)[:, None], aP[None, :], :].transpose(1, 0, 2)
            d = {}
            for c in range(ncomp):
                d[(c, L)] = np.fft.ifft(dmult * ph[c])[:NL].real
                d[(c, P)] = np.fft.ifft(s * np.einsum("pqk,pqk->k", KPl, F[c]))[:NL].real
                d[(c, Q)] = np.fft.ifft(s * np.einsum("pqk,pqk->k", KQl, F[c]))[:NL].real
            if desc.op == "GRAD":
                op_out.append([d[(0, a)] for a in range(3)])
            elif desc.op == "DIV":
                op_out.append([d[(0, 0)] + d[(1, 1)] + d[(2, 2)]])
            else:
                op_out.append([d[(2, 1)] - d[(1, 2)], d[(0, 2)] - d[(2, 0)], d[(1, 0)] - d[(0, 1)]])
    psi_arr = np.array(psi_out)
    op_arr = np.array(op_out) if op_out else None
    return psi_arr, op_arr
