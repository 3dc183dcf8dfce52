"""Transpose of the solve, for gradients (the adjoint of Sec. 2.4's four steps).

The solve is affine in f: psi = A_psi f + c, op_out = A_op f + c'.  The
constants come from the boundary lifting and the Dirichlet fill and do not
depend on f.  For a scalar loss with dL/dpsi = g_psi and dL/dop = g_op,
  dL/df = A_psi^T g_psi + A_op^T g_op.

Each A is a product of plain linear steps (extract/pad, per-axis transforms,
a diagonal multiplier, a per-mode operator matrix, real part).  The oracle
forms the transpose literally: the same steps in reverse order, each replaced
by its plain (non-conjugate) transpose.  For y = Re(B x) with real x and g,
<g, y> = <Re(B^T g), x>, so complex intermediates are handled by taking the
real part once at the end.  Per-axis transposes:
  DFT matrix:     symmetric, so DFT^T = DFT and (DFT^-1)^T = DFT^-1;
  R2R matrices:   the explicit matrix of r2r.py, transposed;
  multipliers:    diagonal (unchanged); operator matrices transposed per mode;
  operators on Dirichlet / Neumann axes: a linear map of psi (bounded_ops.py),
                  transposed as a dense matrix.

Pinned in tests/test_oracle_adjoint.py: the dense matrix of the forward map,
built column by column, transposed and applied, and <A x, y> = <x, A^T y>.
"""
from __future__ import annotations

import numpy as np

from . import bounded, bounded_ops, fft, ops, r2r, semi
from .desc import Desc
from .unbounded import _check, green_hat, multipliers, padded_length


def _apply_matrix_T(kind: str, x: np.ndarray, axis: int, scale: float = 1.0) -> np.ndarray:
    xm = np.moveaxis(x, axis, -1)
    m = r2r.matrix(kind, xm.shape[-1]) * scale
    return np.moveaxis(xm @ m, -1, axis)  # (M^T applied) = x @ M


def _bounded_op_transpose(desc: Desc, g_op) -> np.ndarray:
    """D^T g_op for the operator D = bounded_ops.apply on [ncomp][nodes...]."""
    shape_psi = (desc.ncomp,) + desc.shape()
    size = int(np.prod(shape_psi))
    nop = desc.op_components()
    go = np.asarray(g_op, dtype=np.float64).reshape(nop, -1)
    out = np.zeros(size)
    for i in range(size):  # column i of D: its response to the unit field e_i
        e = np.zeros(size)
        e[i] = 1.0
        col = bounded_ops.apply(desc, e.reshape(shape_psi)).reshape(nop, -1)
        out[i] = np.sum(col * go)
    return out.reshape(shape_psi)


def _bounded_adjoint(desc: Desc, g_psi, g_op):
    dim = desc.dim
    usl = bounded._unknown_slices(desc)
    shape_full = (desc.ncomp,) + desc.shape()
    gp = np.zeros(shape_full) if g_psi is None else np.asarray(g_psi, dtype=np.float64).reshape(shape_full)
    shape_u = gp[usl].shape[1:]

    def inv_T(x):  # transpose of backward_transform
        out = x.astype(np.complex128)
        for ax in range(dim):
            nax = bounded._np_axis(dim, ax)
            if desc.bc[ax] == "P":
                out = fft.idft(out, nax)
            else:
                n = out.shape[nax]
                kind = r2r.BACKWARD[(desc.bc[ax], desc.staggered)]
                out = _apply_matrix_T(kind, out, nax, r2r.backward_scale(desc.bc[ax], desc.staggered, n))
        return out

    def fwd_T(x):  # transpose of forward_transform
        out = x
        for ax in reversed(range(dim)):
            nax = bounded._np_axis(dim, ax)
            if desc.bc[ax] == "P":
                out = fft.dft(out, nax)
            else:
                out = _apply_matrix_T(r2r.FORWARD[(desc.bc[ax], desc.staggered)], out, nax)
        return out

    periodic = all(b == "P" for b in desc.bc[:dim])
    if desc.op != "NONE" and g_op is not None and not periodic:
        # Dirichlet / Neumann axes: the operator is a linear map D of psi
        # (bounded_ops.py), so dL/dpsi gains D^T g_op; D^T is the transposed
        # dense matrix of that map (small grids only)
        gp = gp + _bounded_op_transpose(desc, g_op)
    acc = inv_T(gp[usl])
    if desc.op != "NONE" and g_op is not None and periodic:
        nop = desc.op_components()
        go = np.asarray(g_op, dtype=np.float64).reshape((nop,) + desc.shape())
        gh = inv_T(go[usl])
        mults, laps = bounded.op_multipliers(desc, shape_u)
        if desc.op == "NABLA":
            lap = sum(ops._bcast(laps[a], dim, a) for a in range(dim))
            acc = acc + lap[None] * gh
        else:
            acc = acc + ops.apply_op_transpose(desc.op, dim, gh, mults, desc.ncomp)
    acc = acc * bounded.inverse_eigen(desc, shape_u)[None]
    gf_u = fwd_T(acc).real * desc.rhs_scale
    out = np.zeros(shape_full)
    out[usl] = gf_u
    return out


def _unbounded_adjoint(desc: Desc, g_psi, g_op):
    _check(desc)
    dim = desc.dim
    axes = [1 + (dim - 1 - ax) for ax in range(dim)]
    # node counts (N_c on staggered grids, N_c + 1 on regular grids) and the
    # doubled lengths M of the forward solve (padded_length), [z][y][x] order
    n_arr = tuple(desc.nodes(ax) for ax in reversed(range(dim)))
    padded = tuple(padded_length(desc, ax) for ax in reversed(range(dim)))
    keep = (slice(None),) + tuple(slice(0, n) for n in n_arr)

    def pad(g, c):
        out = np.zeros((c,) + padded)
        out[keep] = np.asarray(g, dtype=np.float64).reshape((c,) + n_arr)
        return out

    acc = np.zeros((desc.ncomp,) + padded, dtype=np.complex128)
    if g_psi is not None:
        acc = acc + fft.idftn(pad(g_psi, desc.ncomp), axes)  # (DFT^-1)^T = DFT^-1
    if desc.op != "NONE" and g_op is not None:
        nop = desc.op_components()
        gh = fft.idftn(pad(g_op, nop), axes)
        mults, laps = multipliers(desc)
        if desc.op == "NABLA":
            lap = sum(ops._bcast(laps[a], dim, a) for a in range(dim))
            acc = acc + lap[None] * gh
        else:
            acc = acc + ops.apply_op_transpose(desc.op, dim, gh, mults, desc.ncomp)
    hd = 1.0
    for ax in range(dim):
        hd *= desc.h(ax)
    acc = acc * ((-desc.rhs_scale * hd) * green_hat(desc))[None]
    return fft.dftn(acc, axes).real[keep]  # DFT^T = DFT, then pad^T = extract


def _semi_adjoint(desc: Desc, g_psi, g_op):
    """Transpose of semi.solve_semi: the same steps reversed, each transposed
    (DFT^T = DFT, (DFT^-1)^T = DFT^-1, crop^T = zero-pad, diagonal multipliers unchanged)."""
    dim = desc.dim
    ua = semi.unbounded_axis(desc)
    uax = 1 + (dim - 1 - ua)
    pax = [1 + (dim - 1 - a) for a in range(dim) if a != ua]
    M = padded_length(desc, ua)
    Nu = desc.nodes(ua)
    n_arr = desc.shape()

    def up(g, c):
        # (crop after IDFT_U, then IDFT_P)^T = IDFT_P, zero-pad along U, IDFT_U
        x = fft.idftn(np.asarray(g, dtype=np.float64).reshape((c,) + n_arr), pax)
        shape = list(x.shape)
        shape[uax] = M
        xp = np.zeros(shape, dtype=np.complex128)
        sl = [slice(None)] * len(shape)
        sl[uax] = slice(0, Nu)
        xp[tuple(sl)] = x
        return fft.idft(xp, uax)

    shape = list((desc.ncomp,) + n_arr)
    shape[uax] = M
    acc = np.zeros(shape, dtype=np.complex128)
    if g_psi is not None:
        acc = acc + up(g_psi, desc.ncomp)
    if desc.op != "NONE" and g_op is not None:
        gh = up(g_op, desc.op_components())
        mults, laps = semi.multipliers(desc)
        if desc.op == "NABLA":
            lap = sum(ops._bcast(laps[a], dim, a) for a in range(dim))
            acc = acc + lap[None] * gh
        else:
            acc = acc + ops.apply_op_transpose(desc.op, dim, gh, mults, desc.ncomp)
    Kh = fft.dft(semi.kernel_rows(desc), uax - 1)
    acc = acc * ((-desc.rhs_scale * desc.h(ua)) * Kh)[None]
    out = fft.dft(acc, uax)  # DFT_U^T = DFT_U
    sl = [slice(None)] * out.ndim
    sl[uax] = slice(0, Nu)
    return fft.dftn(out[tuple(sl)], pax).real  # pad^T = crop, DFT_P^T = DFT_P


def adjoint_solve(desc: Desc, g_psi, g_op=None):
    """dL/df for dL/dpsi = g_psi and dL/dop_out = g_op (either may be None)."""
    if all(b == "U" for b in desc.bc[: desc.dim]):
        return _unbounded_adjoint(desc, g_psi, g_op)
    if semi.is_semi(desc):
        return _semi_adjoint(desc, g_psi, g_op)
    return _bounded_adjoint(desc, g_psi, g_op)
