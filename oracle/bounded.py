"""Bounded solve: periodic / Dirichlet / Neumann axes (Sec. 2.2, 2.5, Table 1).

Steps, in the paper's order (Sec. 2.4, the four-step solve):
  1. take the unknowns out of the node array (regular Dirichlet axes keep their
     boundary nodes as data, Sec. 2.4.2) and scale by rhs_scale;
  2. FD2 only: lift inhomogeneous face data into the right-hand side (the
     "simple weighting of the boundary source terms" of Sec. 2.5.2);
  3. forward transform along x, then y, then z: DFT for periodic axes, the
     forward R2R type of Table 1 for Dirichlet/Neumann axes;
  4. divide by the eigenvalue sum lambda = sum_axis lambda_axis(k_axis); the
     zero eigenvalue gives a zero coefficient (Sec. 2.2: zero mean);
  5. optional spectral operator (Sec. 2.4.3): on periodic axes a product in
     spectral space; on Dirichlet / Neumann axes the derivative of the basis
     series (bounded_ops.py);
  6. inverse transforms in reverse order with their normalisation;
  7. write the unknowns back and fill regular Dirichlet boundary nodes with the
     face values (x faces first, then y, then z; later faces overwrite shared
     edge nodes).
An axis may carry a Dirichlet and a Neumann face ('DN' / 'ND'); it is then
transformed in the quarter-wave sine / cosine basis (r2r.py) and each face
follows its own lifting rule below.

Boundary lifting (our reading; the paper gives no formulas).  With g the face
value (Dirichlet: psi; Neumann: d psi / d x_axis) and h the spacing, the
ghost-node rules of the 3-point stencil move these terms to the right-hand
side of the first/last unknown along the axis:
  Dirichlet regular    lower: f -= g/h^2     upper: f -= g/h^2
  Dirichlet staggered  lower: f -= 2g/h^2    upper: f -= 2g/h^2
  Neumann regular      lower: f += 2g/h      upper: f -= 2g/h
  Neumann staggered    lower: f += g/h       upper: f -= g/h
Contributions add at edges and corners.

Pinned in tests/test_oracle_bounded.py: manufactured PS solutions (exact),
the FD2 residual of an explicit 7-point stencil, second-order convergence, and
a dense LU solve of the assembled FD matrix on small grids.
"""
from __future__ import annotations

from typing import Dict, Optional, Tuple

import numpy as np

from . import bounded_ops, eigen, fft, ops, r2r
from .desc import Desc


def _np_axis(dim: int, ax: int) -> int:
    """numpy axis of physical axis ax for arrays [comp][z][y][x]."""
    return 1 + (dim - 1 - ax)


def _unknown_slices(desc: Desc):
    sl = [slice(None)] * (desc.dim + 1)
    for ax in range(desc.dim):
        a, b = desc.unknown_range(ax)
        sl[_np_axis(desc.dim, ax)] = slice(a, b)
    return tuple(sl)


def _face_on_unknowns(desc: Desc, ax: int, face: np.ndarray) -> np.ndarray:
    """Restrict a face array (node arrays of the other axes) to their unknowns."""
    others = [a for a in reversed(range(desc.dim)) if a != ax]  # array order
    sl = []
    for a in others:
        lo, hi = desc.unknown_range(a)
        sl.append(slice(lo, hi))
    return face[tuple(sl)]


def lift(desc: Desc, rhs: np.ndarray, faces: Optional[Dict[Tuple[int, int], np.ndarray]]) -> np.ndarray:
    """Add the FD2 boundary terms to rhs [ncomp][unknowns...] (in place copy)."""
    out = rhs.copy()
    if not faces:
        return out
    for (ax, side), face in faces.items():
        bc = desc.face(ax, side)
        h = desc.h(ax)
        g = _face_on_unknowns(desc, ax, np.asarray(face, dtype=np.float64))
        if bc == "D":
            w = (-1.0 if not desc.staggered else -2.0) / (h * h)
        elif bc == "N":
            base = (2.0 if not desc.staggered else 1.0) / h
            w = base if side == 0 else -base
        else:
            raise ValueError("faces only for Dirichlet/Neumann axes")
        nax = _np_axis(desc.dim, ax)
        idx = [slice(None)] * out.ndim
        idx[nax] = 0 if side == 0 else out.shape[nax] - 1
        out[tuple(idx)] += w * g[None] if g.ndim == out.ndim - 2 else w * g
    return out


def forward_transform(desc: Desc, x: np.ndarray) -> np.ndarray:
    out = x.astype(np.complex128)
    for ax in range(desc.dim):  # x, then y, then z
        nax = _np_axis(desc.dim, ax)
        if desc.bc[ax] == "P":
            out = fft.dft(out, nax)
        else:
            out = r2r.forward(desc.bc[ax], desc.staggered, out, nax)
    return out


def backward_transform(desc: Desc, x: np.ndarray) -> np.ndarray:
    out = x
    for ax in reversed(range(desc.dim)):  # z, then y, then x
        nax = _np_axis(desc.dim, ax)
        if desc.bc[ax] == "P":
            out = fft.idft(out, nax)
        else:
            out = r2r.backward(desc.bc[ax], desc.staggered, out, nax)
    return out


def eigen_sum(desc: Desc, shape_unknowns) -> np.ndarray:
    lam = 0.0
    for ax in range(desc.dim):
        n = shape_unknowns[desc.dim - 1 - ax]
        v = eigen.eigenvalues(desc.bc[ax], desc.staggered, desc.eig, n, desc.length(ax), desc.h(ax))
        lam = lam + ops._bcast(v, desc.dim, ax)
    return lam


def inverse_eigen(desc: Desc, shape_unknowns) -> np.ndarray:
    lam = eigen_sum(desc, shape_unknowns)
    safe = np.where(lam == 0.0, 1.0, lam)
    return np.where(lam == 0.0, 0.0, 1.0 / safe)


def op_multipliers(desc: Desc, shape_unknowns):
    mults, laps = [], []
    for ax in range(desc.dim):
        if desc.bc[ax] != "P":
            raise NotImplementedError("spectral operators need periodic or unbounded axes")
        n = shape_unknowns[desc.dim - 1 - ax]
        mults.append(ops.deriv_multiplier(n, desc.length(ax)))
        laps.append(ops.laplace_multiplier_1d(n, desc.length(ax)))
    return mults, laps


def apply_operator(desc: Desc, psi_hat: np.ndarray, mults, laps) -> np.ndarray:
    if desc.op == "NABLA":
        lap = sum(ops._bcast(laps[a], desc.dim, a) for a in range(desc.dim))
        return lap[None] * psi_hat
    return ops.apply_op(desc.op, desc.dim, psi_hat, mults)


def _as_fields(desc: Desc, f: np.ndarray) -> np.ndarray:
    f = np.asarray(f, dtype=np.float64)
    if f.ndim == desc.dim:
        f = f[None]
    if f.shape[1:] != desc.shape():
        raise ValueError(f"source shape {f.shape} does not match {desc.shape()}")
    return f


def fill_dirichlet(desc: Desc, psi: np.ndarray, faces) -> None:
    if not faces:
        return
    for ax in range(desc.dim):
        if desc.staggered:
            continue
        for side in (0, 1):
            if desc.face(ax, side) != "D":
                continue
            face = faces.get((ax, side))
            if face is None:
                continue
            nax = _np_axis(desc.dim, ax)
            idx = [slice(None)] * psi.ndim
            idx[nax] = 0 if side == 0 else psi.shape[nax] - 1
            psi[tuple(idx)] = face


def solve_bounded(desc: Desc, f: np.ndarray, faces=None):
    """Return (psi [ncomp][nodes...], op_out [nop][nodes...] or None)."""
    if any(b == "U" for b in desc.bc[: desc.dim]):
        raise NotImplementedError("mixed unbounded/bounded axes")
    if faces and desc.eig != "FD2":
        raise ValueError("inhomogeneous boundary data needs FD2 eigenvalues (Sec. 2.5.2)")
    fields = _as_fields(desc, f)
    usl = _unknown_slices(desc)
    rhs = desc.rhs_scale * fields[usl]
    rhs = lift(desc, rhs, faces)
    shape_u = rhs.shape[1:]
    fh = forward_transform(desc, rhs)
    psi_hat = fh * inverse_eigen(desc, shape_u)[None]
    op_hat = None
    periodic = all(b == "P" for b in desc.bc[: desc.dim])
    if desc.op != "NONE" and periodic:
        mults, laps = op_multipliers(desc, shape_u)
        op_hat = apply_operator(desc, psi_hat, mults, laps)
    psi_u = backward_transform(desc, psi_hat).real
    psi = np.zeros_like(fields)
    psi[usl] = psi_u
    fill_dirichlet(desc, psi, faces)
    op_out = None
    if op_hat is not None:
        op_u = backward_transform(desc, op_hat).real
        op_out = np.zeros((op_u.shape[0],) + fields.shape[1:])
        op_out[usl] = op_u
    elif desc.op != "NONE":  # Dirichlet / Neumann axes: derivatives of the basis series
        op_out = bounded_ops.apply(desc, psi)
    return psi, op_out
