"""Spectral operators on Dirichlet / Neumann axes (Sec. 2.4.3 defines the
operators as products in spectral space; the paper does not say how they act on
DST / DCT axes, so this is our reading).

Along a bounded axis the solution on its unknown nodes is the truncated series
of that axis's transform basis (Table 1, and the quarter-wave bases of an axis
with one Dirichlet and one Neumann face), with s = x - X_l and L_x = X_u - X_l:
    Dirichlet     sin(pi m s / L_x)          m = 1 .. nu
    Neumann       cos(pi m s / L_x)          m = 0 .. nu - 1
    D-N           sin(pi (m + 1/2) s / L_x)  m = 0 .. nu - 1
    N-D           cos(pi (m + 1/2) s / L_x)  m = 0 .. nu - 1
(nu unknowns; the basis matrix on the unknown nodes is square and invertible).
A derivative along an axis differentiates that series analytically (a sine
series becomes a cosine series with the same wavenumbers and vice versa) and
evaluates it at every node of the output array.  Along the other axes the
series takes the solution's values on the unknown nodes and its own value,
zero, on regular-grid Dirichlet face nodes.  The operators combine these
derivatives as on periodic axes:
    GRAD_a = d_a psi,  DIV = sum_a d_a psi_a,  CURL (3D) = (d_y psi_z - d_z psi_y, ...),
    CURL (2D) = (d_y psi, -d_x psi),  NABLA = sum_a d_a^2 psi_c.
First derivatives use the exact wavenumbers also with FD2 eigenvalues (as on
periodic axes).  Pinned in tests/test_oracle_bounded_ops.py by manufactured
single-mode solutions whose derivatives are known in closed form.
"""
from __future__ import annotations

import math

import numpy as np

from .desc import Desc


def _np_axis(dim: int, ax: int) -> int:
    return 1 + (dim - 1 - ax)


def _basis(desc: Desc, ax: int):
    """(s_unknown, s_all, kappa, is_sine) of a bounded axis."""
    h = desc.h(ax)
    off = 0.5 if desc.staggered else 0.0
    lo, hi = desc.unknown_range(ax)
    s_all = (np.arange(desc.nodes(ax)) + off) * h
    s_unk = s_all[lo:hi]
    nu = hi - lo
    bc = desc.bc[ax]
    if bc == "D":
        m = np.arange(1, nu + 1, dtype=np.float64)
    elif bc == "N":
        m = np.arange(0, nu, dtype=np.float64)
    elif bc in ("DN", "ND"):
        m = np.arange(0, nu, dtype=np.float64) + 0.5
    else:
        raise ValueError("bounded axes only")
    kappa = math.pi * m / desc.length(ax)
    return s_unk, s_all, kappa, bc in ("D", "DN")


def derivative(desc: Desc, v: np.ndarray, ax: int, order: int) -> np.ndarray:
    """d^order / dx_ax of the series of the fields v [comp][nodes...], at every node."""
    dim = desc.dim
    v = np.asarray(v, dtype=np.float64)
    # the series vanishes on regular Dirichlet face nodes of the other axes
    w = np.zeros_like(v)
    sl = [slice(None)] * v.ndim
    for b in range(dim):
        lo, hi = desc.unknown_range(b)
        sl[_np_axis(dim, b)] = slice(lo, hi) if b != ax else slice(None)
    w[tuple(sl)] = v[tuple(sl)]
    s_unk, s_all, kappa, sine = _basis(desc, ax)
    arg_u = np.outer(s_unk, kappa)
    phi = np.sin(arg_u) if sine else np.cos(arg_u)  # [unknown node][mode]
    arg_a = np.outer(s_all, kappa)
    if order == 1:
        dphi = kappa * (np.cos(arg_a) if sine else -np.sin(arg_a))
    else:
        dphi = -kappa ** 2 * (np.sin(arg_a) if sine else np.cos(arg_a))
    lo, hi = desc.unknown_range(ax)
    nax = _np_axis(dim, ax)
    vu = np.take(w, np.arange(lo, hi), axis=nax)
    vu = np.moveaxis(vu, nax, -1)  # [..., unknown node]
    coef = np.linalg.solve(phi, vu.reshape(-1, hi - lo).T).T  # series coefficients
    out = coef @ dphi.T  # [..., node]
    out = out.reshape(vu.shape[:-1] + (len(s_all),))
    return np.moveaxis(out, -1, nax)


def apply(desc: Desc, psi: np.ndarray) -> np.ndarray:
    """Operator outputs [nop][nodes...] of the solution psi [ncomp][nodes...]."""
    dim, op = desc.dim, desc.op
    d1 = lambda c, a: derivative(desc, psi[c:c + 1], a, 1)[0]
    if op == "GRAD":
        return np.stack([d1(0, a) for a in range(dim)])
    if op == "DIV":
        return sum(d1(a, a) for a in range(dim))[None]
    if op == "CURL":
        if dim == 3:
            return np.stack([d1(2, 1) - d1(1, 2), d1(0, 2) - d1(2, 0), d1(1, 0) - d1(0, 1)])
        return np.stack([d1(0, 1), -d1(0, 0)])
    if op == "NABLA":
        return np.stack([sum(derivative(desc, psi[c:c + 1], a, 2)[0] for a in range(dim))
                         for c in range(psi.shape[0])])
    raise ValueError(f"unknown operator {op}")
