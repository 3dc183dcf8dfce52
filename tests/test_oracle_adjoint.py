"""Pins for the oracle's adjoint: dense transpose on tiny grids and dot-product tests."""
import numpy as np
import pytest

import oracle
from oracle.desc import Desc


def forward_matrix(desc, faces=None):
    shape = (desc.ncomp,) + desc.shape()
    nin = int(np.prod(shape))
    cols = []
    for i in range(nin):
        e = np.zeros(nin)
        e[i] = 1.0
        psi, op = oracle.solve(desc, e.reshape(shape))
        parts = [psi.ravel()]
        if op is not None:
            parts.append(op.ravel())
        cols.append(np.concatenate(parts))
    return np.array(cols).T


CASES = [
    Desc(3, (4, 4, 4), (-0.5,) * 3, (0.5,) * 3, ("U",) * 3, True, op="CURL", ncomp=3, rhs_scale=-1.0, sigma=0.2),
    Desc(2, (6, 4), (-0.5,) * 2, (0.5, 0.3), ("U",) * 2, True, op="GRAD", ncomp=1, rhs_scale=2.0, sigma=0.1),
    Desc(3, (4, 4, 4), (0,) * 3, (1,) * 3, ("D", "N", "D"), False, "FD2", rhs_scale=0.5),
    Desc(3, (4, 5, 4), (0,) * 3, (1,) * 3, ("N", "N", "D"), True, "PS"),
    Desc(2, (6, 4), (0,) * 2, (1, 2), ("N", "N"), False, "FD2"),
    Desc(3, (4, 4, 6), (0,) * 3, (1,) * 3, ("P",) * 3, True, "PS", op="CURL", ncomp=3),
    Desc(2, (8, 6), (0,) * 2, (1,) * 2, ("P",) * 2, True, "FD2", op="DIV", ncomp=2),
    Desc(3, (4, 3, 4), (0,) * 3, (1,) * 3, ("DN", "N", "ND"), False, "FD2", rhs_scale=0.5),
    Desc(2, (5, 4), (0,) * 2, (1, 2), ("ND", "DN"), True, "PS"),
    # operators on Dirichlet / Neumann axes (derivatives of the basis series)
    Desc(3, (4, 3, 4), (0,) * 3, (1,) * 3, ("D", "N", "DN"), False, "FD2", op="GRAD", ncomp=1),
    Desc(2, (5, 4), (0,) * 2, (1, 2), ("ND", "DN"), True, "PS", op="CURL", ncomp=1),
    Desc(2, (6, 4), (0,) * 2, (1, 1.5), ("D", "N"), False, "PS", op="NABLA", ncomp=1, rhs_scale=0.7),
    Desc(3, (4, 4, 3), (0,) * 3, (1,) * 3, ("N", "D", "N"), True, "PS", op="DIV", ncomp=3),
    Desc(1, (8,), (0.0,), (1.0,), ("DN",), False, "PS", op="GRAD", ncomp=1),
    # unbounded solves on regular grids: N_c + 1 nodes, doubled length 2^p or 3 * 2^p >= 2 N_c + 1
    Desc(3, (4, 3, 4), (-0.5,) * 3, (0.5, 0.4, 0.5), ("U",) * 3, False, op="CURL", ncomp=3, rhs_scale=-1.0,
         sigma=0.2),
    Desc(2, (5, 4), (-0.5,) * 2, (0.5, 0.3), ("U",) * 2, False, op="GRAD", ncomp=1, rhs_scale=2.0, sigma=0.1),
    Desc(1, (6,), (-0.5,), (0.5,), ("U",), False, op="GRAD", ncomp=1, kernel="SPECT"),
    Desc(2, (4, 5), (-0.5,) * 2, (0.5, 0.5), ("U",) * 2, False, op="NABLA", ncomp=1, sigma=0.15),
    # semi-unbounded: one unbounded axis, the others periodic
    Desc(2, (6, 5), (0.0, -0.5), (1.0, 0.5), ("P", "U"), True, "PS", op="GRAD", ncomp=1, rhs_scale=-1.0),
    Desc(3, (4, 4, 5), (0.0,) * 3, (1.0,) * 3, ("P", "U", "P"), False, "FD2", op="CURL", ncomp=3),
    Desc(2, (5, 4), (0.0,) * 2, (1.0, 2.0), ("U", "P"), True, "PS", op="NABLA", ncomp=1, rhs_scale=0.5),
]


@pytest.mark.parametrize("desc", CASES, ids=lambda d: f"{d.dim}D-{'-'.join(d.bc)}-{d.op}")
def test_adjoint_is_dense_transpose(desc):
    A = forward_matrix(desc)
    rng = np.random.default_rng(0)
    g = rng.normal(size=A.shape[0])
    npsi = desc.ncomp * int(np.prod(desc.shape()))
    g_psi = g[:npsi]
    g_op = g[npsi:] if desc.op != "NONE" else None
    got = oracle.adjoint_solve(desc, g_psi, g_op).ravel()
    ref = A.T @ g
    np.testing.assert_allclose(got, ref, atol=1e-12 * max(1.0, np.max(np.abs(ref))))


def test_dot_product_identity_larger():
    d = Desc(3, (12, 10, 8), (-0.5,) * 3, (0.5,) * 3, ("U",) * 3, True, op="CURL", ncomp=3,
             rhs_scale=-1.0, sigma=0.1)
    rng = np.random.default_rng(2)
    x = rng.normal(size=(3,) + d.shape())
    gp = rng.normal(size=(3,) + d.shape())
    gu = rng.normal(size=(3,) + d.shape())
    psi, u = oracle.solve(d, x)
    lhs = np.sum(psi * gp) + np.sum(u * gu)
    rhs = np.sum(x * oracle.adjoint_solve(d, gp, gu))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs) + 1e-13
