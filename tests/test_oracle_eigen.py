"""Pins for the Table 1 eigenvalues.

FD2: the column must be the spectrum of the explicit 3-point second-difference
matrix with the ghost-node rule of each boundary/grid type (built here from
the stencil, independent of any transform).  PS: the inverse transform's basis
functions must be the sampled continuous eigenfunctions whose second
derivative gives the PS value.  Golden: closed-form values for N_c = 4.
"""
import math
import os

import numpy as np
import pytest

from oracle import eigen, r2r


def fd_matrix(bc, staggered, nc, h):
    """3-point Laplacian on the unknowns with homogeneous ghost-node rules."""
    if bc == "P":
        n = nc
        A = np.zeros((n, n))
        for i in range(n):
            A[i, i] = -2
            A[i, (i - 1) % n] += 1
            A[i, (i + 1) % n] += 1
        return A / h ** 2
    if bc == "D" and not staggered:  # unknowns at nodes 1..nc-1, psi_0 = psi_nc = 0
        n = nc - 1
        A = np.diag(-2.0 * np.ones(n)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)
        return A / h ** 2
    if bc == "D" and staggered:  # ghost psi_-1 = -psi_0
        n = nc
        A = np.diag(-2.0 * np.ones(n)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)
        A[0, 0] = -3
        A[-1, -1] = -3
        return A / h ** 2
    if bc == "N" and not staggered:  # unknowns at nodes 0..nc, ghost psi_-1 = psi_1
        n = nc + 1
        A = np.diag(-2.0 * np.ones(n)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)
        A[0, 1] = 2
        A[-1, -2] = 2
        return A / h ** 2
    if bc == "N" and staggered:  # ghost psi_-1 = psi_0
        n = nc
        A = np.diag(-2.0 * np.ones(n)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)
        A[0, 0] = -1
        A[-1, -1] = -1
        return A / h ** 2
    if bc in ("DN", "ND"):
        # one Dirichlet and one Neumann face: unknowns are the N_c nodes off the
        # Dirichlet face (regular) or the N_c cells (staggered)
        n = nc
        A = np.diag(-2.0 * np.ones(n)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)
        d_end, n_end = (0, n - 1) if bc == "DN" else (n - 1, 0)
        if staggered:
            A[d_end, d_end] = -3  # ghost = -psi at a Dirichlet face
            A[n_end, n_end] = -1  # ghost = psi at a Neumann face
        else:
            # Dirichlet face node is data (zero here); Neumann face node is an
            # unknown with ghost psi_{n+1} = psi_{n-1}
            if n > 1:
                A[n_end, n_end - 1 if n_end > 0 else 1] = 2
            else:
                A[0, 0] = -2
        return A / h ** 2
    raise ValueError


CASES = [("P", True), ("D", False), ("D", True), ("N", False), ("N", True),
         ("DN", False), ("DN", True), ("ND", False), ("ND", True)]


@pytest.mark.parametrize("bc,stag", CASES)
@pytest.mark.parametrize("nc", [4, 7, 16])
def test_fd2_is_stencil_spectrum(bc, stag, nc):
    L = 1.7
    h = L / nc
    A = fd_matrix(bc, stag, nc, h)
    n = A.shape[0]
    lam = eigen.eigenvalues(bc, stag, "FD2", n, L, h)
    ev = np.sort(np.linalg.eigvals(A).real)
    np.testing.assert_allclose(np.sort(lam), ev, rtol=1e-10, atol=1e-9)


@pytest.mark.parametrize("bc,stag", [c for c in CASES if c[0] != "P"])
def test_fd2_eigenvectors_are_transform_basis(bc, stag):
    # each row of the inverse transform is an eigenvector of the stencil matrix
    nc, L = 8, 1.0
    h = L / nc
    A = fd_matrix(bc, stag, nc, h)
    n = A.shape[0]
    lam = eigen.eigenvalues(bc, stag, "FD2", n, L, h)
    basis = r2r.backward(bc, stag, np.eye(n), 0)  # column k = k-th basis vector
    for k in range(n):
        v = basis[:, k]
        np.testing.assert_allclose(A @ v, lam[k] * v, atol=1e-9 * max(1, abs(lam[k])))


@pytest.mark.parametrize("bc,stag", [c for c in CASES if c[0] != "P"])
def test_ps_basis_is_continuous_eigenfunction(bc, stag):
    # the transform's k-th basis vector samples sin/cos(pi m x / L) at the grid
    # nodes of Eq. gridpos; the PS eigenvalue is that function's -(pi m/L)^2
    nc, L, lo = 12, 2.5, -0.3
    h = L / nc
    if bc == "D" and not stag:
        x = lo + h * np.arange(1, nc)
    elif bc == "N" and not stag:
        x = lo + h * np.arange(nc + 1)
    elif bc == "DN" and not stag:
        x = lo + h * np.arange(1, nc + 1)
    elif bc == "ND" and not stag:
        x = lo + h * np.arange(nc)
    else:
        x = lo + h * (np.arange(nc) + 0.5)
    n = len(x)
    basis = r2r.backward(bc, stag, np.eye(n), 0)
    lam = eigen.eigenvalues(bc, stag, "PS", n, L, h)
    half = bc in ("DN", "ND")  # quarter-wave modes: m = k + 1/2
    for k in range(n):
        m = math.sqrt(-lam[k]) * L / math.pi
        mm = round(m - 0.5) + 0.5 if half else round(m)
        assert abs(m - mm) < 1e-9
        fn = np.sin if bc in ("D", "DN") else np.cos
        ref = fn(math.pi * mm * (x - lo) / L)
        v = basis[:, k]
        scale = np.dot(v, ref) / np.dot(ref, ref)
        np.testing.assert_allclose(v, scale * ref, atol=1e-12)


def test_ps_periodic_mirrored():
    lam = eigen.eigenvalues("P", True, "PS", 8, 2 * math.pi, 2 * math.pi / 8)
    np.testing.assert_allclose(lam, -np.array([0, 1, 2, 3, 4, 3, 2, 1]) ** 2.0)


def test_golden_table1_n4():
    path = os.path.join(os.path.dirname(__file__), "golden", "table1_fd2_n4.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    for bc, grid, k, val in rows:
        stag = grid == "staggered"
        nc = 4
        n = {"D": nc - 1 if not stag else nc, "N": nc + 1 if not stag else nc, "P": nc}[bc]
        lam = eigen.eigenvalues(bc, stag, "FD2", n, 1.0, 0.25)
        assert abs(lam[int(k)] - float(val)) < 1e-12
