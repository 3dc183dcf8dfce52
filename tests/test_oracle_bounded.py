"""Pins for the oracle's bounded solve (Sec. 2.5, Table 1, Sec. 4.1-4.2).

  * PS on manufactured sine/cosine products is exact (Sec. 4.1; the 3D factor
    of Eq. tfb3D is read as -f/((4 pi)^2 (1/Lx^2 + 1/Ly^2 + 1/Lz^2))).
  * FD2: the explicit 7-point stencil with ghost nodes fixed by the face data,
    applied to the oracle's output, reproduces the right-hand side; written
    here independently of any transform.
  * FD2 with inhomogeneous faces is exact for the paraboloid of Eq. tfih1D on
    the grid types whose ghost rule is exact for quadratics, and converges at
    second order on manufactured solutions (Sec. 4.2).
  * A dense LU solve of the assembled FD system on small grids.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
import workloads
from oracle.desc import Desc


def test_periodic_c1_exact():
    pm = workloads.periodic_modes(32, seed_index=0)
    d = Desc(3, (32,) * 3, (0,) * 3, (2 * math.pi,) * 3, ("P",) * 3, True, "PS")
    psi, _ = oracle.solve(d, pm.f)
    assert np.max(np.abs(psi[0] - pm.psi_exact)) < 1e-12


@pytest.mark.parametrize("bc", ["D", "N"])
@pytest.mark.parametrize("stag", [False, True])
def test_paper_sc_test_functions(bc, stag):
    # Eq. tfb: S = sin(4 pi x/L) (Dirichlet), C = cos(4 pi x/L) (Neumann), products in 3D
    n = (16, 12, 20)
    L = (1.0, 2.0, 0.5)
    d = Desc(3, n, (0.0,) * 3, L, (bc,) * 3, stag, "PS")
    coords = []
    for ax in range(3):
        h = L[ax] / n[ax]
        cnt = n[ax] + 1 if not stag else n[ax]
        x = h * (np.arange(cnt) + (0.5 if stag else 0.0))
        fn = np.sin if bc == "D" else np.cos
        coords.append(fn(4 * math.pi * x / L[ax]))
    f = coords[2][:, None, None] * coords[1][None, :, None] * coords[0][None, None, :]
    psi_a = -f / ((4 * math.pi) ** 2 * sum(1 / l ** 2 for l in L))
    psi, _ = oracle.solve(d, f)
    err = psi[0] - psi_a
    if bc == "N":
        err = err - err.mean()  # all-Neumann: solution up to a constant (Sec. 4.2)
    assert np.max(np.abs(err)) < 1e-12 * np.max(np.abs(psi_a))


def stencil_residual(desc, psi, faces, f):
    """Apply the 3-point stencil per axis with ghost nodes from the faces."""
    dim = desc.dim
    usl = []
    for ax in reversed(range(dim)):
        a, b = desc.unknown_range(ax)
        usl.append(slice(a, b))
    u = psi[tuple(usl)]
    lap = np.zeros_like(u)
    for ax in range(dim):
        nax = dim - 1 - ax
        h = desc.h(ax)
        bc = desc.bc[ax]
        n = u.shape[nax]
        # build the padded array with one ghost layer on each side
        pad_shape = list(u.shape)
        pad_shape[nax] += 2
        w = np.zeros(pad_shape)
        inner = [slice(None)] * dim
        inner[nax] = slice(1, n + 1)
        w[tuple(inner)] = u
        for side in (0, 1):
            g = faces.get((ax, side)) if faces else None
            if g is not None:
                gsl = []
                for a2 in reversed(range(dim)):
                    if a2 == ax:
                        continue
                    lo, hi = desc.unknown_range(a2)
                    gsl.append(slice(lo, hi))
                g = np.expand_dims(g[tuple(gsl)], nax)
            else:
                g = 0.0
            ghost = [slice(None)] * dim
            ghost[nax] = slice(0, 1) if side == 0 else slice(n + 1, n + 2)
            near = [slice(None)] * dim
            near[nax] = slice(1, 2) if side == 0 else slice(n, n + 1)
            near2 = [slice(None)] * dim
            near2[nax] = slice(2, 3) if side == 0 else slice(n - 1, n)
            sgn = -1.0 if side == 0 else 1.0
            bc = desc.face(ax, side)
            if bc == "D" and not desc.staggered:
                w[tuple(ghost)] = g  # boundary node value
            elif bc == "D":
                w[tuple(ghost)] = 2 * g - w[tuple(near)]
            elif bc == "N" and not desc.staggered:
                w[tuple(ghost)] = w[tuple(near2)] + sgn * 2 * h * g
            elif bc == "N":
                w[tuple(ghost)] = w[tuple(near)] + sgn * h * g
        lo_s = [slice(None)] * dim
        lo_s[nax] = slice(0, n)
        hi_s = [slice(None)] * dim
        hi_s[nax] = slice(2, n + 2)
        if desc.bc[ax] == "P":
            lap += (np.roll(u, 1, nax) - 2 * u + np.roll(u, -1, nax)) / h ** 2
        else:
            lap += (w[tuple(lo_s)] - 2 * u + w[tuple(hi_s)]) / h ** 2
    return lap - desc.rhs_scale * f[tuple(usl)]


@pytest.mark.parametrize("bcs", list(itertools.product("DN", repeat=3)))
@pytest.mark.parametrize("stag", [False, True])
def test_fd2_residual_inhomogeneous(bcs, stag):
    if bcs == ("N", "N", "N"):
        pytest.skip("all-Neumann needs a compatible source; covered by the paraboloid test")
    man = workloads.manufactured(seed_index=11)
    n = (10, 12, 8)
    case = workloads.bounded_case(man, n, bcs, stag)
    d = Desc(3, n, (0,) * 3, (1.0,) * 3, bcs, stag, "FD2", rhs_scale=0.7)
    f = case["f"] / 0.7
    psi, _ = oracle.solve(d, f, case["faces"])
    res = stencil_residual(d, psi[0], case["faces"], f)
    assert np.max(np.abs(res)) < 1e-9 * np.max(np.abs(f))
    # regular Dirichlet boundary nodes carry the face values
    for ax in range(3):
        if bcs[ax] == "D" and not stag:
            sl = [slice(None)] * 3
            sl[2 - ax] = 0
            # interior of the face (edges may be overwritten by later axes)
            inner = [slice(1, -1)] * 2
            np.testing.assert_allclose(psi[0][tuple(sl)][tuple(inner)], case["faces"][(ax, 0)][tuple(inner)], atol=1e-12)


@pytest.mark.parametrize("bcs,stag", [(("D", "D", "D"), False), (("N", "D", "N"), False),
                                      (("N", "N", "N"), False), (("N", "N", "N"), True),
                                      (("D", "N", "N"), False)])
def test_fd2_exact_for_paraboloid(bcs, stag):
    # Eq. tfih1D: psi_a = a(1-x/L)^2 + b(x/L)^2 per axis, f = 2(a+b)/L^2;
    # Eq. tfih1Dgrad (with the 1/L factor restored) for the Neumann faces.
    n = (8, 6, 10)
    L = (1.0, 1.5, 0.8)
    ab = [(0.3, -1.2), (2.0, 0.5), (-0.7, 1.1)]
    d = Desc(3, n, (0,) * 3, L, bcs, stag, "FD2")
    coords = []
    for ax in range(3):
        h = L[ax] / n[ax]
        cnt = d.nodes(ax)
        coords.append(h * (np.arange(cnt) + (0.5 if stag else 0.0)))

    def par(ax, x):
        a, b = ab[ax]
        return a * (1 - x / L[ax]) ** 2 + b * (x / L[ax]) ** 2

    def dpar(ax, x):
        a, b = ab[ax]
        return (2 * a * (x / L[ax] - 1) + 2 * b * x / L[ax]) / L[ax]

    xs, ys, zs = coords
    psi_a = par(0, xs)[None, None, :] + par(1, ys)[None, :, None] + par(2, zs)[:, None, None]
    f = np.full(psi_a.shape, sum(2 * (a + b) / L[i] ** 2 for i, (a, b) in enumerate(ab)))
    faces = {}
    for ax in range(3):
        for side, xb in ((0, 0.0), (1, L[ax])):
            pts = [xs, ys, zs]
            if bcs[ax] == "D":
                vals = [par(i, p) for i, p in enumerate(pts)]
                vals[ax] = np.array([par(ax, xb)])
            else:
                vals = [np.zeros_like(p) for p in pts]
                vals[ax] = np.array([dpar(ax, xb)])
            face = vals[0][None, None, :] + vals[1][None, :, None] + vals[2][:, None, None]
            faces[(ax, side)] = np.squeeze(face, axis=2 - ax)
    psi, _ = oracle.solve(d, f, faces)
    err = psi[0] - psi_a
    if all(b == "N" for b in bcs):
        err = err - err.mean()
    assert np.max(np.abs(err)) < 1e-10


def test_fd2_second_order_convergence():
    man = workloads.manufactured(seed_index=1)
    errs = []
    ns = (16, 32, 64)
    for n in ns:
        case = workloads.bounded_case(man, (n, n, n), ("D", "N", "D"), False)
        d = Desc(3, (n,) * 3, (0,) * 3, (1,) * 3, ("D", "N", "D"), False, "FD2")
        psi, _ = oracle.solve(d, case["f"], case["faces"])
        errs.append(np.max(np.abs(psi[0] - case["psi_exact"])))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert all(1.85 < o < 2.15 for o in orders), orders


def assemble_fd(desc):
    mats = []
    from tests.test_oracle_eigen import fd_matrix
    for ax in range(desc.dim):
        mats.append(fd_matrix(desc.bc[ax], desc.staggered, desc.n[ax], desc.h(ax)))
    # Kronecker sum in [z][y][x] order
    sizes = [m.shape[0] for m in mats]
    A = 0
    for ax in range(desc.dim):
        parts = []
        for a2 in reversed(range(desc.dim)):
            parts.append(mats[a2] if a2 == ax else np.eye(sizes[a2]))
        K = parts[0]
        for p in parts[1:]:
            K = np.kron(K, p)
        A = A + K
    return A


@pytest.mark.parametrize("bcs,stag", [(("D", "D", "D"), False), (("D", "N", "D"), True),
                                      (("N", "D", "D"), False), (("D", "D", "N"), True)])
def test_fd2_dense_lu(bcs, stag):
    n = (5, 6, 4)
    d = Desc(3, n, (0,) * 3, (1.0, 0.8, 1.3), bcs, stag, "FD2")
    rng = np.random.default_rng(3)
    f = rng.normal(size=d.shape())
    psi, _ = oracle.solve(d, f)
    A = assemble_fd(d)
    usl = tuple(slice(*d.unknown_range(ax)) for ax in reversed(range(3)))
    ref = np.linalg.solve(A, f[usl].ravel()).reshape(f[usl].shape)
    np.testing.assert_allclose(psi[0][usl], ref, atol=1e-11)


def test_2d_periodic_grad_of_modes():
    # GRAD on a periodic 2D field: analytic derivative of the exact potential
    n, L = 32, 2 * math.pi
    x = (np.arange(n) + 0.5) * L / n
    X = x[None, :]
    Y = x[:, None]
    psi_a = np.sin(3 * X) * np.cos(2 * Y)
    f = -13.0 * psi_a
    d = Desc(2, (n, n), (0, 0), (L, L), ("P", "P"), True, "PS", op="GRAD")
    psi, g = oracle.solve(d, f)
    np.testing.assert_allclose(psi[0], psi_a, atol=1e-12)
    np.testing.assert_allclose(g[0], 3 * np.cos(3 * X) * np.cos(2 * Y), atol=1e-11)
    np.testing.assert_allclose(g[1], -2 * np.sin(3 * X) * np.sin(2 * Y), atol=1e-11)


MIXED = [("DN", "D", "N"), ("ND", "N", "D"), ("DN", "ND", "D"), ("N", "DN", "ND")]


@pytest.mark.parametrize("bcs", MIXED)
@pytest.mark.parametrize("stag", [False, True])
def test_fd2_residual_mixed_faces(bcs, stag):
    # one Dirichlet and one Neumann face on an axis (the quarter-wave bases):
    # the explicit stencil with each face's own ghost rule reproduces the rhs
    man = workloads.manufactured(seed_index=12)
    n = (10, 12, 8)
    case = workloads.bounded_case(man, n, bcs, stag)
    d = Desc(3, n, (0,) * 3, (1.0,) * 3, bcs, stag, "FD2", rhs_scale=1.3)
    f = case["f"] / 1.3
    psi, _ = oracle.solve(d, f, case["faces"])
    res = stencil_residual(d, psi[0], case["faces"], f)
    assert np.max(np.abs(res)) < 1e-9 * np.max(np.abs(f))


@pytest.mark.parametrize("bcs,stag", [(("DN", "D", "N"), False), (("ND", "DN", "N"), True),
                                      (("D", "ND", "DN"), False), (("DN", "DN", "ND"), True)])
def test_fd2_dense_lu_mixed_faces(bcs, stag):
    n = (5, 6, 4)
    d = Desc(3, n, (0,) * 3, (1.0, 0.8, 1.3), bcs, stag, "FD2")
    rng = np.random.default_rng(4)
    f = rng.normal(size=d.shape())
    psi, _ = oracle.solve(d, f)
    A = assemble_fd(d)
    usl = tuple(slice(*d.unknown_range(ax)) for ax in reversed(range(3)))
    ref = np.linalg.solve(A, f[usl].ravel()).reshape(f[usl].shape)
    np.testing.assert_allclose(psi[0][usl], ref, atol=1e-11)


@pytest.mark.parametrize("bc", ["DN", "ND"])
@pytest.mark.parametrize("stag", [False, True])
def test_ps_quarter_wave_modes_exact(bc, stag):
    # psi = product of quarter-wave modes sin/cos((m + 1/2) pi x / L) is exact for PS
    n = (12, 10, 8)
    L = (1.0, 1.5, 0.75)
    m = (2, 0, 1)
    d = Desc(3, n, (0.0,) * 3, L, (bc,) * 3, stag, "PS")
    coords = []
    for ax in range(3):
        h = L[ax] / n[ax]
        cnt = d.nodes(ax)
        x = h * (np.arange(cnt) + (0.5 if stag else 0.0))
        fn = np.sin if bc == "DN" else np.cos
        coords.append(fn((m[ax] + 0.5) * math.pi * x / L[ax]))
    psi_a = coords[2][:, None, None] * coords[1][None, :, None] * coords[0][None, None, :]
    lam = -sum(((m[ax] + 0.5) * math.pi / L[ax]) ** 2 for ax in range(3))
    psi, _ = oracle.solve(d, lam * psi_a)
    usl = tuple(slice(*d.unknown_range(ax)) for ax in reversed(range(3)))
    np.testing.assert_allclose(psi[0][usl], psi_a[usl], atol=1e-12)
