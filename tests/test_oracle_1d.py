"""Pins for the oracle's 1D solves (Sec. 2.4: the 1D solver classes).

  * The 1D spectral kernel: -G'' equals the band-limited delta sin(kc x)/(pi x)
    (fourth-order finite differences of the closed form), G(0) = -1/(pi kc),
    and G + |x|/2 -> 0 in the far field.
  * Unbounded: a resolved Gaussian source gives the exact free-space potential
    (x/2) erf(x/(sqrt2 s)) + s/sqrt(2 pi) exp(-x^2/(2 s^2)) of -d^2/dx^2 to
    rounding, and its exact derivative and Laplacian through GRAD / NABLA.
  * PS: single eigenmodes of every boundary type are solved exactly.
  * FD2: a dense LU solve of the assembled 3-point system, the stencil
    residual with inhomogeneous face values, and second-order convergence to a
    manufactured solution whose face data are its values and derivatives.
"""
import math

import numpy as np
import pytest
from scipy import special

import oracle
from oracle.desc import Desc
from oracle.green import green
from tests.test_oracle_bounded import assemble_fd, stencil_residual


def coords(d):
    h = d.h(0)
    cnt = d.nodes(0)
    if d.staggered:
        return d.lo[0] + h * (np.arange(cnt) + 0.5)
    return d.lo[0] + h * np.arange(cnt)


def test_spectral_1d_kernel_closed_form():
    kc = 7.0
    x = np.linspace(0.05, 6.0, 400)
    e = 1e-3
    g = lambda v: green(1, v, 0.0, "SPECT", kc)
    d2 = (-g(x + 2 * e) + 16 * g(x + e) - 30 * g(x) + 16 * g(x - e) - g(x - 2 * e)) / (12 * e * e)
    np.testing.assert_allclose(-d2, np.sin(kc * x) / (math.pi * x), atol=1e-6)
    assert abs(g(np.array(0.0)) + 1.0 / (math.pi * kc)) < 1e-15
    # even, and its far field is the free-space kernel -|x|/2
    np.testing.assert_allclose(g(-x), g(x), rtol=0, atol=0)
    far = np.array([50.0, 200.0, 1000.0])
    assert np.all(np.abs(g(far) + far / 2) <= 1.0 / (math.pi * kc * kc * far) + 1e-12)


@pytest.mark.parametrize("stag", [True, False])
@pytest.mark.parametrize("op", ["NONE", "GRAD", "NABLA"])
def test_unbounded_1d_gaussian_is_exact(stag, op):
    n = 96
    d = Desc(1, (n,), (-1.0,), (1.3,), ("U",), stag, op=op, rhs_scale=0.7, kernel="SPECT")
    x = coords(d)
    s, x0 = 5 * d.h(0), 0.1
    u = x - x0
    f = np.exp(-u * u / (2 * s * s)) / (math.sqrt(2 * math.pi) * s)
    psi, out = oracle.solve(d, f[None])
    exact = 0.7 * (u / 2 * special.erf(u / (math.sqrt(2) * s)) + s / math.sqrt(2 * math.pi) * np.exp(-u * u / (2 * s * s)))
    np.testing.assert_allclose(psi[0], exact, atol=1e-12)
    if op == "GRAD":
        np.testing.assert_allclose(out[0], 0.7 * 0.5 * special.erf(u / (math.sqrt(2) * s)), atol=1e-12)
    if op == "NABLA":
        np.testing.assert_allclose(out[0], 0.7 * f, atol=1e-10 * np.max(f))


BCS = [("P", 2.0), ("D", 1.0), ("N", 1.0), ("DN", 0.5), ("ND", 0.5)]


@pytest.mark.parametrize("bc,period", BCS, ids=[b for b, _ in BCS])
@pytest.mark.parametrize("stag", [True, False])
def test_ps_eigenmodes_exact(bc, period, stag):
    # f = mode with wavenumber k; PS solves lap psi = s f exactly: psi = -s f / k^2
    if bc == "P" and not stag:
        stag = True  # periodic grids carry N cells either way
    n, L = 24, 1.7
    d = Desc(1, (n,), (0.0,), (L,), (bc,), stag, "PS", rhs_scale=1.3)
    x = coords(d)
    m = 5
    k = math.pi * (m + (0.5 if bc in ("DN", "ND") else 0.0)) / L
    if bc == "P":
        k = 2 * math.pi * m / L
        f = np.cos(k * x + 0.4)
    elif bc in ("D", "DN"):
        f = np.sin(k * x)
    else:
        f = np.cos(k * x)
    psi, _ = oracle.solve(d, f[None])
    np.testing.assert_allclose(psi[0], -1.3 * f / (k * k), atol=1e-13)


@pytest.mark.parametrize("bc,stag", [("D", True), ("D", False), ("DN", True), ("DN", False), ("ND", True),
                                     ("ND", False)])
def test_fd2_dense_lu_1d(bc, stag):
    d = Desc(1, (9,), (0.0,), (1.4,), (bc,), stag, "FD2")
    f = np.random.default_rng(5).normal(size=d.shape())
    psi, _ = oracle.solve(d, f[None])
    A = assemble_fd(d)
    a, b = d.unknown_range(0)
    ref = np.linalg.solve(A, f[a:b])
    np.testing.assert_allclose(psi[0][a:b], ref, atol=1e-11)


@pytest.mark.parametrize("bc,stag", [("D", True), ("D", False), ("DN", True), ("ND", False), ("N", True)])
def test_fd2_residual_inhomogeneous_1d(bc, stag):
    d = Desc(1, (16,), (0.0,), (1.0,), (bc,), stag, "FD2", rhs_scale=0.6)
    f = np.random.default_rng(6).normal(size=d.shape())
    faces = {(0, 0): np.array(0.35), (0, 1): np.array(-0.8)}
    if bc == "N":
        # all-Neumann: the source must balance the face fluxes; the 1D compatible
        # mean is fixed by the discrete divergence theorem of the stencil
        h = d.h(0)
        f = f - f.mean() + (faces[(0, 1)] - faces[(0, 0)]) / (0.6 * h * len(f))
    psi, _ = oracle.solve(d, f[None], faces)
    res = stencil_residual(d, psi[0], faces, f)
    assert np.max(np.abs(res)) < 1e-9 * np.max(np.abs(f))


@pytest.mark.parametrize("bc", ["D", "DN", "ND"])
@pytest.mark.parametrize("stag", [True, False])
def test_fd2_second_order_with_inhomogeneous_faces_1d(bc, stag):
    # psi = sin 2x + 0.3 x^2 on [0, 1.3]; Dirichlet faces carry psi, Neumann faces psi'
    L = 1.3
    psi_f = lambda x: np.sin(2 * x) + 0.3 * x * x
    dpsi_f = lambda x: 2 * np.cos(2 * x) + 0.6 * x
    errs = []
    for n in (32, 64, 128):
        d = Desc(1, (n,), (0.0,), (L,), (bc,), stag, "FD2")
        x = coords(d)
        f = -4 * np.sin(2 * x) + 0.6
        faces = {}
        for side, xf in ((0, 0.0), (1, L)):
            faces[(0, side)] = np.array(psi_f(xf) if d.face(0, side) == "D" else dpsi_f(xf))
        psi, _ = oracle.solve(d, f[None], faces)
        errs.append(np.max(np.abs(psi[0] - psi_f(x))))
    rate = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rate) > 1.8, (errs, rate)
