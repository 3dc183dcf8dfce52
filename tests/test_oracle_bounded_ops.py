"""Pins for the spectral operators on Dirichlet / Neumann axes (oracle/bounded_ops.py).

A product of single modes, one per axis, is an exact PS solution: with
lap(psi) = s f and f = prod_a phi_a(x_a), psi = -s f / sum_a kappa_a^2.  Its
gradient, divergence, curl and Laplacian are written out here by calculus
(a sine mode differentiates to kappa times the cosine, a cosine to -kappa
times the sine) and compared at every node of the arrays, face nodes
included.  A wrong sign, wavenumber, node placement or face-node rule fails.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from oracle.desc import Desc

# (mode function, derivative) of each kind for the wavenumber k; s = x - X_l
KINDS = {
    "D": (lambda k, s: np.sin(k * s), lambda k, s: k * np.cos(k * s)),
    "N": (lambda k, s: np.cos(k * s), lambda k, s: -k * np.sin(k * s)),
    "DN": (lambda k, s: np.sin(k * s), lambda k, s: k * np.cos(k * s)),
    "ND": (lambda k, s: np.cos(k * s), lambda k, s: -k * np.sin(k * s)),
}


def setup(bcs, stag, n, L, modes, op, ncomp, rhs=0.9):
    dim = len(bcs)
    d = Desc(dim, n, (0.0,) * dim, L, bcs, stag, "PS", op=op, ncomp=ncomp, rhs_scale=rhs)
    s, k = [], []
    for a in range(dim):
        h = L[a] / n[a]
        cnt = d.nodes(a)
        s.append(h * (np.arange(cnt) + (0.5 if stag else 0.0)))
        half = 0.5 if bcs[a] in ("DN", "ND") else 0.0
        k.append(math.pi * (modes[a] + half) / L[a])
    return d, s, k


def outer(vecs):
    """[z][y][x] product of per-axis vectors given in x, y, z order."""
    out = vecs[0]
    for v in vecs[1:]:
        out = np.multiply.outer(v, out)
    return out


def mode_field(bcs, s, k, deriv_axis=None):
    vecs = []
    for a, bc in enumerate(bcs):
        f, df = KINDS[bc]
        vecs.append(df(k[a], s[a]) if a == deriv_axis else f(k[a], s[a]))
    return outer(vecs)


def mask_faces(d, arr):
    """Zero the regular Dirichlet face nodes (the series vanishes there)."""
    out = arr.copy()
    for a in range(d.dim):
        lo, hi = d.unknown_range(a)
        idx = [slice(None)] * d.dim
        nax = d.dim - 1 - a
        for j in list(range(0, lo)) + list(range(hi, d.nodes(a))):
            idx[nax] = j
            out[tuple(idx)] = 0.0
    return out


CASES3 = [("D", "N", "DN"), ("N", "ND", "D"), ("DN", "DN", "ND"), ("ND", "D", "N")]


@pytest.mark.parametrize("bcs", CASES3, ids=lambda b: "-".join(b))
@pytest.mark.parametrize("stag", [False, True])
def test_grad_of_a_mode_3d(bcs, stag):
    n, L, modes = (8, 6, 10), (1.0, 0.7, 1.3), (2, 3, 1)
    d, s, k = setup(bcs, stag, n, L, modes, "GRAD", 1)
    f = mask_faces(d, mode_field(bcs, s, k))
    psi, g = oracle.solve(d, f[None])
    scale = -0.9 / sum(kk * kk for kk in k)
    np.testing.assert_allclose(psi[0], scale * f, atol=1e-13)
    for a in range(3):
        exact = mask_faces_except(d, scale * mode_field(bcs, s, k, deriv_axis=a), a)
        np.testing.assert_allclose(g[a], exact, atol=1e-12)


def mask_faces_except(d, arr, keep_axis):
    """Zero regular Dirichlet face nodes of every axis but keep_axis."""
    out = arr.copy()
    for a in range(d.dim):
        if a == keep_axis:
            continue
        lo, hi = d.unknown_range(a)
        idx = [slice(None)] * d.dim
        nax = d.dim - 1 - a
        for j in list(range(0, lo)) + list(range(hi, d.nodes(a))):
            idx[nax] = j
            out[tuple(idx)] = 0.0
    return out


@pytest.mark.parametrize("bcs", [("D", "N"), ("DN", "ND"), ("N", "D"), ("ND", "DN")], ids=lambda b: "-".join(b))
@pytest.mark.parametrize("stag", [False, True])
def test_curl_and_nabla_2d(bcs, stag):
    n, L, modes = (12, 8), (1.2, 0.9), (3, 2)
    d, s, k = setup(bcs, stag, n, L, modes, "CURL", 1)
    f = mask_faces(d, mode_field(bcs, s, k))
    _, u = oracle.solve(d, f[None])
    scale = -0.9 / sum(kk * kk for kk in k)
    np.testing.assert_allclose(u[0], mask_faces_except(d, scale * mode_field(bcs, s, k, 1), 1), atol=1e-12)
    np.testing.assert_allclose(u[1], -mask_faces_except(d, scale * mode_field(bcs, s, k, 0), 0), atol=1e-12)
    # NABLA of a PS solution returns s f on the unknowns (zero on Dirichlet face nodes)
    d2, _, _ = setup(bcs, stag, n, L, modes, "NABLA", 1)
    _, lap = oracle.solve(d2, f[None])
    np.testing.assert_allclose(lap[0], 0.9 * f, atol=1e-11)


@pytest.mark.parametrize("bcs", CASES3[:2], ids=lambda b: "-".join(b))
@pytest.mark.parametrize("stag", [False, True])
def test_div_and_curl_3d(bcs, stag):
    # psi_c = (c + 1) * mode: DIV = sum_a (a + 1) d_a mode; CURL from the same partials
    n, L, modes = (6, 8, 6), (1.0, 1.1, 0.8), (1, 2, 3)
    scale = -0.9 / sum((math.pi * (m + (0.5 if b in ("DN", "ND") else 0)) / l) ** 2
                       for m, b, l in zip(modes, bcs, L))
    d, s, k = setup(bcs, stag, n, L, modes, "DIV", 3)
    base = mask_faces(d, mode_field(bcs, s, k))
    f = np.stack([(c + 1) * base for c in range(3)])
    _, div = oracle.solve(d, f)
    part = [mask_faces_except(d, scale * mode_field(bcs, s, k, a), a) for a in range(3)]
    np.testing.assert_allclose(div[0], sum((a + 1) * part[a] for a in range(3)), atol=1e-12)
    dc, _, _ = setup(bcs, stag, n, L, modes, "CURL", 3)
    _, u = oracle.solve(dc, f)
    np.testing.assert_allclose(u[0], 3 * part[1] - 2 * part[2], atol=1e-12)
    np.testing.assert_allclose(u[1], 1 * part[2] - 3 * part[0], atol=1e-12)
    np.testing.assert_allclose(u[2], 2 * part[0] - 1 * part[1], atol=1e-12)


@pytest.mark.parametrize("bc", ["D", "N", "DN", "ND"])
@pytest.mark.parametrize("stag", [False, True])
def test_1d_grad_of_every_mode(bc, stag):
    # every mode of the basis at once: the series is exact for any combination
    n, L = 10, 1.5
    d = Desc(1, (n,), (0.0,), (L,), (bc,), stag, "PS", op="GRAD", rhs_scale=1.0)
    lo, hi = d.unknown_range(0)
    nu = hi - lo
    rng = np.random.default_rng(4)
    amp = rng.normal(size=nu)
    s = (np.arange(d.nodes(0)) + (0.5 if stag else 0.0)) * (L / n)
    first = 1 if bc == "D" else 0
    half = 0.5 if bc in ("DN", "ND") else 0.0
    f_fun, df_fun = KINDS[bc]
    f = np.zeros(d.nodes(0))
    dpsi = np.zeros(d.nodes(0))
    for j in range(nu):
        kk = math.pi * (first + j + half) / L
        if kk == 0.0:
            continue  # the Neumann zero mode has no solution component
        f += amp[j] * f_fun(kk, s)
        dpsi += -amp[j] / kk ** 2 * df_fun(kk, s)
    f[:lo] = 0.0
    f[hi:] = 0.0
    _, g = oracle.solve(d, f[None])
    np.testing.assert_allclose(g[0], dpsi, atol=1e-11)


def test_fd2_uses_the_exact_wavenumbers_for_first_derivatives():
    # FD2 changes psi, not the derivative rule: GRAD equals the series derivative of psi
    d = Desc(2, (10, 12), (0.0, 0.0), (1.0, 1.0), ("D", "N"), False, "FD2", op="GRAD")
    f = np.random.default_rng(8).normal(size=d.shape())
    psi, g = oracle.solve(d, f[None])
    dp = Desc(2, (10, 12), (0.0, 0.0), (1.0, 1.0), ("D", "N"), False, "PS", op="NONE")
    from oracle import bounded_ops
    np.testing.assert_allclose(g[0], bounded_ops.derivative(dp, psi, 0, 1)[0], atol=1e-12)
    assert np.max(np.abs(g)) > 0
