"""Pins for the oracle's semi-unbounded solve (one unbounded axis, the others periodic).

  * Brute force: per periodic mode (numpy's FFT along the periodic axes), the
    aperiodic sum along the unbounded axis evaluated directly, O(N^2), with the
    kernels exp(-kappa |z|) / (2 kappa) and -|z| / 2 -- no doubling, no oracle FFT.
  * Continuum: a Gaussian source g(z) (1 + a cos(m x)) on a periodic x axis has
    the closed-form solution psi_0(z) + a cos(m x) psi_m(z) with
      psi_0(z) = (z erf(z / (s sqrt 2)) + s sqrt(2/pi) exp(-z^2 / (2 s^2))) / 2,
      psi_k(z) = -exp(k^2 s^2 / 2) [exp(-k z) erfc((k s^2 - z)/(s sqrt 2))
                                     + exp(k z) erfc((k s^2 + z)/(s sqrt 2))] / (4 k);
    the discrete solve must converge to it at second order (trapezoidal sums
    of a kernel with a kink), for psi and for the spectral d/dz.
  * Operators: d/dx of a single periodic mode, and no y derivative without y dependence.
"""
import math

import numpy as np
import pytest
from scipy import special

import oracle
from oracle import semi
from oracle.desc import Desc


def brute_force(desc, f):
    """psi by numpy FFTs along the periodic axes and direct sums along the unbounded one."""
    dim = desc.dim
    ua = semi.unbounded_axis(desc)
    uax = dim - 1 - ua
    pax = tuple(dim - 1 - a for a in range(dim) if a != ua)
    F = np.fft.fftn(f, axes=pax)
    k2 = np.broadcast_to(semi.kappa2(desc), F.shape)
    z = np.arange(desc.nodes(ua)) * desc.h(ua)
    out = np.zeros_like(F)
    Fm = np.moveaxis(F, uax, -1)
    Om = np.moveaxis(out, uax, -1)
    Km = np.moveaxis(k2, uax, -1)
    for idx in np.ndindex(Fm.shape[:-1]):
        k = math.sqrt(Km[idx][0])
        dz = np.abs(z[:, None] - z[None, :])
        G = np.exp(-k * dz) / (2 * k) if k > 0 else -0.5 * dz
        Om[idx] = -desc.rhs_scale * desc.h(ua) * (G @ Fm[idx])
    return np.fft.ifftn(out, axes=pax).real


@pytest.mark.parametrize("n,bc,stag,eig", [((8, 6), ("P", "U"), True, "PS"), ((6, 7), ("U", "P"), False, "FD2"),
                                           ((6, 4, 5), ("P", "P", "U"), True, "PS"),
                                           ((4, 5, 6), ("U", "P", "P"), False, "PS"),
                                           ((6, 5, 4), ("P", "U", "P"), True, "FD2")])
def test_semi_matches_direct_sums(n, bc, stag, eig):
    dim = len(n)
    d = Desc(dim, n, (-0.5,) * dim, (0.5, 0.8, 0.6)[:dim], bc, stag, eig, rhs_scale=-1.3)
    f = np.random.default_rng(3).normal(size=d.shape())
    psi, _ = oracle.solve(d, f[None])
    np.testing.assert_allclose(psi[0], brute_force(d, f), rtol=1e-11, atol=1e-13)


def _continuum(x, z, s, m, a):
    r2 = math.sqrt(2.0)
    psi0 = 0.5 * (z * special.erf(z / (s * r2)) + s * math.sqrt(2 / math.pi) * np.exp(-z * z / (2 * s * s)))
    k = float(m)
    e = math.exp(0.5 * k * k * s * s)
    psik = -e * (np.exp(-k * z) * special.erfc((k * s * s - z) / (s * r2)) +
                 np.exp(k * z) * special.erfc((k * s * s + z) / (s * r2))) / (4 * k)
    dpsi0 = 0.5 * special.erf(z / (s * r2))
    dpsik = -e * (-k * np.exp(-k * z) * special.erfc((k * s * s - z) / (s * r2)) +
                  k * np.exp(k * z) * special.erfc((k * s * s + z) / (s * r2))) / (4 * k)
    psi = psi0[:, None] + a * np.cos(m * x)[None, :] * psik[:, None]
    dz = dpsi0[:, None] + a * np.cos(m * x)[None, :] * dpsik[:, None]
    return psi, dz


def test_semi_converges_to_the_continuous_solution_at_second_order():
    # x periodic on [0, 2 pi) (PS: the mode cos(3x) is exact), z unbounded on [-1, 1]
    s, m, a = 0.12, 3, 0.7
    errs, derrs = [], []
    for nz in (32, 64, 128):
        nx = 16
        d = Desc(2, (nx, nz), (0.0, -1.0), (2 * math.pi, 1.0), ("P", "U"), True, "PS", op="GRAD", rhs_scale=1.0)
        x = (np.arange(nx) + 0.5) * (2 * math.pi / nx)
        z = -1.0 + (np.arange(nz) + 0.5) * (2.0 / nz)
        g = np.exp(-z * z / (2 * s * s)) / (s * math.sqrt(2 * math.pi))
        f = g[:, None] * (1 + a * np.cos(m * x))[None, :]
        psi, grad = oracle.solve(d, f[None])
        exact, dz = _continuum(x, z, s, m, a)
        errs.append(np.max(np.abs(psi[0] - exact)))
        derrs.append(np.max(np.abs(grad[1] - dz)))
    for e in (errs, derrs):
        order = math.log2(e[1] / e[2])
        assert 1.8 < order < 2.3, e
    assert errs[-1] < 2e-4


def test_semi_periodic_derivative_of_one_mode():
    # a source that is one periodic mode cos(2 pi 2 x) along x gives psi and d/dx psi
    # in that mode only: d/dx psi = -(2 pi 2) tan(2 pi 2 x) psi point by point
    d = Desc(3, (8, 6, 10), (0.0,) * 3, (1.0, 1.5, 1.0), ("P", "P", "U"), True, "PS", op="GRAD", ncomp=1)
    x = (np.arange(8) + 0.5) / 8
    z = (np.arange(10) + 0.5) * 0.1
    fm = (np.cos(2 * math.pi * 2 * x)[None, None, :] * np.exp(-((z - 0.5) ** 2) / 0.02)[:, None, None]
          * np.ones((1, 6, 1)))
    psi, grad = oracle.solve(d, fm[None])
    keep = np.abs(np.cos(2 * math.pi * 2 * x)) > 0.3
    want = -2 * math.pi * 2 * np.tan(2 * math.pi * 2 * x)
    np.testing.assert_allclose((grad[0] / psi[0])[..., keep], np.broadcast_to(want, psi[0].shape)[..., keep],
                               rtol=1e-9)
    # no y dependence in the source: the y derivative vanishes
    assert np.max(np.abs(grad[1])) < 1e-12 * np.max(np.abs(grad[0]))
