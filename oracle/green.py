"""Regularised Green's functions (Sec. 2.6.2): Gaussian kernels "G2" to "G10" (2D, 3D)
and the spectral kernel "SPECT" in 1D, 2D and 3D (a sharp cut-off at the
grid wavenumber pi / max h).

Convention: -lap G = zeta_sigma, the normalised Gaussian of width sigma, so
that G > 0 and the solution of lap(psi) = s f is psi = -s (G * f).

  3D:  G(r) = erf(r / (sigma sqrt 2)) / (4 pi r),       G(0) = sqrt(2) / (4 pi^{3/2} sigma)
  2D:  G(r) = -(1/(2 pi)) [ln r + E1(r^2 / (2 sigma^2)) / 2],
       G(0) = (1/(2 pi)) (gamma/2 - ln(sqrt(2) sigma))

(The paper names the kernels but prints no formula; these are the standard
Gaussian-smoothed kernels and their r -> 0 limits.)  erf and E1 come from
scipy.special.

Order P = 2m (Sec. 2.6.2: P-th order approximations to the inverse Gaussian
regularisation).  Our reading: the smoothing zeta_P has the transform
  zeta_P^(k) = exp(-(k sigma)^2 / 2) * sum_{j<m} (k sigma)^{2j} / (2^j j!),
the Gaussian times the Taylor series of its inverse cut below order P, so
that zeta_P^ = 1 + O(k^P).  In real space zeta_P = sum_{j<m} sigma^{2j} /
(2^j j!) (-lap)^j zeta_sigma, and since -lap G2 = zeta_sigma,
  G_P = G2 + sum_{j=1}^{m-1} sigma^{2j} / (2^j j!) (-lap)^{j-1} zeta_sigma.
With u = r^2/sigma^2, (-lap)^j zeta_sigma = zeta_sigma p_j(u) / sigma^{2j}
where the polynomials follow from the radial Laplacian in d dimensions:
  p_0 = 1,  p_{j+1} = -[4u p_j'' + (2d - 4u) p_j' + (u - d) p_j].
Pinned in tests/test_oracle_unbounded.py against the Fourier definition of
zeta_P (radial quadrature), its vanishing moments, and the order of
convergence on a Gaussian blob.

Pinned in tests/test_oracle_unbounded.py: lap G = -zeta checked by finite
differences of the closed form, the r -> 0 limit, and the Gaussian-blob
closed form erf(r/sqrt(2(s^2+sigma^2)))/(4 pi r).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special

EULER_GAMMA = 0.57721566490153286060651209008240243


def g2_3d(r: np.ndarray, sigma: float) -> np.ndarray:
    r = np.asarray(r, dtype=np.float64)
    safe = np.where(r > 0.0, r, 1.0)
    val = special.erf(safe / (sigma * math.sqrt(2.0))) / (4.0 * math.pi * safe)
    return np.where(r > 0.0, val, math.sqrt(2.0) / (4.0 * math.pi ** 1.5 * sigma))


def g2_2d(r: np.ndarray, sigma: float) -> np.ndarray:
    r = np.asarray(r, dtype=np.float64)
    safe = np.where(r > 0.0, r, 1.0)
    val = -(np.log(safe) + 0.5 * special.exp1(safe * safe / (2.0 * sigma * sigma))) / (2.0 * math.pi)
    g0 = (0.5 * EULER_GAMMA - math.log(math.sqrt(2.0) * sigma)) / (2.0 * math.pi)
    return np.where(r > 0.0, val, g0)


def smoothing_poly(dim: int, j: int) -> np.polynomial.Polynomial:
    """p_j(u) with (-lap)^j zeta_sigma = zeta_sigma p_j(u) / sigma^{2j}, u = r^2 / sigma^2."""
    P = np.polynomial.Polynomial
    p = P([1.0])
    u = P([0.0, 1.0])
    for _ in range(j):
        p = -(4.0 * u * p.deriv(2) + (2.0 * dim - 4.0 * u) * p.deriv(1) + (u - dim) * p)
    return p


def gaussian(dim: int, r: np.ndarray, sigma: float) -> np.ndarray:
    """zeta_sigma: the normalised Gaussian of width sigma in dim dimensions."""
    r = np.asarray(r, dtype=np.float64)
    return np.exp(-r * r / (2.0 * sigma * sigma)) / (2.0 * math.pi * sigma * sigma) ** (dim / 2.0)


def spectral_3d(r: np.ndarray, kc: float) -> np.ndarray:
    """Sharp spectral cut-off in 3D: G^(k) = 1/k^2 for |k| <= kc, 0 beyond, i.e.
    G(r) = Si(kc r) / (2 pi^2 r), G(0) = kc / (2 pi^2).  Si from scipy.special.sici."""
    r = np.asarray(r, dtype=np.float64)
    safe = np.where(r > 0.0, r, 1.0)
    val = special.sici(kc * safe)[0] / (2.0 * math.pi ** 2 * safe)
    return np.where(r > 0.0, val, kc / (2.0 * math.pi ** 2))


def int_one_minus_j0(x: np.ndarray) -> np.ndarray:
    """F(x) = int_0^x (1 - J0(t)) / t dt for x >= 0.

    Integrating J0's power series term by term gives the closed form
    F(x) = (x^2 / 8) 2F3(1, 1; 2, 2, 2; -x^2 / 4), evaluated for every distinct
    argument by mpmath's generalised hypergeometric function at 30 significant
    digits (it switches to its asymptotic expansion for large arguments) and
    rounded to FP64.  Without mpmath, the fallback is adaptive quadrature of
    the integrand (int_one_minus_j0_quad).
    """
    x = np.asarray(x, dtype=np.float64)
    try:
        import mpmath
    except ImportError:
        return int_one_minus_j0_quad(x)
    xs, inv = np.unique(x, return_inverse=True)
    vals = np.empty_like(xs)
    with mpmath.workdps(30):
        for i, v in enumerate(xs):
            if v == 0.0:
                vals[i] = 0.0
                continue
            t = mpmath.mpf(float(v))
            vals[i] = float(t * t / 8 * mpmath.hyp2f3(1, 1, 2, 2, 2, -t * t / 4))
    return vals[inv].reshape(x.shape)


def int_one_minus_j0_quad(x: np.ndarray) -> np.ndarray:
    """F(x) by adaptive quadrature (scipy.integrate.quad, J0 from scipy.special;
    below t = 0.5 the integrand from J0's power series) over chunks of length
    <= 20 between the sorted distinct arguments, accumulated from 0."""
    from scipy import integrate
    x = np.asarray(x, dtype=np.float64)
    xs = np.unique(x)

    def f(t):
        if t < 0.5:  # (1 - J0(t)) / t from J0's series: 1 - J0 cancels for small t
            q, term, acc = 0.25 * t * t, 1.0, 0.0
            for m in range(1, 12):
                term *= -q / (m * m)
                acc -= term
            return acc / t
        return (1.0 - special.j0(t)) / t

    import warnings
    vals = np.empty_like(xs)
    acc, prev = 0.0, 0.0
    with warnings.catch_warnings():
        warnings.simplefilter("ignore", integrate.IntegrationWarning)  # tolerance set at rounding level
        for i, b in enumerate(xs):
            if b > prev:
                # chunks of at most 20 (about three periods of J0) for the oscillatory tail
                edges = np.linspace(prev, b, int(math.ceil((b - prev) / 20.0)) + 1)
                for a0, a1 in zip(edges[:-1], edges[1:]):
                    acc += integrate.quad(f, a0, a1, limit=200, epsabs=1e-17, epsrel=1e-14)[0]
            vals[i] = acc
            prev = b
    return vals[np.searchsorted(xs, x)]


def spectral_2d(r: np.ndarray, kc: float) -> np.ndarray:
    """Sharp spectral cut-off in 2D: G^(k) = 1/k^2 for |k| <= kc.  The inverse
    transform (1/2 pi) int_0^kc J0(k r) / k dk diverges at k = 0, so G is fixed
    up to a constant: G(r) = -(1/2 pi) F(kc r) + C with F(x) = int_0^x
    (1 - J0(t)) / t dt.  Since F(x) - ln x -> gamma - ln 2, the constant
    C = (ln(kc/2) + gamma) / (2 pi) gives G + ln(r) / (2 pi) -> 0 (our reading:
    the far field of the 2D free-space kernel -ln(r) / (2 pi), as the Gaussian
    kernels have).  G(0) = (ln(kc/2) + gamma) / (2 pi)."""
    r = np.asarray(r, dtype=np.float64)
    return (math.log(0.5 * kc) + EULER_GAMMA - int_one_minus_j0(kc * r)) / (2.0 * math.pi)


def spectral_1d(r: np.ndarray, kc: float) -> np.ndarray:
    """Sharp spectral cut-off in 1D (the only kernel the paper uses in 1D,
    Sec. 4.3): -G'' = sin(kc x) / (pi x), the band-limited delta.  Integrating
    twice, G(x) = -(1/pi) [|x| Si(kc |x|) + cos(kc x) / kc], with the free
    constant fixed (our reading) so that G + |x|/2 -> 0 as |x| -> infinity:
    the same far field as the 1D free-space kernel -|x|/2 of -d^2/dx^2.
    G(0) = -1 / (pi kc).  Si from scipy.special.sici."""
    r = np.abs(np.asarray(r, dtype=np.float64))
    si, _ = special.sici(kc * r)
    return -(r * si + np.cos(kc * r) / kc) / math.pi


def green(dim: int, r: np.ndarray, sigma: float, kernel: str = "G2", kc: float = 0.0) -> np.ndarray:
    if kernel == "SPECT":
        if dim == 3:
            return spectral_3d(r, kc)
        if dim == 1:
            return spectral_1d(r, kc)
        return spectral_2d(r, kc)
    if dim == 1:
        raise ValueError("1D unbounded solves use the spectral kernel (Sec. 4.3)")
    g = g2_3d(r, sigma) if dim == 3 else g2_2d(r, sigma)
    order = int(kernel[1:])
    if kernel[0] != "G" or order not in (2, 4, 6, 8, 10):
        raise ValueError(f"unknown kernel {kernel}")
    m = order // 2
    r = np.asarray(r, dtype=np.float64)
    u = r * r / (sigma * sigma)
    corr = np.zeros_like(u)
    for j in range(1, m):
        corr = corr + smoothing_poly(dim, j - 1)(u) * sigma ** 2 / (2.0 ** j * math.factorial(j))
    return g + gaussian(dim, r, sigma) * corr
