"""Gaussian-regularised Green's functions (Sec. 2.6.2, the order-2 kernel "G2").

Convention: -lap G = zeta_sigma, the normalised Gaussian of width sigma, so
that G > 0 and the solution of lap(psi) = s f is psi = -s (G * f).

  3D:  G(r) = erf(r / (sigma sqrt 2)) / (4 pi r),       G(0) = sqrt(2) / (4 pi^{3/2} sigma)
  2D:  G(r) = -(1/(2 pi)) [ln r + E1(r^2 / (2 sigma^2)) / 2],
       G(0) = (1/(2 pi)) (gamma/2 - ln(sqrt(2) sigma))

(The paper names the kernels but prints no formula; these are the standard
Gaussian-smoothed kernels and their r -> 0 limits.)  erf and E1 come from
scipy.special.

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


def green(dim: int, r: np.ndarray, sigma: float) -> np.ndarray:
    return g2_3d(r, sigma) if dim == 3 else g2_2d(r, sigma)
