"""Spectral eigenvalues of Table 1 (Sec. 2.5.1-2.5.2).

For an axis with n transformed points, domain length L and spacing h = L/N_c,
indexed by the transform's own output index k (FFTW ordering):

  BC / grid            PS                          FD2
  Dirichlet regular    -(pi (k+1)/L)^2             -(4/h^2) sin^2(pi (k+1) / (2(n+1)))
  Dirichlet staggered  -(pi (k+1)/L)^2             -(4/h^2) sin^2(pi (k+1) / (2n))
  Neumann regular      -(pi k/L)^2                 -(4/h^2) sin^2(pi k / (2(n-1)))
  Neumann staggered    -(pi k/L)^2                 -(4/h^2) sin^2(pi k / (2n))
  Periodic             -(2 pi k'/L)^2, k'=min(k, n-k)   -(4/h^2) sin^2(pi k / n)
  Dirichlet-Neumann,   -(pi (k+1/2)/L)^2           -(4/h^2) sin^2(pi (k+1/2) / (2n))
  Neumann-Dirichlet    (either grid; n = N_c unknowns)

Pinned in tests/test_oracle_eigen.py: the FD2 column must equal the spectrum
of the explicit 3-point finite-difference matrix with the ghost-node rules,
and the PS column the second derivative of the continuous eigenfunction.
"""
from __future__ import annotations

import numpy as np


def eigenvalues(bc: str, staggered: bool, eig: str, n: int, L: float, h: float) -> np.ndarray:
    k = np.arange(n, dtype=np.float64)
    if bc == "P":
        if eig == "PS":
            kk = np.where(k < n / 2.0, k, n - k)
            return -(2.0 * np.pi * kk / L) ** 2
        return -(4.0 / h ** 2) * np.sin(np.pi * k / n) ** 2
    if bc == "D":
        m = k + 1.0
        denom = 2.0 * (n + 1) if not staggered else 2.0 * n
    elif bc == "N":
        m = k
        denom = 2.0 * (n - 1) if not staggered else 2.0 * n
    elif bc in ("DN", "ND"):
        m = k + 0.5
        denom = 2.0 * n
    else:
        raise ValueError(bc)
    if eig == "PS":
        return -(np.pi * m / L) ** 2
    return -(4.0 / h ** 2) * np.sin(np.pi * m / denom) ** 2
