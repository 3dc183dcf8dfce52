"""Real-to-real transforms of Table 1 as direct O(n^2) sums (FFTW conventions).

The paper names the transforms by type and cites FFTW for their definitions
(Sec. 2.5.1).  With n input samples x_j, unnormalised:

  DST-I   y_k = 2 sum_{j=0}^{n-1} x_j sin(pi (j+1)(k+1) / (n+1))
  DST-II  y_k = 2 sum_{j=0}^{n-1} x_j sin(pi (j+1/2)(k+1) / n)
  DST-III y_k = (-1)^k x_{n-1} + 2 sum_{j=0}^{n-2} x_j sin(pi (j+1)(k+1/2) / n)
  DCT-I   y_k = x_0 + (-1)^k x_{n-1} + 2 sum_{j=1}^{n-2} x_j cos(pi j k / (n-1))
  DCT-II  y_k = 2 sum_{j=0}^{n-1} x_j cos(pi (j+1/2) k / n)
  DCT-III y_k = x_0 + 2 sum_{j=1}^{n-1} x_j cos(pi j (k+1/2) / n)
  DST-IV  y_k = 2 sum_{j=0}^{n-1} x_j sin(pi (j+1/2)(k+1/2) / n)
  DCT-IV  y_k = 2 sum_{j=0}^{n-1} x_j cos(pi (j+1/2)(k+1/2) / n)

Inverses used by the solver (Table 1, backward column):
  DST-I   -> DST-I   / (2(n+1))
  DST-II  -> DST-III / (2n)
  DCT-I   -> DCT-I   / (2(n-1))
  DCT-II  -> DCT-III / (2n)     (Table 1 prints "DST-III" here; read as DCT-III)

Axes with a Dirichlet and a Neumann face (the quarter-wave sine / cosine
bases, modes k + 1/2; the paper's next step beyond equal faces):
  Dirichlet-Neumann regular   DST-III forward (unknowns at nodes 1..n, the
                              Neumann node n carrying half weight), DST-II / (2n) back
  Dirichlet-Neumann staggered DST-IV forward, DST-IV / (2n) back
  Neumann-Dirichlet regular   DCT-III forward (unknowns at nodes 0..n-1, the
                              Neumann node 0 carrying half weight), DCT-II / (2n) back
  Neumann-Dirichlet staggered DCT-IV forward, DCT-IV / (2n) back

Each function builds the transform matrix entry by entry from its definition
and contracts it with the data along one axis.  Pinned in
tests/test_oracle_transforms.py against scipy.fft (same conventions), the
orthogonality relations and the eigenfunction property.
"""
from __future__ import annotations

import numpy as np


def matrix(kind: str, n: int) -> np.ndarray:
    """Transform matrix M with y = M @ x for a length-n input."""
    k = np.arange(n)[:, None].astype(np.float64)
    j = np.arange(n)[None, :].astype(np.float64)
    if kind == "DST1":
        return 2.0 * np.sin(np.pi * (j + 1) * (k + 1) / (n + 1))
    if kind == "DST2":
        return 2.0 * np.sin(np.pi * (j + 0.5) * (k + 1) / n)
    if kind == "DST3":
        m = 2.0 * np.sin(np.pi * (j + 1) * (k + 0.5) / n)
        m[:, n - 1] = (-1.0) ** np.arange(n)
        return m
    if kind == "DCT1":
        if n < 2:
            raise ValueError("DCT-I needs n >= 2")
        m = 2.0 * np.cos(np.pi * j * k / (n - 1))
        m[:, 0] = 1.0
        m[:, n - 1] = (-1.0) ** np.arange(n)
        return m
    if kind == "DCT2":
        return 2.0 * np.cos(np.pi * (j + 0.5) * k / n)
    if kind == "DCT3":
        m = 2.0 * np.cos(np.pi * j * (k + 0.5) / n)
        m[:, 0] = 1.0
        return m
    if kind == "DST4":
        return 2.0 * np.sin(np.pi * (j + 0.5) * (k + 0.5) / n)
    if kind == "DCT4":
        return 2.0 * np.cos(np.pi * (j + 0.5) * (k + 0.5) / n)
    raise ValueError(kind)


def apply(kind: str, x: np.ndarray, axis: int) -> np.ndarray:
    xm = np.moveaxis(np.asarray(x), axis, -1)
    m = matrix(kind, xm.shape[-1])
    return np.moveaxis(xm @ m.T, -1, axis)


FORWARD = {("D", False): "DST1", ("D", True): "DST2", ("N", False): "DCT1", ("N", True): "DCT2",
           ("DN", False): "DST3", ("DN", True): "DST4", ("ND", False): "DCT3", ("ND", True): "DCT4"}
BACKWARD = {("D", False): "DST1", ("D", True): "DST3", ("N", False): "DCT1", ("N", True): "DCT3",
            ("DN", False): "DST2", ("DN", True): "DST4", ("ND", False): "DCT2", ("ND", True): "DCT4"}


def backward_scale(bc: str, staggered: bool, n: int) -> float:
    if bc in ("DN", "ND"):
        return 1.0 / (2.0 * n)
    if bc == "D" and not staggered:
        return 1.0 / (2.0 * (n + 1))
    if bc == "N" and not staggered:
        return 1.0 / (2.0 * (n - 1))
    return 1.0 / (2.0 * n)


def forward(bc: str, staggered: bool, x: np.ndarray, axis: int) -> np.ndarray:
    return apply(FORWARD[(bc, staggered)], x, axis)


def backward(bc: str, staggered: bool, x: np.ndarray, axis: int) -> np.ndarray:
    n = x.shape[axis]
    return apply(BACKWARD[(bc, staggered)], x, axis) * backward_scale(bc, staggered, n)
