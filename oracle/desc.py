"""Problem description used by the oracle (its own type; not shared with the library).

Fields mirror the solver options of Sec. 2.4: dimension, cell counts N_c per
axis, domain bounds X_l/X_u (Eq. gridpos), boundary type per axis ('P'
periodic, 'D' Dirichlet, 'N' Neumann, 'U' unbounded), grid type, eigenvalue
type ('PS' or 'FD2', Sec. 2.5.2), spectral operator (Sec. 2.4.3), number of
field components (1, or 3 for the vector solver) and rhs_scale: the oracle
solves lap(psi) = rhs_scale * f.
"""
from __future__ import annotations

import dataclasses
from typing import Tuple


@dataclasses.dataclass
class Desc:
    dim: int
    n: Tuple[int, ...]  # cells per axis (x, y[, z])
    lo: Tuple[float, ...]
    hi: Tuple[float, ...]
    bc: Tuple[str, ...]  # per axis: 'P', 'D', 'N', 'U', or 'DN' / 'ND' (lower face, upper face)
    staggered: bool = True
    eig: str = "PS"  # 'PS' or 'FD2'
    op: str = "NONE"  # 'NONE', 'GRAD', 'DIV', 'CURL', 'NABLA'
    ncomp: int = 1
    rhs_scale: float = 1.0
    sigma: float = 0.0  # Gaussian core width of the regularised Green's function
    kernel: str = "G2"  # unbounded kernel: Gaussian regularisation of order 2, 4, 6, 8 or 10

    def h(self, ax: int) -> float:
        return (self.hi[ax] - self.lo[ax]) / self.n[ax]

    def length(self, ax: int) -> float:
        return self.hi[ax] - self.lo[ax]

    def face(self, ax: int, side: int) -> str:
        """Boundary type of one face of an axis ('P', 'D', 'N', 'U')."""
        b = self.bc[ax]
        return b[side] if len(b) == 2 else b

    def nodes(self, ax: int) -> int:
        """Node count of the input/output array along an axis (Sec. 2.4.2)."""
        if self.bc[ax] in ("D", "N", "DN", "ND", "U") and not self.staggered:
            return self.n[ax] + 1
        return self.n[ax]

    def unknown_range(self, ax: int) -> Tuple[int, int]:
        """[start, stop) of the unknowns inside the node array.

        On regular grids a Dirichlet face node is given data (filled from the
        face), a Neumann face node is an unknown; staggered and periodic axes
        solve for every node.
        """
        if self.staggered or self.bc[ax] in ("P", "U"):
            return 0, self.nodes(ax)
        lo = 1 if self.face(ax, 0) == "D" else 0
        hi = self.n[ax] if self.face(ax, 1) == "D" else self.n[ax] + 1
        return lo, hi

    def shape(self) -> Tuple[int, ...]:
        """Array shape of one field component in [z][y][x] order."""
        return tuple(self.nodes(ax) for ax in reversed(range(self.dim)))

    def op_components(self) -> int:
        if self.op == "NONE":
            return 0
        if self.op == "GRAD":  # scalar -> vector
            return self.dim
        if self.op == "DIV":  # vector (dim components) -> scalar
            return 1
        if self.op == "CURL":  # 3D: vector -> vector; 2D: scalar (z) -> in-plane vector
            return 3 if self.dim == 3 else 2
        if self.op == "NABLA":
            return self.ncomp
        raise ValueError(self.op)
