"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module only *draws* inputs: source fields, face values, analytic reference
fields and problem descriptions.  It contains none of the solver's arithmetic
(no transforms, no eigenvalues, no Green's functions) so that the CPU oracle and
the CUDA library can both be fed from it without sharing any solver code.

Every generator takes a seed and returns float64 numpy arrays; callers cast to
the precision they need.  Array order is [component][z][y][x] (x fastest).

Workloads follow the paper's validation cases (Sec. 4):
  * manufactured sine/cosine products (Sec. 4.1, Eq. tfb / tfb3D),
  * inhomogeneous face data derived from an analytic potential (Sec. 4.2),
  * compact vorticity distributions for the unbounded solver (Sec. 4.3),
with the concrete sizes of the five benchmark configurations.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Tuple

import numpy as np

BASE_SEED = 1145

# --------------------------------------------------------------------------
# grid helpers (positions only, Eq. gridpos of Sec. 2.4.2)
# --------------------------------------------------------------------------


def node_positions(lo: float, hi: float, n_cells: int, staggered: bool, count: int) -> np.ndarray:
    """Grid coordinates: regular = cell boundaries, staggered = cell centres."""
    h = (hi - lo) / n_cells
    i = np.arange(count, dtype=np.float64)
    return lo + (i + 0.5) * h if staggered else lo + i * h


def rng_for(config_index: int, salt: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(BASE_SEED + config_index + 1000 * salt))


# --------------------------------------------------------------------------
# C1: periodic 64^3 on [0, 2pi)^3, cell centred, sum of 8 sine modes
# --------------------------------------------------------------------------


@dataclasses.dataclass
class PeriodicModes:
    n: int
    k: np.ndarray  # [m, 3] integer wavenumbers (kx, ky, kz)
    a: np.ndarray  # [m] amplitudes
    f: np.ndarray  # [n, n, n] source  (z, y, x)
    psi_exact: np.ndarray  # analytic potential of lap(psi) = f


def periodic_modes(n: int = 64, n_modes: int = 8, seed_index: int = 0, kmax: int = 8) -> PeriodicModes:
    rng = rng_for(seed_index)
    k = rng.integers(1, kmax + 1, size=(n_modes, 3))
    a = rng.uniform(-1.0, 1.0, size=n_modes)
    x = node_positions(0.0, 2 * math.pi, n, True, n)
    f = np.zeros((n, n, n))
    psi = np.zeros((n, n, n))
    for m in range(n_modes):
        sx = np.sin(k[m, 0] * x)[None, None, :]
        sy = np.sin(k[m, 1] * x)[None, :, None]
        sz = np.sin(k[m, 2] * x)[:, None, None]
        mode = a[m] * sz * sy * sx
        f += mode
        psi -= mode / float(k[m, 0] ** 2 + k[m, 1] ** 2 + k[m, 2] ** 2)
    return PeriodicModes(n, k, a, f, psi)


# --------------------------------------------------------------------------
# C2: manufactured sin/cos products with inhomogeneous D/N faces
# --------------------------------------------------------------------------


@dataclasses.dataclass
class Manufactured:
    """psi = sum_m a_m prod_axis phi_{m,axis}(k_{m,axis} * pi * x_axis / L_axis).

    phi is sin or cos (drawn per factor).  f = lap(psi) and the face data are
    analytic.  Coordinates are taken relative to the lower domain bound.
    """

    a: np.ndarray  # [m]
    k: np.ndarray  # [m, 3]  (x, y, z)
    use_cos: np.ndarray  # [m, 3] bool
    lo: Tuple[float, float, float]
    hi: Tuple[float, float, float]

    def _factor(self, m: int, axis: int, x: np.ndarray, deriv: int) -> np.ndarray:
        L = self.hi[axis] - self.lo[axis]
        w = self.k[m, axis] * math.pi / L
        t = w * (x - self.lo[axis])
        if self.use_cos[m, axis]:
            vals = [np.cos(t), -w * np.sin(t), -w * w * np.cos(t)]
        else:
            vals = [np.sin(t), w * np.cos(t), -w * w * np.sin(t)]
        return vals[deriv]

    def field(self, xs, ys, zs, deriv=(0, 0, 0)) -> np.ndarray:
        out = np.zeros((len(zs), len(ys), len(xs)))
        for m in range(len(self.a)):
            fx = self._factor(m, 0, xs, deriv[0])[None, None, :]
            fy = self._factor(m, 1, ys, deriv[1])[None, :, None]
            fz = self._factor(m, 2, zs, deriv[2])[:, None, None]
            out += self.a[m] * fz * fy * fx
        return out

    def laplacian(self, xs, ys, zs) -> np.ndarray:
        return (self.field(xs, ys, zs, (2, 0, 0)) + self.field(xs, ys, zs, (0, 2, 0))
                + self.field(xs, ys, zs, (0, 0, 2)))


def manufactured(n_modes: int = 6, kmax: int = 6, seed_index: int = 1,
                 lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)) -> Manufactured:
    rng = rng_for(seed_index)
    a = rng.uniform(-1.0, 1.0, size=n_modes)
    k = rng.integers(1, kmax + 1, size=(n_modes, 3))
    use_cos = rng.integers(0, 2, size=(n_modes, 3)).astype(bool)
    return Manufactured(a, k, use_cos, tuple(lo), tuple(hi))


def bounded_case(man: Manufactured, n_cells: Tuple[int, int, int], bc: Tuple[str, str, str],
                 staggered: bool) -> Dict[str, object]:
    """Source, faces and exact potential on the solver's node arrays.

    bc[axis] in {'D', 'N', 'P', 'DN', 'ND'} ('DN': Dirichlet lower face,
    Neumann upper face).  Regular D/N axes carry n+1 nodes, staggered and
    periodic axes n nodes.  Faces are evaluated on the node arrays of the two
    other axes: D faces hold psi, N faces hold d psi / d x_axis, both at the
    boundary plane itself (x = X_l or X_u).
    """
    coords = []
    for ax in range(3):
        nc = n_cells[ax]
        reg_nodes = (bc[ax] in ("D", "N", "DN", "ND")) and not staggered
        cnt = nc + 1 if reg_nodes else nc
        coords.append(node_positions(man.lo[ax], man.hi[ax], nc, staggered, cnt))
    xs, ys, zs = coords
    f = man.laplacian(xs, ys, zs)
    psi = man.field(xs, ys, zs)
    faces = {}
    for ax in range(3):
        if bc[ax] not in ("D", "N", "DN", "ND"):
            continue
        for side, xb in ((0, man.lo[ax]), (1, man.hi[ax])):
            kind = bc[ax][side] if len(bc[ax]) == 2 else bc[ax]
            pts = [xs, ys, zs]
            pts[ax] = np.array([xb])
            deriv = [0, 0, 0]
            if kind == "N":
                deriv[ax] = 1
            val = man.field(pts[0], pts[1], pts[2], tuple(deriv))
            faces[(ax, side)] = np.squeeze(val, axis=2 - ax)
    return {"f": f, "faces": faces, "psi_exact": psi, "coords": coords}


# --------------------------------------------------------------------------
# C3 / C5: compact vorticity for the unbounded solver
# --------------------------------------------------------------------------


def _unit_vector(rng: np.random.Generator) -> np.ndarray:
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def vortex_ring(n: int = 256, radius: float = 0.25, core: float = 0.05, seed_index: int = 2,
                lo: float = -0.5, hi: float = 0.5) -> Dict[str, object]:
    """Gaussian-core vortex ring, omega = exp(-rho^2/(2 s^2)) / (2 pi s^2) * t_hat.

    rho is the distance to the ring's centre line (a circle of the given radius
    about the origin whose axis is drawn uniformly on the sphere) and t_hat the
    circle's tangent.  Returns omega [3][n][n][n] on the staggered grid.
    """
    rng = rng_for(seed_index)
    axis = _unit_vector(rng)
    x = node_positions(lo, hi, n, True, n)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    P = np.stack([X, Y, Z], axis=0)  # [3][z][y][x] positions
    along = np.tensordot(axis, P, axes=(0, 0))  # component along the ring axis
    radial = P - axis[:, None, None, None] * along[None]
    rr = np.sqrt((radial ** 2).sum(axis=0))
    rho2 = (rr - radius) ** 2 + along ** 2
    amp = np.exp(-rho2 / (2 * core * core)) / (2 * math.pi * core * core)
    safe = np.where(rr > 1e-300, rr, 1.0)
    e_r = radial / safe[None]
    # tangent = axis x e_r
    t = np.stack([
        axis[1] * e_r[2] - axis[2] * e_r[1],
        axis[2] * e_r[0] - axis[0] * e_r[2],
        axis[0] * e_r[1] - axis[1] * e_r[0],
    ], axis=0)
    omega = amp[None] * t
    return {"omega": omega, "axis": axis, "h": (hi - lo) / n, "lo": lo, "hi": hi}


def gaussian_blobs(n: int = 128, count: int = 4, seed_index: int = 4, lo: float = -0.5,
                   hi: float = 0.5, vector: bool = True) -> Dict[str, object]:
    """Sum of Gaussian blobs with seeded centres, widths and (vector) amplitudes.

    Each blob is amp * exp(-|x-c|^2/(2 s^2)) / ((2 pi)^{3/2} s^3), widths s in
    [2h, 6h], centres in [-0.25, 0.25]^3, amplitudes in [-1, 1] (per component).
    Also returns a seeded loss weight w ~ U[0,1] of the same grid shape.
    """
    rng = rng_for(seed_index)
    h = (hi - lo) / n
    centres = rng.uniform(-0.25, 0.25, size=(count, 3))
    widths = rng.uniform(2 * h, 6 * h, size=count)
    amps = rng.uniform(-1.0, 1.0, size=(count, 3 if vector else 1))
    x = node_positions(lo, hi, n, True, n)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    ncomp = 3 if vector else 1
    field = np.zeros((ncomp, n, n, n))
    for b in range(count):
        r2 = (X - centres[b, 0]) ** 2 + (Y - centres[b, 1]) ** 2 + (Z - centres[b, 2]) ** 2
        s = widths[b]
        g = np.exp(-r2 / (2 * s * s)) / ((2 * math.pi) ** 1.5 * s ** 3)
        for c in range(ncomp):
            field[c] += amps[b, c] * g
    w = rng.uniform(0.0, 1.0, size=(n, n, n))
    return {"omega": field, "w": w, "centres": centres, "widths": widths, "amps": amps, "h": h,
            "lo": lo, "hi": hi}


def gaussian_blob_field(n: int, centre, width: float, lo: float = -0.5, hi: float = 0.5,
                        dim: int = 3) -> np.ndarray:
    """A single unit-mass Gaussian blob sampled on a staggered n^dim grid."""
    x = node_positions(lo, hi, n, True, n)
    if dim == 3:
        Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
        r2 = (X - centre[0]) ** 2 + (Y - centre[1]) ** 2 + (Z - centre[2]) ** 2
        return np.exp(-r2 / (2 * width ** 2)) / ((2 * math.pi) ** 1.5 * width ** 3)
    Y, X = np.meshgrid(x, x, indexing="ij")
    r2 = (X - centre[0]) ** 2 + (Y - centre[1]) ** 2
    return np.exp(-r2 / (2 * width ** 2)) / (2 * math.pi * width ** 2)


# --------------------------------------------------------------------------
# C4: a batch of uneven problems
# --------------------------------------------------------------------------

SIZES_2D = (64, 96, 128, 192, 256, 384, 512, 768, 1024)
SIZES_3D = (32, 48, 64, 96, 128)


@dataclasses.dataclass
class BatchProblem:
    dim: int
    n_cells: Tuple[int, ...]  # (nx, ny[, nz])
    bc: str  # one of 'P', 'D', 'N', 'U' (uniform over axes)
    staggered: bool
    seed: int

    def node_counts(self) -> Tuple[int, ...]:
        reg = (self.bc in ("D", "N")) and not self.staggered
        return tuple(n + 1 if reg else n for n in self.n_cells)

    def out_points(self) -> int:
        p = 1
        for n in self.n_cells:
            p *= n
        return p


def batch_problems(count: int = 512, seed_index: int = 3) -> List[BatchProblem]:
    rng = rng_for(seed_index)
    out = []
    for i in range(count):
        dim = 2 if rng.uniform() < 0.5 else 3
        sizes = SIZES_2D if dim == 2 else SIZES_3D
        n_cells = tuple(int(sizes[rng.integers(0, len(sizes))]) for _ in range(dim))
        bc = "PDNU"[rng.integers(0, 4)]
        if bc in ("P", "U"):
            staggered = True
        else:
            staggered = bool(rng.integers(0, 2))
        out.append(BatchProblem(dim, n_cells, bc, staggered, int(rng.integers(0, 2 ** 31 - 1))))
    return out


def lowpass_noise(shape: Tuple[int, ...], seed: int, cutoff: float = 0.25) -> np.ndarray:
    """N(0,1) noise with every Fourier mode above |k/n| > cutoff removed.

    The filter is applied with numpy's FFT as part of input synthesis only;
    shape is the array shape in [z][y][x] order (or [y][x]).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.standard_normal(size=shape)
    X = np.fft.rfftn(x)
    grids = []
    for ax, n in enumerate(shape):
        if ax == len(shape) - 1:
            k = np.arange(n // 2 + 1) / n
        else:
            k = np.fft.fftfreq(n)
        sh = [1] * len(shape)
        sh[ax] = -1
        grids.append((k ** 2).reshape(sh))
    k2 = sum(grids)
    X = np.where(k2 <= cutoff * cutoff, X, 0.0)
    return np.fft.irfftn(X, s=shape, axes=tuple(range(len(shape))))


def random_field(shape: Tuple[int, ...], seed: int) -> np.ndarray:
    return np.random.Generator(np.random.PCG64(seed)).standard_normal(size=shape)
