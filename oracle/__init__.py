"""Plain, slow FP64 CPU oracle for the fast Poisson solver (test infrastructure).

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and
the benchmark's CPU-baseline / reference leg may import it.  The CUDA library
and its Python binding never import, call or link anything in here, and this
package imports nothing from them: the two share no code.

What it computes (SailFFish, Sec. 2): the four-step spectral solve of
lap(psi) = rhs_scale * f -- forward transform, point-wise multiply by the
eigenvalues (Table 1) or by the transformed Green's function (Sec. 2.6),
optional spectral operator (Sec. 2.4.3, Eq. ft_sd), inverse transform -- for
periodic (DFT), Dirichlet (DST) and Neumann (DCT) axes on regular or staggered
grids (Eq. gridpos) and for unbounded domains by Hockney-Eastwood doubling.

Everything is written for clarity rather than speed:
  * fft.py       -- own recursive radix-2 FFT, direct DFT for odd lengths
  * r2r.py       -- DST-I/II/III and DCT-I/II/III as direct O(n^2) sums
  * eigen.py     -- the PS and FD2 eigenvalues of Table 1
  * bounded.py   -- bounded solve incl. FD2 boundary lifting (Sec. 2.5.2)
  * green.py     -- Gaussian-regularised Green's functions (Sec. 2.6.2)
  * unbounded.py -- Hockney-Eastwood solve with spectral operators
  * semi.py      -- one unbounded axis with periodic axes (doubling of that axis only)
  * adjoint.py   -- the transpose of the solve (for gradients)

Every function is pinned by tests in tests/test_oracle_*.py against closed
forms, brute force or library routines; see each module's header.
"""
from .desc import Desc  # noqa: F401
from .bounded import solve_bounded  # noqa: F401
from .unbounded import solve_unbounded, green_hat  # noqa: F401
from .semi import solve_semi, is_semi  # noqa: F401
from .adjoint import adjoint_solve  # noqa: F401


def solve(desc, f, faces=None):
    """Dispatch on boundary type: all-unbounded -> Hockney-Eastwood, one unbounded
    axis with periodic axes -> semi-unbounded, else bounded."""
    if all(b == "U" for b in desc.bc[: desc.dim]):
        return solve_unbounded(desc, f)
    if is_semi(desc):
        return solve_semi(desc, f)
    return solve_bounded(desc, f, faces)
