"""Edge cases of the CUDA path against the FP64 oracle: the smallest grids each
boundary type admits (including a single unknown per axis), the largest FFT
length of the general engine (L = 2048, 2D), ragged non-power-of-two shapes
(3 * 2^p lengths, unequal axes), zero sources, and solve-without-source state
errors.  Tolerances as in the parity tests (relative L2 per field).
"""
import numpy as np
import pytest

import oracle
from tests.gpu_helpers import TOL, gpu_plan, oracle_desc, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built(gpu_available):
    import __graft_entry__ as g
    g.build()


def check(dim, n, bc, grid, prec, eig="PS", op="NONE", ncomp=1, sigma=0.0, rhs_scale=1.0, seed=3, lo=None, hi=None):
    lo = lo or (0.0,) * 3
    hi = hi or (1.0, 1.5, 0.75)
    d = oracle_desc(dim, n, lo, hi, bc, grid, eig, op, sigma, ncomp, rhs_scale)
    f = np.random.default_rng(seed).normal(size=(ncomp,) + d.shape())
    plan = gpu_plan(dim, n, lo, hi, bc, grid, eig, op, sigma, ncomp, prec, rhs_scale)
    psi, opo = plan.empty_outputs()
    plan.execute(to_dev(f, prec), psi, opo)
    plan.sync()
    ref_psi, ref_op = oracle.solve(d, f)
    pairs = [(to_np(psi), ref_psi)] + ([(to_np(opo), ref_op)] if opo is not None else [])
    for got, ref in pairs:
        for c in range(ref.shape[0]):
            assert rel_l2(got[c], ref[c]) <= TOL[prec], (n, bc, grid, c)
    plan.close()


# smallest admitted grids: FFT length >= 4 (periodic n >= 4, even in x), regular
# Dirichlet n >= 3 (one or two unknowns per axis), all others n >= 2
MINIMAL = [
    (3, (4, 4, 4), "PPP", "staggered"),
    (3, (3, 3, 3), "DDD", "regular"),
    (3, (2, 2, 2), "DDD", "staggered"),
    (3, (2, 2, 2), "NNN", "regular"),
    (3, (2, 2, 2), "NNN", "staggered"),
    (3, (2, 2, 2), "UUU", "staggered"),
    (2, (4, 6), "PP", "staggered"),
    (2, (3, 2), "DN", "regular"),
    (2, (2, 3), "UU", "staggered"),
]


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("dim,n,bc,grid", MINIMAL, ids=lambda v: str(v))
def test_minimal_grids(dim, n, bc, grid, prec):
    sigma = 2.0 / max(n) if bc[0] == "U" else 0.0
    check(dim, n, bc, grid, prec, sigma=sigma, rhs_scale=-1.0 if bc[0] == "U" else 1.0)


# the largest FFT length of the general engine is 2048 (periodic n = 2048;
# doubled axes n = 1024), on thin 2D grids the oracle finishes in seconds
MAXIMAL = [
    (2, (2048, 4), "PP", "staggered"),
    (2, (4, 2048), "PP", "staggered"),
    (2, (1024, 3), "UU", "staggered"),
    (2, (1024, 4), "DD", "regular"),
    (2, (6, 1024), "NN", "staggered"),
]


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("dim,n,bc,grid", MAXIMAL, ids=lambda v: str(v))
def test_maximal_fft_length(dim, n, bc, grid, prec):
    sigma = 2.0 / max(n) if bc[0] == "U" else 0.0
    check(dim, n, bc, grid, prec, sigma=sigma, rhs_scale=-1.0 if bc[0] == "U" else 1.0)


# ragged shapes: 3 * 2^p FFT lengths on unequal axes, odd unknown counts
RAGGED = [
    (3, (6, 12, 24), "PPP", "staggered", "FD2"),
    (3, (3, 6, 12), "DND", "regular", "PS"),
    (3, (3, 12, 6), "NDN", "regular", "FD2"),
    (3, (6, 3, 12), "UUU", "staggered", "PS"),
    (3, (24, 6, 3), "DDD", "staggered", "PS"),
]


@pytest.mark.parametrize("dim,n,bc,grid,eig", RAGGED, ids=lambda v: str(v))
def test_ragged_shapes(dim, n, bc, grid, eig):
    sigma = 2.0 / max(n) if bc[0] == "U" else 0.0
    check(dim, n, bc, grid, "f32", eig=eig, sigma=sigma, rhs_scale=-1.0 if bc[0] == "U" else 1.0)


@pytest.mark.parametrize("bc,grid,op,ncomp", [("PPP", "staggered", "CURL", 3), ("UUU", "staggered", "CURL", 3),
                                               ("DDD", "regular", "NONE", 1), ("NNN", "staggered", "NONE", 2)])
def test_zero_source_gives_zero(bc, grid, op, ncomp):
    # the map is linear: a zero source (no boundary data) gives exactly zero everywhere
    import torch
    n = (16, 12, 8)
    sigma = 0.125 if bc[0] == "U" else 0.0
    plan = gpu_plan(3, n, (0,) * 3, (1,) * 3, bc, grid, op=op, ncomp=ncomp, sigma=sigma)
    psi, opo = plan.empty_outputs()
    psi.fill_(float("nan"))
    if opo is not None:
        opo.fill_(float("nan"))
    plan.execute(torch.zeros(plan.in_shape, device="cuda"), psi, opo)
    plan.sync()
    assert torch.count_nonzero(psi).item() == 0
    if opo is not None:
        assert torch.count_nonzero(opo).item() == 0
    plan.close()


def test_get_output_before_solve_is_a_state_error():
    import paper_2301_01145_gb300 as sf
    plan = gpu_plan(3, (8, 8, 8), (0,) * 3, (1,) * 3, "PPP")
    psi, _ = plan.empty_outputs()
    with pytest.raises(sf.SolverError):
        plan.get_output(psi)
    plan.close()


# operators on Dirichlet / Neumann axes at the smallest grids: one or two
# unknowns per axis, regular Dirichlet faces (lines of zeros in every term),
# the quarter-wave pairs, both precisions
MINIMAL_OPS = [
    (3, (3, 3, 3), ("D", "D", "D"), "regular", "GRAD", 1),
    (3, (2, 3, 2), ("N", "D", "DN"), "regular", "CURL", 3),
    (3, (2, 2, 2), ("ND", "N", "D"), "staggered", "DIV", 3),
    (2, (3, 2), ("D", "N"), "regular", "CURL", 1),
    (2, (2, 2), ("DN", "ND"), "staggered", "GRAD", 1),
    (2, (2, 3), ("N", "D"), "regular", "DIV", 2),
    (1, (3,), ("D",), "regular", "GRAD", 1),
    (1, (2,), ("ND",), "staggered", "GRAD", 1),
]


@pytest.mark.parametrize("case", MINIMAL_OPS, ids=lambda c: f"{c[0]}D-{'-'.join(c[2])}-{c[3]}-{c[4]}")
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_minimal_grids_with_operators(case, prec):
    dim, n, bc, grid, op, ncomp = case
    check(dim, n, bc, grid, prec, op=op, ncomp=ncomp)


@pytest.mark.parametrize("bc,grid,op,ncomp", [(("D", "N", "DN"), "regular", "CURL", 3),
                                               (("N", "D", "N"), "staggered", "GRAD", 1),
                                               (("DN", "D", "N"), "regular", "DIV", 3)])
def test_bounded_operator_writes_every_output_node(bc, grid, op, ncomp):
    # outputs filled with NaN first: every node of every operator output is
    # written (the derivative terms cover face lines and face nodes with zeros)
    import torch
    n = (12, 16, 8)
    plan = gpu_plan(3, n, (0,) * 3, (1,) * 3, bc, grid, op=op, ncomp=ncomp)
    psi, opo = plan.empty_outputs()
    psi.fill_(float("nan"))
    opo.fill_(float("nan"))
    f = to_dev(np.random.default_rng(4).normal(size=plan.in_shape), "f32")
    plan.execute(f, psi, opo)
    plan.sync()
    assert not torch.isnan(psi).any() and not torch.isnan(opo).any()
    d = oracle_desc(3, n, (0,) * 3, (1,) * 3, bc, grid, "PS", op, 0.0, ncomp, 1.0)
    ref_psi, ref_op = oracle.solve(d, to_np(f))
    for o in range(ref_op.shape[0]):
        assert rel_l2(to_np(opo)[o], ref_op[o]) <= TOL["f32"], o
    plan.close()
