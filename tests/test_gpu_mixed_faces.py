"""GPU parity for axes with one Dirichlet and one Neumann face ('DN': Dirichlet
lower, Neumann upper; 'ND' the reverse), the quarter-wave sine / cosine
bases, against the FP64 oracle: PS and FD2 eigenvalues, regular and
staggered grids, inhomogeneous face data (FD2 lifting, one rule per face),
2D and 3D, the adjoint, and a batch.
"""
import itertools

import numpy as np
import pytest

import oracle
import workloads
from tests.gpu_helpers import TOL, gpu_plan, oracle_desc, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built(gpu_available):
    import __graft_entry__ as g
    g.build()


def solve_both(dim, n, bc, grid, eig, prec, faces=None, seed=0, hi=(1.0, 1.5, 0.75), rhs_scale=1.0, f=None):
    lo = (0.0,) * 3
    d = oracle_desc(dim, n, lo, hi, bc, grid, eig, rhs_scale=rhs_scale)
    if f is None:
        f = np.random.default_rng(seed).normal(size=(1,) + d.shape())
    plan = gpu_plan(dim, n, lo, hi, bc, grid, eig, prec=prec, rhs_scale=rhs_scale)
    if faces:
        for (ax, side), g in faces.items():
            plan.set_boundary(ax, side, to_dev(g, prec))
    psi, _ = plan.empty_outputs()
    plan.execute(to_dev(f, prec), psi)
    plan.sync()
    ref, _ = oracle.solve(d, f, faces)
    plan.close()
    return to_np(psi)[0], ref[0]


MIXED3 = [("DN", "D", "N"), ("ND", "N", "D"), ("DN", "ND", "D"), ("N", "DN", "ND"), ("DN", "DN", "DN"),
          ("ND", "ND", "ND")]


@pytest.mark.parametrize("bc", MIXED3, ids=lambda b: "-".join(b))
@pytest.mark.parametrize("grid", ["regular", "staggered"])
def test_mixed_faces_3d_fp64_ps(bc, grid):
    got, ref = solve_both(3, (12, 8, 6), bc, grid, "PS", "f64")
    assert rel_l2(got, ref) <= TOL["f64"]


@pytest.mark.parametrize("bc", MIXED3, ids=lambda b: "-".join(b))
@pytest.mark.parametrize("grid", ["regular", "staggered"])
def test_mixed_faces_3d_fp32_fd2_inhomogeneous(bc, grid):
    n = (16, 12, 24)
    man = workloads.manufactured(seed_index=13)
    case = workloads.bounded_case(man, n, bc, grid == "staggered")
    got, ref = solve_both(3, n, bc, grid, "FD2", "f32", faces=case["faces"], hi=(1.0, 1.0, 1.0), f=case["f"][None])
    assert rel_l2(got, ref) <= TOL["f32"]


@pytest.mark.parametrize("bc", [("DN", "ND"), ("ND", "P"), ("DN", "D"), ("N", "ND")], ids=lambda b: "-".join(b))
@pytest.mark.parametrize("grid", ["regular", "staggered"])
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_mixed_faces_2d(bc, grid, prec):
    if "P" in bc:
        pytest.skip("periodic axes do not mix with Dirichlet / Neumann axes")
    got, ref = solve_both(2, (48, 24), bc, grid, "FD2", prec, seed=2)
    assert rel_l2(got, ref) <= TOL[prec]


@pytest.mark.parametrize("bc,grid", [(("DN", "N", "ND"), "regular"), (("ND", "DN"), "staggered")],
                         ids=["3D-regular", "2D-staggered"])
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_mixed_faces_adjoint_vs_oracle(bc, grid, prec):
    import paper_2301_01145_gb300 as sf
    dim = len(bc)
    n = (12, 8, 16)[:dim]
    lo, hi = (0.0,) * dim, (1.0, 1.5, 0.75)[:dim]
    eig = "FD2" if grid == "regular" else "PS"
    d = oracle_desc(dim, n, lo, hi, bc, grid, eig, rhs_scale=0.5)
    g = np.random.default_rng(7).normal(size=(1,) + d.shape())
    ref = oracle.adjoint_solve(d, g, None)
    plan = gpu_plan(dim, n, lo, hi, bc, grid, eig, prec=prec, rhs_scale=0.5)
    gf = plan.adjoint(to_dev(g, prec))
    plan.sync()
    assert rel_l2(to_np(gf)[0], ref[0]) <= TOL[prec]
    plan.close()


def test_mixed_faces_in_a_batch():
    import torch
    import paper_2301_01145_gb300 as sf
    probs = [dict(dim=3, n=(8, 12, 6), bc=("DN", "D", "ND"), grid="regular"),
             dict(dim=2, n=(32, 24), bc=("ND", "DN"), grid="staggered"),
             dict(dim=3, n=(6, 8, 12), bc=("N", "DN", "D"), grid="staggered")]
    plans, fs, psis, refs = [], [], [], []
    for i, p in enumerate(probs):
        dim = p["dim"]
        lo, hi = (0.0,) * dim, (1.0,) * dim
        plan = sf.Plan(dim, p["n"], lo, hi, list(p["bc"]), grid=p["grid"], eig="PS", generic=True)
        d = oracle_desc(dim, p["n"], lo, hi, p["bc"], p["grid"], "PS")
        f = np.random.default_rng(30 + i).normal(size=(1,) + d.shape())
        plans.append(plan)
        fs.append(to_dev(f, "f32"))
        psis.append(torch.empty(plan.out_shape, dtype=torch.float32, device="cuda"))
        refs.append(oracle.solve(d, f)[0])
    batch = sf.Batch(plans)
    batch.solve(fs, psis)
    batch.sync()
    for i, plan in enumerate(plans):
        single = plan(fs[i])
        plan.sync()
        assert torch.equal(single, psis[i])
        assert rel_l2(to_np(psis[i])[0], refs[i][0]) <= TOL["f32"]
    batch.close()
    for p in plans:
        p.close()
