"""GPU parity of the spectral operators on Dirichlet / Neumann axes (GRAD, DIV,
CURL, NABLA as derivatives of the basis series, sine <-> cosine) against the
FP64 oracle: 1D, 2D and 3D, regular and staggered grids, every face kind
including the quarter-wave pairs, PS and FD2 (with inhomogeneous faces), FP32
and FP64, the fused and unfused executors, a batch, and the refused adjoint.
"""
import numpy as np
import pytest

import oracle
import workloads
from oracle.desc import Desc
from tests.gpu_helpers import TOL, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built(gpu_available):
    import __graft_entry__ as g
    g.build()


def make(dim, n, bc, grid, eig, op, ncomp, prec, fused=True, rhs_scale=0.9):
    import paper_2301_01145_gb300 as sf
    lo, hi = (0.0,) * dim, (1.0, 1.4, 0.8)[:dim]
    plan = sf.Plan(dim, n, lo, hi, list(bc), grid=grid, eig=eig, op=op, ncomp=ncomp, prec=prec, fused=fused,
                   rhs_scale=rhs_scale)
    d = Desc(dim, tuple(n), lo, hi, tuple(bc), grid == "staggered", eig, op, ncomp, rhs_scale, 0.0)
    return plan, d


# First derivatives on Dirichlet / Neumann axes are formed where their axis is
# still spectral (x from the x-spectral field, the stage axis in the spectral
# stage, 3D y in the y-inverse term pass), so their rounding scales with the
# derivative itself and every output is held to the stated tolerance.
def op_tol(d, prec):
    return TOL[prec]


def check(plan, d, f, prec, faces=None):
    psi, opo = plan.empty_outputs()
    if faces:
        for (ax, side), g in faces.items():
            plan.set_boundary(ax, side, to_dev(g, prec))
    plan.execute(to_dev(f, prec), psi, opo)
    plan.sync()
    rp, ro = oracle.solve(d, f, faces)
    for c in range(rp.shape[0]):
        assert rel_l2(to_np(psi)[c], rp[c]) <= TOL[prec]
    for o in range(ro.shape[0]):
        assert rel_l2(to_np(opo)[o], ro[o]) <= op_tol(d, prec), o


OPS3 = [("GRAD", 1), ("DIV", 3), ("CURL", 3), ("NABLA", 2)]
BCS3 = [("D", "N", "DN"), ("ND", "D", "N"), ("N", "DN", "ND")]


@pytest.mark.parametrize("op,ncomp", OPS3, ids=[o for o, _ in OPS3])
@pytest.mark.parametrize("bc", BCS3, ids=lambda b: "-".join(b))
@pytest.mark.parametrize("grid", ["regular", "staggered"])
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_ops_3d(op, ncomp, bc, grid, prec):
    n = (12, 16, 8)
    plan, d = make(3, n, bc, grid, "PS", op, ncomp, prec)
    f = np.random.default_rng(11).normal(size=(ncomp,) + d.shape())
    check(plan, d, f, prec)
    plan.close()


@pytest.mark.parametrize("op,ncomp", [("GRAD", 1), ("DIV", 2), ("CURL", 1), ("NABLA", 1)])
@pytest.mark.parametrize("bc", [("D", "N"), ("DN", "ND"), ("N", "N"), ("D", "D")], ids=lambda b: "-".join(b))
@pytest.mark.parametrize("grid", ["regular", "staggered"])
@pytest.mark.parametrize("eig", ["PS", "FD2"])
def test_ops_2d(op, ncomp, bc, grid, eig):
    n = (48, 24)
    plan, d = make(2, n, bc, grid, eig, op, ncomp, "f32")
    f = np.random.default_rng(5).normal(size=(ncomp,) + d.shape())
    check(plan, d, f, "f32")
    plan.close()


@pytest.mark.parametrize("op", ["GRAD", "NABLA"])
@pytest.mark.parametrize("bc", ["D", "N", "DN", "ND"])
@pytest.mark.parametrize("grid", ["regular", "staggered"])
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_ops_1d(op, bc, grid, prec):
    plan, d = make(1, (96,), (bc,), grid, "PS", op, 1, prec)
    f = np.random.default_rng(6).normal(size=(1,) + d.shape())
    check(plan, d, f, prec)
    plan.close()


@pytest.mark.parametrize("bc", [("D", "DN", "D"), ("DN", "D", "ND")], ids=lambda b: "-".join(b))
@pytest.mark.parametrize("grid", ["regular", "staggered"])
@pytest.mark.parametrize("fused", [True, False])
def test_grad_fd2_inhomogeneous_faces(bc, grid, fused):
    import paper_2301_01145_gb300 as sf
    n = (16, 12, 24)
    man = workloads.manufactured(seed_index=17)
    case = workloads.bounded_case(man, n, bc, grid == "staggered")
    plan = sf.Plan(3, n, (0.0,) * 3, (1.0,) * 3, list(bc), grid=grid, eig="FD2", op="GRAD", fused=fused)
    d = Desc(3, n, (0.0,) * 3, (1.0,) * 3, bc, grid == "staggered", "FD2", "GRAD", 1, 1.0, 0.0)
    check(plan, d, case["f"][None], "f32", case["faces"])
    plan.close()


def test_larger_2d_grad():
    plan, d = make(2, (512, 384), ("N", "D"), "staggered", "PS", "GRAD", 1, "f32")
    f = np.random.default_rng(7).normal(size=(1,) + d.shape())
    check(plan, d, f, "f32")
    plan.close()


def test_bounded_op_plans_in_a_batch():
    import torch
    import paper_2301_01145_gb300 as sf
    plans, ds, fs, outs = [], [], [], []
    for i, (dim, n, bc, op, nc) in enumerate([(3, (8, 12, 6), ("D", "N", "D"), "CURL", 3),
                                              (2, (24, 16), ("DN", "N"), "GRAD", 1),
                                              (1, (48,), ("ND",), "NABLA", 1),
                                              (2, (16, 16), ("P", "P"), "GRAD", 1)]):
        plan, d = make(dim, n, bc, "regular" if i % 2 == 0 else "staggered", "PS", op, nc, "f32")
        if bc == ("P", "P"):
            plan.close()
            plan, d = make(dim, n, bc, "staggered", "PS", op, nc, "f32")
        f = np.random.default_rng(20 + i).normal(size=(nc,) + d.shape())
        plans.append(plan)
        ds.append(d)
        fs.append(to_dev(f, "f32"))
        outs.append(plan.empty_outputs())
    batch = sf.Batch(plans)
    batch.solve(fs, [o[0] for o in outs], [o[1] for o in outs])
    batch.sync()
    for i, plan in enumerate(plans):
        psi, opo = plan(fs[i])
        plan.sync()
        assert torch.equal(psi, outs[i][0]) and torch.equal(opo, outs[i][1])
        rp, ro = oracle.solve(ds[i], to_np(fs[i]))
        for o in range(ro.shape[0]):
            assert rel_l2(to_np(opo)[o], ro[o]) <= op_tol(ds[i], "f32")
    batch.close()
    for p in plans:
        p.close()


ADJ = [(3, (8, 12, 6), ("D", "N", "DN"), "regular", "FD2", "GRAD", 1),
       (3, (6, 8, 12), ("ND", "D", "N"), "staggered", "PS", "CURL", 3),
       (3, (8, 6, 8), ("N", "DN", "D"), "regular", "PS", "DIV", 3),
       (2, (24, 16), ("DN", "ND"), "staggered", "PS", "CURL", 1),
       (2, (16, 12), ("D", "N"), "regular", "FD2", "NABLA", 2),
       (1, (48,), ("ND",), "regular", "PS", "GRAD", 1),
       (1, (48,), ("D",), "staggered", "PS", "NABLA", 1)]


@pytest.mark.parametrize("dim,n,bc,grid,eig,op,ncomp", ADJ, ids=[f"{a[0]}D-{'-'.join(a[2])}-{a[5]}" for a in ADJ])
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_adjoint_with_bounded_operator_vs_oracle(dim, n, bc, grid, eig, op, ncomp, prec):
    plan, d = make(dim, n, bc, grid, eig, op, ncomp, prec)
    rng = np.random.default_rng(13)
    g = rng.normal(size=(ncomp,) + d.shape())
    go = rng.normal(size=(d.op_components(),) + d.shape())
    ref = oracle.adjoint_solve(d, g, go)
    gf = plan.adjoint(to_dev(g, prec), to_dev(go, prec))
    plan.sync()
    for c in range(ncomp):
        assert rel_l2(to_np(gf)[c], ref[c]) <= TOL[prec], c
    # the psi gradient alone, and the operator gradient alone
    ref_o = oracle.adjoint_solve(d, None, go)
    gf = plan.adjoint(None, to_dev(go, prec))
    plan.sync()
    assert rel_l2(to_np(gf)[0], ref_o[0]) <= TOL[prec]
    plan.close()


def test_autograd_through_a_bounded_gradient():
    import torch
    from paper_2301_01145_gb300.autograd import poisson_solve
    plan, d = make(2, (24, 16), ("D", "N"), "staggered", "PS", "GRAD", 1, "f64")
    rng = np.random.default_rng(3)
    f0 = rng.normal(size=(1,) + d.shape())
    w = torch.tensor(rng.normal(size=(2,) + d.shape()), device="cuda")
    f = torch.tensor(f0, device="cuda", requires_grad=True)
    psi, grad = poisson_solve(f, plan)
    loss = (w * grad).sum() + (psi * psi).sum()
    loss.backward()
    # the same derivative from the oracle: d loss / d f = A_psi^T (2 psi) + A_op^T w
    rp, _ = oracle.solve(d, f0)
    ref = oracle.adjoint_solve(d, 2 * rp, w.cpu().numpy())
    assert rel_l2(to_np(f.grad)[0], ref[0]) <= TOL["f64"]
    plan.close()
