"""GPU parity of the 1D solves (Sec. 2.4: the 1D solver classes) against the FP64
oracle: periodic with operators, Dirichlet / Neumann / mixed faces on both
grids with PS and FD2 (inhomogeneous faces for FD2), unbounded with the 1D
spectral kernel on both grids, the adjoint, and 1D plans inside a batch.
Sizes run from the smallest valid axis to the largest FFT length (2048).
"""
import numpy as np
import pytest

import oracle
from oracle.desc import Desc
from tests.gpu_helpers import TOL, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built(gpu_available):
    import __graft_entry__ as g
    g.build()


def both(n, bc, grid="staggered", eig="PS", op="NONE", ncomp=1, prec="f32", rhs_scale=0.8, kernel="G2",
         lo=-0.4, hi=1.1):
    import paper_2301_01145_gb300 as sf
    plan = sf.Plan(1, (n,), (lo,), (hi,), [bc], grid=grid, eig=eig, op=op, ncomp=ncomp, prec=prec,
                   rhs_scale=rhs_scale, kernel=kernel)
    d = Desc(1, (n,), (lo,), (hi,), (bc,), grid == "staggered", eig, op, ncomp, rhs_scale, 0.0, kernel=kernel)
    return plan, d


def run(plan, d, f, prec, faces=None):
    psi, opo = plan.empty_outputs()
    if faces:
        for (ax, side), g in faces.items():
            plan.set_boundary(ax, side, to_dev(np.atleast_1d(g), prec))
    plan.execute(to_dev(f, prec), psi, opo)
    plan.sync()
    ref_psi, ref_op = oracle.solve(d, f, faces)
    return to_np(psi), (to_np(opo) if opo is not None else None), ref_psi, ref_op


@pytest.mark.parametrize("n", [4, 24, 96, 2048])
@pytest.mark.parametrize("op,ncomp", [("NONE", 3), ("GRAD", 1), ("DIV", 1), ("NABLA", 2)])
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_periodic_1d(n, op, ncomp, prec):
    plan, d = both(n, "P", op=op, ncomp=ncomp, prec=prec)
    f = np.random.default_rng(n).normal(size=(ncomp,) + d.shape())
    psi, opo, rp, ro = run(plan, d, f, prec)
    for c in range(ncomp):
        assert rel_l2(psi[c], rp[c]) <= TOL[prec]
    if ro is not None:
        for o in range(ro.shape[0]):
            assert rel_l2(opo[o], ro[o]) <= TOL[prec]
    plan.close()


@pytest.mark.parametrize("n", [3, 24, 1024])
@pytest.mark.parametrize("bc", ["D", "N", "DN", "ND"])
@pytest.mark.parametrize("grid", ["regular", "staggered"])
@pytest.mark.parametrize("eig", ["PS", "FD2"])
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_bounded_1d(n, bc, grid, eig, prec):
    if len(bc) == 2 and n == 1024:
        n = 512  # 4 n <= 2048
    if n == 3 and (len(bc) == 2 or grid == "staggered" or bc == "N"):
        n = 4  # FFT lengths 2^p or 3 * 2^p
    plan, d = both(n, bc, grid, eig, prec=prec)
    f = np.random.default_rng(7 * n).normal(size=(2,) + d.shape())[:1]
    psi, _, rp, _ = run(plan, d, f, prec)
    assert rel_l2(psi[0], rp[0]) <= TOL[prec]
    plan.close()


@pytest.mark.parametrize("bc", ["D", "DN", "ND"])
@pytest.mark.parametrize("grid", ["regular", "staggered"])
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_bounded_1d_inhomogeneous_faces(bc, grid, prec):
    n = 48
    plan, d = both(n, bc, grid, "FD2", prec=prec)
    f = np.random.default_rng(3).normal(size=(1,) + d.shape())
    faces = {(0, 0): np.array(0.35), (0, 1): np.array(-0.8)}
    psi, _, rp, _ = run(plan, d, f, prec, faces)
    assert rel_l2(psi[0], rp[0]) <= TOL[prec]
    plan.close()


@pytest.mark.parametrize("n", [8, 96, 1024])
@pytest.mark.parametrize("grid", ["staggered", "regular"])
@pytest.mark.parametrize("op", ["NONE", "GRAD", "NABLA"])
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_unbounded_1d_spectral(n, grid, op, prec):
    if grid == "regular" and n == 1024:
        n = 1023  # pad 2 n + 1 <= 2048
    plan, d = both(n, "U", grid, op=op, prec=prec, kernel="SPECT")
    f = np.random.default_rng(n + 1).normal(size=(1,) + d.shape())
    psi, opo, rp, ro = run(plan, d, f, prec)
    # The 1D kernel grows like |x|/2, so its transform spans
    # |G^(0)| / |G^(k_max)| ~ (L / pi)^2 (4e5 at L = 2048); both sides' table
    # transforms round relative to G^(0) and the operators weight the high modes
    # by kappa or kappa^2.  In FP64 that bounds the agreement by
    # eps * (L / pi)^2 ~ 1e-10 rather than the 1e-12 of the decaying 3D kernels.
    tol = 1e-10 if prec == "f64" else TOL[prec]
    assert rel_l2(psi[0], rp[0]) <= tol
    if ro is not None:
        assert rel_l2(opo[0], ro[0]) <= tol
    plan.close()


@pytest.mark.parametrize("bc,grid,eig,op,kernel", [("P", "staggered", "PS", "GRAD", "G2"),
                                                   ("D", "regular", "FD2", "NONE", "G2"),
                                                   ("ND", "staggered", "PS", "NONE", "G2"),
                                                   ("U", "staggered", "PS", "NABLA", "SPECT"),
                                                   ("U", "regular", "PS", "GRAD", "SPECT")])
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_adjoint_1d_vs_oracle(bc, grid, eig, op, kernel, prec):
    n = 48
    plan, d = both(n, bc, grid, eig, op=op, prec=prec, kernel=kernel)
    rng = np.random.default_rng(9)
    g = rng.normal(size=(1,) + d.shape())
    go = rng.normal(size=(1,) + d.shape()) if op != "NONE" else None
    ref = oracle.adjoint_solve(d, g, go)
    gf = plan.adjoint(to_dev(g, prec), to_dev(go, prec) if go is not None else None)
    plan.sync()
    tol = 1e-10 if (prec == "f64" and bc == "U") else TOL[prec]  # the 1D kernel's range, as above
    assert rel_l2(to_np(gf)[0], ref[0]) <= tol
    plan.close()


def test_1d_plans_in_a_batch():
    import torch
    import paper_2301_01145_gb300 as sf
    specs = [dict(n=64, bc="P"), dict(n=96, bc="D", grid="regular", eig="FD2"), dict(n=96, bc="U", kernel="SPECT"),
             dict(n=48, bc="DN")]
    plans, ds, fs, psis = [], [], [], []
    for i, s in enumerate(specs):
        plan, d = both(s["n"], s["bc"], s.get("grid", "staggered"), s.get("eig", "PS"), kernel=s.get("kernel", "G2"))
        f = np.random.default_rng(40 + i).normal(size=(1,) + d.shape())
        plans.append(plan)
        ds.append(d)
        fs.append(to_dev(f, "f32"))
        psis.append(torch.empty(plan.out_shape, dtype=torch.float32, device="cuda"))
    # a 2D problem in the same batch
    p2 = sf.Plan(2, (32, 24), (0, 0), (1, 1), "PP")
    d2 = Desc(2, (32, 24), (0, 0), (1, 1), ("P", "P"), True)
    plans.append(p2)
    ds.append(d2)
    fs.append(to_dev(np.random.default_rng(50).normal(size=(1,) + d2.shape()), "f32"))
    psis.append(torch.empty(p2.out_shape, dtype=torch.float32, device="cuda"))
    batch = sf.Batch(plans)
    batch.solve(fs, psis)
    batch.sync()
    for i, plan in enumerate(plans):
        single = plan(fs[i])
        plan.sync()
        assert torch.equal(single, psis[i])
        ref, _ = oracle.solve(ds[i], to_np(fs[i]))
        assert rel_l2(to_np(psis[i])[0], ref[0]) <= TOL["f32"]
    batch.close()
    for p in plans:
        p.close()
