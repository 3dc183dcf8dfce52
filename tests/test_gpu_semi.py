"""Semi-unbounded solves on the GPU (one unbounded axis, the others periodic) against the oracle.

Every case compares each output field with oracle.solve (semi.py) at relative
L2 1e-5 (FP32) and 1e-12 (FP64): both grids, PS and FD2 periodic eigenvalues,
the unbounded axis in every position, the operators, the adjoint against the
oracle's transpose, and a batch that mixes semi-unbounded plans with others.
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


def make(dim, n, bc, grid="staggered", eig="PS", op="NONE", ncomp=1, prec="f32", rhs_scale=-1.0):
    import paper_2301_01145_gb300 as sf
    lo, hi = (-0.5,) * dim, (0.5, 0.75, 0.6)[:dim]
    plan = sf.Plan(dim, n, lo, hi, list(bc), grid=grid, eig=eig, op=op, ncomp=ncomp, prec=prec, rhs_scale=rhs_scale)
    d = Desc(dim, tuple(n), lo, hi, tuple(bc), grid == "staggered", eig, op, ncomp, rhs_scale)
    return plan, d


CASES = [
    (2, (64, 48), "PU", "staggered", "PS", "NONE", 1),
    (2, (48, 32), "UP", "regular", "FD2", "GRAD", 1),
    (2, (32, 64), "PU", "regular", "PS", "CURL", 1),
    (3, (32, 24, 16), "PPU", "staggered", "PS", "CURL", 3),
    (3, (16, 32, 24), "UPP", "regular", "FD2", "GRAD", 1),
    (3, (24, 16, 32), "PUP", "staggered", "PS", "DIV", 3),
    (3, (32, 16, 16), "PPU", "staggered", "PS", "NABLA", 2),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}D-{c[2]}-{c[3]}-{c[4]}-{c[5]}")
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_semi_vs_oracle(case, prec):
    dim, n, bc, grid, eig, op, ncomp = case
    plan, d = make(dim, n, bc, grid, eig, op, ncomp, prec)
    f = np.random.default_rng(sum(n)).normal(size=(ncomp,) + d.shape())
    out = plan(to_dev(f, prec))
    plan.sync()
    psi, opo = out if isinstance(out, tuple) else (out, None)
    rp, ro = oracle.solve(d, f)
    for c in range(ncomp):
        assert rel_l2(to_np(psi)[c], rp[c]) <= TOL[prec], ("psi", c)
    if opo is not None:
        for c in range(ro.shape[0]):
            assert rel_l2(to_np(opo)[c], ro[c]) <= TOL[prec], ("op", c)
    plan.close()


@pytest.mark.parametrize("case", [CASES[1], CASES[3]], ids=lambda c: f"{c[0]}D-{c[2]}-{c[5]}")
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_semi_adjoint_vs_oracle(case, prec):
    dim, n, bc, grid, eig, op, ncomp = case
    plan, d = make(dim, n, bc, grid, eig, op, ncomp, prec)
    rng = np.random.default_rng(7)
    gp = rng.normal(size=(ncomp,) + d.shape())
    go = rng.normal(size=(d.op_components(),) + d.shape())
    ref = oracle.adjoint_solve(d, gp, go)
    gf = plan.adjoint(to_dev(gp, prec), to_dev(go, prec))
    plan.sync()
    for c in range(ncomp):
        assert rel_l2(to_np(gf)[c], ref[c]) <= TOL[prec]
    plan.close()


def test_semi_refusals():
    import paper_2301_01145_gb300 as sf
    from paper_2301_01145_gb300 import SolverError
    for bc in ("UUP", "UD", "PUD"):
        dim = len(bc)
        with pytest.raises(SolverError) as e:
            sf.Plan(dim, (16,) * dim, (0.0,) * dim, (1.0,) * dim, list(bc))
        assert e.value.status == -2


def test_semi_plans_in_a_batch():
    import torch
    import paper_2301_01145_gb300 as sf
    specs = [(2, (64, 32), "PU"), (3, (16, 16, 32), "PPU"), (2, (32, 32), "UU"), (2, (64, 64), "PP")]
    plans, ds, fs, psis = [], [], [], []
    for i, (dim, n, bc) in enumerate(specs):
        kw = dict(sigma=2.0 / max(n)) if bc == "U" * dim else {}
        plan = sf.Plan(dim, n, (-0.5,) * dim, (0.5,) * dim, list(bc), rhs_scale=-1.0, generic=True, **kw)
        d = Desc(dim, n, (-0.5,) * dim, (0.5,) * dim, tuple(bc), True, rhs_scale=-1.0, **kw)
        f = np.random.default_rng(50 + i).normal(size=(1,) + d.shape())
        plans.append(plan)
        ds.append(d)
        fs.append(to_dev(f, "f32"))
        psis.append(torch.empty(plan.out_shape, dtype=torch.float32, device="cuda"))
    batch = sf.Batch(plans)
    batch.solve(fs, psis)
    batch.sync()
    for plan, d, f, psi in zip(plans, ds, fs, psis):
        ref, _ = oracle.solve(d, to_np(f))
        assert rel_l2(to_np(psi)[0], ref[0]) <= TOL["f32"], d.bc
    batch.close()
    for p in plans:
        p.close()
