"""Batched uneven solves in one persistent launch (512 seeded problems: 2D 64^2..1024^2
and 3D 32^3..128^3, periodic / Dirichlet / Neumann / unbounded, regular and staggered).

Each problem of the batch must equal its own single solve bit for bit (same
engine, same tiles), and a sample of the problems is checked against the
oracle within the FP32 tolerance.
"""
import numpy as np
import pytest

import oracle
import workloads
from tests.gpu_helpers import TOL, oracle_desc, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built(gpu_available):
    import __graft_entry__ as g
    g.build()


def problem_kwargs(bp):
    dim = bp.dim
    n = bp.n_cells
    lo, hi = (-0.5,) * dim, (0.5,) * dim
    grid = "staggered" if bp.staggered else "regular"
    sigma = 2.0 / max(n) if bp.bc == "U" else 0.0
    return dict(dim=dim, n=n, lo=lo, hi=hi, bc=bp.bc * dim, grid=grid, eig="PS", sigma=sigma,
                rhs_scale=-1.0 if bp.bc == "U" else 1.0)


def source(bp):
    shape = tuple(reversed(bp.node_counts()))
    return workloads.lowpass_noise(shape, bp.seed)[None]


def test_batch_512_matches_single_solves_and_oracle():
    import torch
    import paper_2301_01145_gb300 as sf
    probs = workloads.batch_problems(512)
    plans, fs, psis = [], [], []
    for bp in probs:
        kw = problem_kwargs(bp)
        plan = sf.Plan(**kw, generic=True)
        plans.append(plan)
        fs.append(to_dev(source(bp), "f32"))
        psis.append(torch.empty(plan.out_shape, dtype=torch.float32, device="cuda"))
    batch = sf.Batch(plans)
    batch.solve(fs, psis)      # captures the graph
    batch.sync()
    first = [p.clone() for p in psis]
    batch.solve(fs, psis)      # replays it
    batch.sync()
    for i in range(len(probs)):
        assert torch.equal(first[i], psis[i])
        single = plans[i](fs[i])
        plans[i].sync()
        assert torch.equal(single, psis[i]), f"problem {i} ({probs[i]}) differs from its single solve"
    # oracle on a sample covering every boundary type, both grids and both dimensions
    picked, seen = [], set()
    for i, bp in enumerate(probs):
        key = (bp.dim, bp.bc, bp.staggered)
        pts = bp.out_points()
        if key not in seen and pts <= 300_000:
            seen.add(key)
            picked.append(i)
    assert len(picked) >= 8
    for i in picked:
        bp = probs[i]
        kw = problem_kwargs(bp)
        d = oracle_desc(kw["dim"], kw["n"], kw["lo"], kw["hi"], kw["bc"], kw["grid"], "PS", sigma=kw["sigma"],
                        rhs_scale=kw["rhs_scale"])
        ref, _ = oracle.solve(d, source(bp))
        assert rel_l2(to_np(psis[i])[0], ref[0]) <= TOL["f32"], (i, bp)
    batch.close()
    for p in plans:
        p.close()


def test_scheduler_wait_times_out_cleanly():
    # a dependency nothing satisfies: every wait gives up after its bound, the
    # kernel exits, the host reads SF_ERR_TIMEOUT, and the context stays usable
    import time
    import torch
    import paper_2301_01145_gb300 as sf
    t0 = time.time()
    assert sf._lib.sf_selftest_timeout(200) == -6
    assert time.time() - t0 < 30
    plan = sf.Plan(2, (64, 64), (0, 0), (1, 1), "PP")
    f = torch.randn(plan.in_shape, device="cuda")
    plan(f)
    plan.sync()
    plan.close()


def test_clean_batch_reports_no_timeout():
    import torch
    import paper_2301_01145_gb300 as sf
    plans = [sf.Plan(2, (64, 64), (0, 0), (1, 1), "PP", generic=True) for _ in range(3)]
    fs = [torch.randn(p.in_shape, device="cuda") for p in plans]
    ps = [p.empty_outputs()[0] for p in plans]
    batch = sf.Batch(plans)
    batch.solve(fs, ps)
    batch.sync()  # raises SolverError(SF_ERR_TIMEOUT) if a wait gave up
    batch.close()
    for p in plans:
        p.close()
