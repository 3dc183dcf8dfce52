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


def test_batch_runs_register_path_members_on_their_own_launches():
    # members eligible for the register fast path (3D unbounded 128^3 curl:
    # padded 256-point axes; 3D periodic 256^3) run their own launches in the
    # batch's graph, the others the persistent launch; every member equals its
    # single solve bit for bit, also after the buffers change (re-capture)
    import torch
    import paper_2301_01145_gb300 as sf
    specs = [dict(dim=3, n=(128,) * 3, lo=(-0.5,) * 3, hi=(0.5,) * 3, bc="UUU", op="CURL", ncomp=3, sigma=2.0 / 128,
                  rhs_scale=-1.0),
             dict(dim=2, n=(256, 192), lo=(0.0, 0.0), hi=(1.0, 1.0), bc="DN", grid="regular"),
             dict(dim=3, n=(256,) * 3, lo=(0.0,) * 3, hi=(1.0,) * 3, bc="PPP"),
             dict(dim=3, n=(32, 48, 64), lo=(-0.5,) * 3, hi=(0.5,) * 3, bc="UUU", sigma=1.0 / 24, rhs_scale=-1.0)]
    plans = [sf.Plan(**s) for s in specs]
    batch = sf.Batch(plans)
    assert batch.launches() == 1 + 3 * 2
    rng = np.random.default_rng(21)
    for rep in range(2):
        fs = [to_dev(rng.normal(size=pl.in_shape), "f32") for pl in plans]
        psis = [torch.empty(pl.out_shape, dtype=torch.float32, device="cuda") for pl in plans]
        ops = [torch.empty(pl.op_shape, dtype=torch.float32, device="cuda") if pl.op_shape else None for pl in plans]
        batch.solve(fs, psis, ops)
        batch.sync()
        for pl, f, psi, opo in zip(plans, fs, psis, ops):
            out = pl(f)
            pl.sync()
            ref_psi, ref_op = out if isinstance(out, tuple) else (out, None)
            assert torch.equal(psi, ref_psi)
            if opo is not None:
                assert torch.equal(opo, ref_op)
    batch.close()
    for pl in plans:
        pl.close()


def test_batch_refuses_missing_buffers():
    # a member with an operator and no op output, or a null source, is refused
    # on the host (SF_ERR_ARG) before anything is launched
    import torch
    import paper_2301_01145_gb300 as sf
    from paper_2301_01145_gb300 import SolverError
    plans = [sf.Plan(3, (32,) * 3, (-0.5,) * 3, (0.5,) * 3, "UUU", op="CURL", ncomp=3, sigma=1.0 / 16, rhs_scale=-1.0),
             sf.Plan(2, (64, 32), (0.0, 0.0), (1.0, 1.0), "PP")]
    batch = sf.Batch(plans)
    fs = [torch.randn(pl.in_shape, device="cuda") for pl in plans]
    psis = [torch.empty(pl.out_shape, device="cuda") for pl in plans]
    with pytest.raises(SolverError) as e:
        batch.solve(fs, psis, None)
    assert e.value.status == -1
    with pytest.raises(SolverError) as e:
        batch.solve(fs, psis, [None, None])
    assert e.value.status == -1
    ops = [torch.empty(plans[0].op_shape, device="cuda"), None]
    batch.solve(fs, psis, ops)
    batch.sync()
    batch.close()
    for pl in plans:
        pl.close()
