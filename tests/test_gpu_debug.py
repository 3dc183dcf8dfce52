"""Failure handling on the GPU without a GPU fault: the debug-checks flag (guard
bands around every device buffer of a plan, scanned by sf_sync) and the
allocation-failure injection hook.  The corruption is a host-issued write into
the plan's own guard band, and the allocation failures are refused by the
library before cudaMalloc is called, so nothing here faults or hangs a GPU.
"""
import numpy as np
import pytest

import workloads
from tests.gpu_helpers import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built(gpu_available):
    import __graft_entry__ as g
    g.build()


def unbounded_plan(n, debug_checks=False):
    import paper_2301_01145_gb300 as sf
    return sf.Plan(3, (n,) * 3, (-0.5,) * 3, (0.5,) * 3, "UUU", op="CURL", ncomp=3, sigma=2.0 / n, rhs_scale=-1.0,
                   debug_checks=debug_checks)


def bounded_plan(debug_checks=False):
    import paper_2301_01145_gb300 as sf
    return sf.Plan(3, (24, 16, 12), (0.0,) * 3, (1.0,) * 3, ["D", "N", "DN"], grid="regular", eig="FD2",
                   debug_checks=debug_checks)


@pytest.mark.parametrize("which", ["fast-128", "general-unbounded-24", "bounded-mixed"])
def test_debug_checks_solve_is_clean_and_identical(which):
    # guard bands change only the addresses of the plan's buffers: the outputs
    # are bit-identical to a plan without them and every band survives the solve
    import torch
    mk = {"fast-128": lambda dbg: unbounded_plan(128, dbg),
          "general-unbounded-24": lambda dbg: unbounded_plan(24, dbg),
          "bounded-mixed": lambda dbg: bounded_plan(dbg)}[which]
    plain, dbg = mk(False), mk(True)
    f = torch.tensor(np.random.default_rng(5).normal(size=plain.in_shape), dtype=torch.float32, device="cuda")
    outs_plain = plain(f)
    plain.sync()
    for _ in range(2):
        outs_dbg = dbg(f)
        dbg.sync()  # raises SolverError(SF_ERR_CORRUPT) if a band changed
    outs_plain = outs_plain if isinstance(outs_plain, tuple) else (outs_plain,)
    outs_dbg = outs_dbg if isinstance(outs_dbg, tuple) else (outs_dbg,)
    for a, b in zip(outs_plain, outs_dbg):
        assert torch.equal(a, b)
    # the adjoint path runs over the same guarded workspace
    g = dbg.adjoint(outs_dbg[0]) if which == "bounded-mixed" else None
    dbg.sync()
    plain.close()
    dbg.close()
    del g


def test_overwritten_guard_band_is_reported():
    from paper_2301_01145_gb300 import _lib
    plan = unbounded_plan(24, debug_checks=True)
    f = to_dev(workloads.gaussian_blobs(24)["omega"], "f32")
    plan(f)
    plan.sync()
    _lib.sf_debug_corrupt_guard(plan.handle)
    with pytest.raises(_lib.SolverError) as e:
        plan.sync()
    assert e.value.status == -7 and "guard band 0" in str(e.value)  # SF_ERR_CORRUPT
    plan.close()
    # a plan without guard bands refuses the hook
    plain = unbounded_plan(24)
    with pytest.raises(_lib.SolverError) as e:
        _lib.sf_debug_corrupt_guard(plain.handle)
    assert e.value.status == -5  # SF_ERR_STATE
    plain.close()


@pytest.mark.parametrize("which", ["fast-128", "bounded-mixed"])
def test_allocation_failure_at_every_point_releases_everything(which):
    # make the k-th device allocation of plan creation fail, for every k: each
    # attempt returns SF_ERR_OOM and frees what it had allocated; with the hook
    # off again a plan builds and solves as before
    import torch
    from paper_2301_01145_gb300 import _lib
    mk = (lambda: unbounded_plan(128)) if which == "fast-128" else bounded_plan
    ref_plan = mk()
    f = torch.tensor(np.random.default_rng(9).normal(size=ref_plan.in_shape), dtype=torch.float32, device="cuda")
    ref = ref_plan(f)
    ref = ref if isinstance(ref, tuple) else (ref,)
    ref_plan.sync()
    ref_plan.close()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failures = 0
    try:
        for after in range(400):
            _lib.sf_debug_fail_alloc(after)
            try:
                p = mk()
            except _lib.SolverError as e:
                assert e.status == -4, str(e)  # SF_ERR_OOM
                failures += 1
                continue
            _lib.sf_debug_fail_alloc(-1)
            p.close()
            break
        else:
            pytest.fail("plan creation never succeeded")
    finally:
        _lib.sf_debug_fail_alloc(-1)
    assert failures == after and failures >= 10
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 >= free0 - (64 << 20), (free0, free1)  # one leaked workspace would be hundreds of MB
    plan = mk()
    out = plan(f)
    out = out if isinstance(out, tuple) else (out,)
    plan.sync()
    for a, b in zip(ref, out):
        assert torch.equal(a, b)
    plan.close()
