"""sf_solve_static: the solve for callers that cannot allocate device memory.

It must give the same result as the plan-based entry point (sf_plan_create +
sf_execute) within the FP32 tolerance of the other tests, on two calls in a
row (the second call reuses the workspace the first one left behind), and it
must refuse a problem whose workspace exceeds its fixed device array.  This
file is collected last so that a failure here never hides the other tests.
"""
import numpy as np
import pytest

from tests.gpu_helpers import TOL, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu

CASES = [
    dict(dim=3, n=(64, 48, 32), lo=(0, 0, 0), hi=(1.0, 0.8, 1.3), bc="PPP", grid="staggered", eig="PS"),
    dict(dim=3, n=(32, 24, 16), lo=(0, 0, 0), hi=(1, 1, 1), bc="DND", grid="regular", eig="FD2"),
    dict(dim=2, n=(128, 96), lo=(-1, 0), hi=(1, 1), bc="NN", grid="staggered", eig="PS"),
    dict(dim=2, n=(64, 256), lo=(0, 0), hi=(1, 2), bc="DD", grid="regular", eig="FD2"),
]


@pytest.fixture(scope="module", autouse=True)
def _built(gpu_available):
    import __graft_entry__ as g
    g.build()


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c['dim']}D-{c['bc']}-{c['grid']}")
def test_static_matches_plan_twice(case):
    import torch
    import paper_2301_01145_gb300 as sf
    from paper_2301_01145_gb300 import _lib
    plan = sf.Plan(case["dim"], case["n"], case["lo"], case["hi"], case["bc"], grid=case["grid"], eig=case["eig"],
                   rhs_scale=-1.5)
    rng = np.random.default_rng(sum(case["n"]))
    f = to_dev(rng.normal(size=plan.in_shape), "f32")
    ref = to_np(plan(f))
    plan.sync()
    desc = _lib.make_desc(case["dim"], case["n"], case["lo"], case["hi"], list(case["bc"]), case["grid"],
                          case["eig"], rhs_scale=-1.5)
    for call in range(2):
        psi = torch.full(plan.out_shape, float("nan"), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        if call == 1:
            # the second call must allocate nothing: the library's allocation hook
            # refuses any allocation, and the device's free memory must not move
            free_before = torch.cuda.mem_get_info()[0]
            _lib.sf_debug_fail_alloc(0)
        try:
            _lib.sf_solve_static(desc, f, psi)
            torch.cuda.synchronize()
        finally:
            _lib.sf_debug_fail_alloc(-1)
        if call == 1:
            assert torch.cuda.mem_get_info()[0] == free_before
        got = to_np(psi)
        assert np.all(np.isfinite(got))
        assert rel_l2(got[0], ref[0]) <= TOL["f32"]
    plan.close()


def test_static_refuses_oversized_problem():
    import torch
    from paper_2301_01145_gb300 import _lib
    desc = _lib.make_desc(3, (512, 512, 512), (0, 0, 0), (1, 1, 1), list("PPP"))
    f = torch.zeros(1, device="cuda")
    with pytest.raises(_lib.SolverError) as e:
        _lib.sf_solve_static(desc, f, f)
    assert e.value.status == -1
    # the refusal says how much workspace the problem would need
    assert "bytes of workspace" in str(e.value)
