"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, element
by element, at sizes the oracle finishes in seconds.  Sizes are chosen to span
several tiles with ragged tails (odd unknown counts, 3*2^p lengths).

Tolerances (relative L2 per output field): 1e-5 for FP32, 1e-12 for FP64.
"""
import itertools
import math

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


def run_both(dim, n, lo, hi, bc, grid="staggered", eig="PS", op="NONE", sigma=0.0, ncomp=1, prec="f32",
             rhs_scale=1.0, faces=None, seed=0, fused=True, f=None):
    d = oracle_desc(dim, n, lo, hi, bc, grid, eig, op, sigma, ncomp, rhs_scale)
    shape = (ncomp,) + d.shape()
    if f is None:
        f = np.random.default_rng(seed).normal(size=shape)
    plan = gpu_plan(dim, n, lo, hi, bc, grid, eig, op, sigma, ncomp, prec, rhs_scale, fused)
    ft = to_dev(f, prec)
    if faces:
        for (ax, side), g in faces.items():
            plan.set_boundary(ax, side, to_dev(g, prec))
    psi, opo = plan.empty_outputs()
    plan.execute(ft, psi, opo)
    plan.sync()
    ref_psi, ref_op = oracle.solve(d, f, faces)
    out = {"psi": (to_np(psi), ref_psi)}
    if opo is not None:
        out["op"] = (to_np(opo), ref_op)
    plan.close()
    return out


def assert_close(out, prec, factor=1.0):
    for name, (g, r) in out.items():
        for c in range(r.shape[0]):
            e = rel_l2(g[c], r[c])
            assert e <= TOL[prec] * factor, f"{name}[{c}] rel L2 {e:.3e}"


# ---------------------------------------------------------------------------
# periodic (Table 1 last row), C1 configuration and variations
# ---------------------------------------------------------------------------

def test_c1_periodic_64_fp64_exact():
    pm = workloads.periodic_modes(64, seed_index=0)
    out = run_both(3, (64,) * 3, (0,) * 3, (2 * math.pi,) * 3, "PPP", prec="f64", f=pm.f[None])
    assert_close(out, "f64")
    assert np.max(np.abs(out["psi"][0][0] - pm.psi_exact)) < 1e-12


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("eig", ["PS", "FD2"])
@pytest.mark.parametrize("n", [(32, 24, 16), (12, 48, 6), (96, 4, 8)])
def test_periodic_3d(prec, eig, n):
    out = run_both(3, n, (0, -1, 0.5), (1.0, 1.5, 2.0), "PPP", eig=eig, prec=prec, seed=sum(n))
    assert_close(out, prec)


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("n", [(64, 48), (6, 128), (1024, 8)])
def test_periodic_2d(prec, n):
    out = run_both(2, n, (0, 0), (1.0, 0.7), "PP", eig="PS", prec=prec, seed=n[0])
    assert_close(out, prec)


@pytest.mark.parametrize("op,ncomp", [("GRAD", 1), ("DIV", 3), ("CURL", 3), ("NABLA", 1), ("NABLA", 3)])
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_periodic_operators_3d(op, ncomp, prec):
    out = run_both(3, (16, 24, 12), (0, 0, 0), (1.0, 1.3, 0.8), "PPP", op=op, ncomp=ncomp, prec=prec, seed=3)
    assert_close(out, prec)


@pytest.mark.parametrize("op,ncomp", [("GRAD", 1), ("DIV", 2), ("CURL", 1), ("NABLA", 2)])
def test_periodic_operators_2d(op, ncomp):
    out = run_both(2, (48, 32), (0, 0), (1.0, 2.0), "PP", op=op, ncomp=ncomp, prec="f64", seed=4)
    assert_close(out, "f64")


# ---------------------------------------------------------------------------
# Dirichlet / Neumann (DST/DCT types of Table 1), homogeneous and FD2 lifted
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("bcs", ["".join(p) for p in itertools.product("DN", repeat=3)])
@pytest.mark.parametrize("grid", ["regular", "staggered"])
def test_bounded_3d_fp64_ps(bcs, grid):
    out = run_both(3, (12, 8, 16), (0, 0, 0), (1.0, 0.5, 2.0), bcs, grid=grid, eig="PS", prec="f64", seed=7)
    assert_close(out, "f64")


@pytest.mark.parametrize("bcs", ["".join(p) for p in itertools.product("DN", repeat=3)])
@pytest.mark.parametrize("grid", ["regular", "staggered"])
def test_bounded_3d_fp32_fd2_inhomogeneous(bcs, grid):
    man = workloads.manufactured(seed_index=5)
    n = (12, 24, 8)
    case = workloads.bounded_case(man, n, tuple(bcs), grid == "staggered")
    out = run_both(3, n, (0, 0, 0), (1.0, 1.0, 1.0), bcs, grid=grid, eig="FD2", prec="f32", rhs_scale=1.0,
                   faces=case["faces"], f=case["f"][None])
    assert_close(out, "f32")


@pytest.mark.parametrize("bcs", ["".join(p) for p in itertools.product("DN", repeat=2)])
@pytest.mark.parametrize("grid", ["regular", "staggered"])
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_bounded_2d(bcs, grid, prec):
    out = run_both(2, (24, 12), (0, 0), (1.0, 0.6), bcs, grid=grid, eig="FD2", prec=prec, seed=9, rhs_scale=-2.5)
    assert_close(out, prec)


def test_bounded_vector_components():
    out = run_both(3, (8, 16, 12), (0, 0, 0), (1, 1, 1), "DND", grid="regular", eig="PS", ncomp=3, prec="f64", seed=2)
    assert_close(out, "f64")


# ---------------------------------------------------------------------------
# unbounded (Hockney-Eastwood, G2 kernel)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("n", [(16, 16, 16), (16, 12, 8), (6, 24, 32)])
def test_unbounded_curl_3d(prec, n):
    h = 1.0 / max(n)
    out = run_both(3, n, (-0.5,) * 3, (0.5,) * 3, "UUU", op="CURL", ncomp=3, sigma=2 * h, rhs_scale=-1.0,
                   prec=prec, seed=11)
    assert_close(out, prec)


@pytest.mark.parametrize("op,ncomp", [("NONE", 1), ("GRAD", 1), ("DIV", 3), ("NABLA", 2)])
def test_unbounded_ops_3d(op, ncomp):
    out = run_both(3, (12, 16, 8), (-0.5, -0.4, -0.3), (0.5, 0.6, 0.7), "UUU", op=op, ncomp=ncomp, sigma=0.1,
                   rhs_scale=0.7, prec="f64", seed=12)
    assert_close(out, "f64")


@pytest.mark.parametrize("op,ncomp", [("NONE", 1), ("GRAD", 1), ("CURL", 1)])
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_unbounded_2d(op, ncomp, prec):
    out = run_both(2, (48, 32), (-0.5, -0.5), (0.5, 0.5), "UU", op=op, ncomp=ncomp, sigma=0.04, rhs_scale=-1.0,
                   prec=prec, seed=13)
    assert_close(out, prec)


def test_unbounded_ring_fp32():
    ring = workloads.vortex_ring(32)
    out = run_both(3, (32,) * 3, (-0.5,) * 3, (0.5,) * 3, "UUU", op="CURL", ncomp=3, sigma=2 / 32, rhs_scale=-1.0,
                   prec="f32", f=ring["omega"])
    assert_close(out, "f32")


# ---------------------------------------------------------------------------
# execution modes and API paths
# ---------------------------------------------------------------------------

def test_fused_equals_unfused_bitwise():
    import torch
    f = np.random.default_rng(1).normal(size=(3, 16, 12, 8))
    res = []
    for fused in (True, False):
        plan = gpu_plan(3, (8, 12, 16), (-0.5,) * 3, (0.5,) * 3, "UUU", op="CURL", ncomp=3, sigma=0.1,
                        rhs_scale=-1.0, fused=fused)
        psi, u = plan(to_dev(f, "f32"))
        plan.sync()
        res.append((psi.clone(), u.clone()))
        plan.close()
    assert torch.equal(res[0][0], res[1][0]) and torch.equal(res[0][1], res[1][1])


def test_solve_then_get_output_matches_execute():
    import torch
    f = to_dev(np.random.default_rng(2).normal(size=(1, 17, 9, 13)), "f64")
    plan = gpu_plan(3, (12, 8, 16), (0,) * 3, (1,) * 3, "NDN", grid="regular", eig="FD2", prec="f64")
    psi1, _ = plan.empty_outputs()
    plan.execute(f, psi1)
    psi2, _ = plan.empty_outputs()
    plan.set_source(f)
    plan.solve()
    plan.get_output(psi2)
    plan.sync()
    assert torch.equal(psi1, psi2)
    plan.close()


def test_solve_host_matches_device():
    import torch
    f = np.random.default_rng(3).normal(size=(3, 16, 16, 16))
    plan = gpu_plan(3, (16,) * 3, (-0.5,) * 3, (0.5,) * 3, "UUU", op="CURL", ncomp=3, sigma=0.1, rhs_scale=-1.0)
    fd = to_dev(f, "f32")
    psi, u = plan(fd)
    hf = fd.cpu().pin_memory()
    hpsi = torch.empty(psi.shape, dtype=psi.dtype).pin_memory()
    hu = torch.empty(u.shape, dtype=u.dtype).pin_memory()
    plan.solve_host(hf, hpsi, hu)
    assert torch.equal(hpsi, psi.cpu()) and torch.equal(hu, u.cpu())
    plan.close()


def test_repeated_solves_are_deterministic():
    import torch
    f = to_dev(np.random.default_rng(4).normal(size=(1, 32, 24, 16)), "f32")
    plan = gpu_plan(3, (16, 24, 32), (0,) * 3, (1,) * 3, "PPP")
    a = plan(f).clone()
    for _ in range(3):
        b = plan(f)
    plan.sync()
    assert torch.equal(a, b)
    plan.close()


def test_gpu_error_paths():
    import paper_2301_01145_gb300 as sf
    plan = gpu_plan(3, (16,) * 3, (0,) * 3, (1,) * 3, "PPP")
    with pytest.raises(sf.SolverError):
        plan.set_boundary(0, 0, to_dev(np.zeros((16, 16)), "f32"))  # periodic axis has no face data
    with pytest.raises(sf.SolverError):
        sf.sf_get_output(plan.handle, to_dev(np.zeros((1, 16, 16, 16)), "f32"))  # before any solve
    plan.close()
    plan = gpu_plan(3, (16,) * 3, (0,) * 3, (1,) * 3, "DDD", eig="PS")
    with pytest.raises(sf.SolverError):
        plan.set_boundary(0, 0, to_dev(np.zeros((17, 17)), "f32"))  # inhomogeneous needs FD2
    plan.close()


# ---------------------------------------------------------------------------
# adjoint (transposed solve) against the oracle's transpose
# ---------------------------------------------------------------------------

ADJ_CASES = [
    dict(dim=3, n=(8, 12, 16), lo=(-0.5,) * 3, hi=(0.5,) * 3, bc="UUU", op="CURL", ncomp=3, sigma=0.1, rhs_scale=-1.0),
    dict(dim=3, n=(8, 8, 12), lo=(-0.5,) * 3, hi=(0.5,) * 3, bc="UUU", op="GRAD", ncomp=1, sigma=0.15, rhs_scale=2.0),
    dict(dim=2, n=(16, 12), lo=(0, 0), hi=(1, 1), bc="PP", op="DIV", ncomp=2),
    dict(dim=3, n=(12, 8, 16), lo=(0,) * 3, hi=(1,) * 3, bc="NDN", grid="regular", eig="FD2", rhs_scale=0.5),
    dict(dim=3, n=(12, 8, 16), lo=(0,) * 3, hi=(1,) * 3, bc="DNN", grid="staggered", eig="PS"),
    dict(dim=2, n=(12, 24), lo=(0, 0), hi=(1, 2), bc="NN", grid="regular", eig="FD2"),
]


@pytest.mark.parametrize("case", ADJ_CASES, ids=lambda c: f"{c['dim']}D-{c['bc']}-{c.get('op', 'NONE')}")
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_adjoint_vs_oracle(case, prec):
    c = dict(case)
    dim = c.pop("dim")
    d = oracle_desc(dim, c["n"], c["lo"], c["hi"], c["bc"], c.get("grid", "staggered"), c.get("eig", "PS"),
                    c.get("op", "NONE"), c.get("sigma", 0.0), c.get("ncomp", 1), c.get("rhs_scale", 1.0))
    plan = gpu_plan(dim, c["n"], c["lo"], c["hi"], c["bc"], c.get("grid", "staggered"), c.get("eig", "PS"),
                    c.get("op", "NONE"), c.get("sigma", 0.0), c.get("ncomp", 1), prec, c.get("rhs_scale", 1.0))
    rng = np.random.default_rng(21)
    gp = rng.normal(size=(d.ncomp,) + d.shape())
    go = rng.normal(size=(d.op_components(),) + d.shape()) if d.op != "NONE" else None
    gf = plan.adjoint(to_dev(gp, prec), to_dev(go, prec) if go is not None else None)
    plan.sync()
    ref = oracle.adjoint_solve(d, gp, go)
    for comp in range(ref.shape[0]):
        assert rel_l2(to_np(gf)[comp], ref[comp]) <= TOL[prec]
    plan.close()


# ---------------------------------------------------------------------------
# batch: one persistent launch over uneven problems
# ---------------------------------------------------------------------------

def test_small_batch_matches_single_solves_and_oracle():
    import torch
    import paper_2301_01145_gb300 as sf
    probs = [
        dict(dim=2, n=(64, 48), bc="PP"), dict(dim=3, n=(16, 12, 8), bc="UUU"), dict(dim=2, n=(24, 96), bc="DD", grid="regular"),
        dict(dim=3, n=(8, 16, 12), bc="NNN", grid="staggered"), dict(dim=2, n=(32, 32), bc="UU"),
        dict(dim=3, n=(12, 12, 12), bc="DDD", grid="staggered"), dict(dim=2, n=(128, 6), bc="NN", grid="regular"),
    ]
    plans, fs, psis, refs = [], [], [], []
    for i, p in enumerate(probs):
        dim = p["dim"]
        grid = p.get("grid", "staggered")
        lo, hi = (-0.5,) * dim, (0.5,) * dim
        sigma = 2.0 / max(p["n"]) if p["bc"][0] == "U" else 0.0
        plan = gpu_plan(dim, p["n"], lo, hi, p["bc"], grid, "PS", sigma=sigma)
        d = oracle_desc(dim, p["n"], lo, hi, p["bc"], grid, "PS", sigma=sigma)
        f = np.random.default_rng(100 + i).normal(size=(1,) + d.shape())
        plans.append(plan)
        fs.append(to_dev(f, "f32"))
        psis.append(torch.empty(plan.out_shape, dtype=torch.float32, device="cuda"))
        refs.append(oracle.solve(d, f)[0])
    batch = sf.Batch(plans)
    for _ in range(2):
        batch.solve(fs, psis)
    batch.sync()
    for i, plan in enumerate(plans):
        single = plan(fs[i])
        plan.sync()
        assert torch.equal(single, psis[i]), f"problem {i} differs from its single solve"
        assert rel_l2(to_np(psis[i])[0], refs[i][0]) <= TOL["f32"]
    batch.close()
    for p in plans:
        p.close()


def test_kernel_timing_slots():
    # per-kernel CUDA-event timing: 3 slots on the register path, 1 on the general engine
    import torch
    import paper_2301_01145_gb300 as sf
    for generic, nslot in ((False, 3), (True, 1)):
        plan = sf.Plan(3, (128,) * 3, (-0.5,) * 3, (0.5,) * 3, "UUU", op="CURL", ncomp=3, sigma=2 / 128,
                       rhs_scale=-1.0, generic=generic)
        f = torch.randn(plan.in_shape, device="cuda")
        psi, u = plan.empty_outputs()
        ms, nsol = plan.kernel_ms()
        assert nsol == 0
        plan.timing(True)
        for _ in range(3):
            plan.execute(f, psi, u)
        ms, nsol = plan.kernel_ms()
        assert nsol == 3 and len(ms) == nslot and all(t > 0 for t in ms)
        plan.timing(False)
        plan.execute(f, psi, u)
        plan.sync()
        plan.close()


def test_fp32_fma_probe():
    # measured FMA stream vs the unit-count peak (152 SMs x 128 lanes x 2 x up to 2.07 GHz)
    import paper_2301_01145_gb300 as sf
    tf = sf._lib.sf_probe_fp32_fma()
    assert 10.0 < tf < 90.0


def test_solve_host_many_matches_device_solves():
    # pipelined host solves (uploads / downloads overlapping the solves) equal device solves
    import torch
    import paper_2301_01145_gb300 as sf
    n = 64
    plan = sf.Plan(3, (n,) * 3, (-0.5,) * 3, (0.5,) * 3, "UUU", op="CURL", ncomp=3, sigma=2 / n, rhs_scale=-1.0)
    fs = [torch.randn(plan.in_shape).pin_memory() for _ in range(5)]
    ps = [torch.empty(plan.out_shape).pin_memory() for _ in range(5)]
    us = [torch.empty(plan.op_shape).pin_memory() for _ in range(5)]
    plan.solve_host_many(fs, ps, us)
    for i in range(5):
        psi, u = plan(fs[i].cuda())
        plan.sync()
        assert torch.equal(psi.cpu(), ps[i]) and torch.equal(u.cpu(), us[i])
    # repeated input buffer, two alternating outputs
    plan.solve_host_many([fs[0]] * 4, [ps[0], ps[1]] * 2, [us[0], us[1]] * 2)
    psi, u = plan(fs[0].cuda())
    plan.sync()
    assert torch.equal(psi.cpu(), ps[0]) and torch.equal(psi.cpu(), ps[1])
    plan.close()
