"""Differentiable unbounded solve (128^3 doubled to 256^3, curl), the adjoint path.

The loss L = sum w |u|^2 with u = curl psi(omega) is quadratic in omega, so
central differences are exact up to rounding: the FP64 solve gives the
finite-difference reference, the FP32 gradient must agree to 1e-4 relative to
max|g| and the FP64 gradient to 1e-9.  The gradient is also checked against
the oracle's transposed solve and by the dot-product identity.
"""
import numpy as np
import pytest

import oracle
import workloads
from oracle.desc import Desc
from tests.gpu_helpers import rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu

N = 128


@pytest.fixture(scope="module", autouse=True)
def _built(gpu_available):
    import __graft_entry__ as g
    g.build()


def make(prec):
    import paper_2301_01145_gb300 as sf
    return sf.Plan(3, (N,) * 3, (-0.5,) * 3, (0.5,) * 3, "UUU", op="CURL", ncomp=3, sigma=2.0 / N, rhs_scale=-1.0,
                   prec=prec)


def loss_and_grad(plan, omega, w, prec):
    import torch
    from paper_2301_01145_gb300.autograd import poisson_solve
    x = to_dev(omega, prec).requires_grad_(True)
    wt = to_dev(w, prec)
    psi, u = poisson_solve(x, plan)
    L = (wt[None] * u * u).sum()
    L.backward()
    return float(L.detach().double()), x.grad.detach()


def test_c5_gradient_fd_and_oracle():
    import torch
    data = workloads.gaussian_blobs(N)
    omega, w = data["omega"], data["w"]
    p32, p64 = make("f32"), make("f64")
    _, g32 = loss_and_grad(p32, omega, w, "f32")
    L64, g64 = loss_and_grad(p64, omega, w, "f64")
    g32 = to_np(g32)
    g64 = to_np(g64)
    gmax = np.max(np.abs(g64))
    # central differences on 32 seeded voxels with the FP64 solve (h = 1e-3)
    rng = np.random.default_rng(5)
    h = 1e-3
    o64 = to_dev(omega, "f64")
    wt = to_dev(w, "f64")
    for _ in range(32):
        c = int(rng.integers(0, 3))
        z, y, xx = (int(v) for v in rng.integers(0, N, size=3))
        vals = []
        for s in (+1, -1):
            o = o64.clone()
            o[c, z, y, xx] += s * h
            psi, u = p64(o)
            vals.append(float((wt[None] * u * u).sum()))
        fd = (vals[0] - vals[1]) / (2 * h)
        # L is quadratic: central differences are exact up to the rounding of L itself
        fd_round = 64 * np.finfo(np.float64).eps * abs(L64) / h
        assert abs(g64[c, z, y, xx] - fd) <= 1e-9 * gmax + fd_round, (fd, g64[c, z, y, xx], fd_round)
        assert abs(g32[c, z, y, xx] - fd) <= 1e-4 * gmax
    # whole-field agreement of the FP32 gradient with the FP64 one
    for c in range(3):
        assert rel_l2(g32[c], g64[c]) <= 1e-5
    p32.close()
    p64.close()


def test_adjoint_vs_oracle_transpose_small():
    # the oracle's literal transpose at a size it handles in full
    import torch
    import paper_2301_01145_gb300 as sf
    n = 32
    d = Desc(3, (n,) * 3, (-0.5,) * 3, (0.5,) * 3, ("U",) * 3, True, op="CURL", ncomp=3, rhs_scale=-1.0, sigma=2 / n)
    rng = np.random.default_rng(8)
    gp = rng.normal(size=(3, n, n, n))
    gu = rng.normal(size=(3, n, n, n))
    ref = oracle.adjoint_solve(d, gp, gu)
    for prec, tol in (("f32", 1e-5), ("f64", 1e-12)):
        plan = sf.Plan(3, (n,) * 3, (-0.5,) * 3, (0.5,) * 3, "UUU", op="CURL", ncomp=3, sigma=2 / n,
                       rhs_scale=-1.0, prec=prec)
        gf = plan.adjoint(to_dev(gp, prec), to_dev(gu, prec))
        plan.sync()
        for c in range(3):
            assert rel_l2(to_np(gf)[c], ref[c]) <= tol
        plan.close()


def test_c5_dot_product_identity_fp32_fast_path():
    # <A x, y> = <x, A^T y> on the register fast path (L = 256)
    import torch
    data = workloads.gaussian_blobs(N)
    plan = make("f32")
    x = to_dev(data["omega"], "f32")
    rng = np.random.default_rng(3)
    yp = to_dev(rng.normal(size=(3, N, N, N)), "f32")
    yu = to_dev(rng.normal(size=(3, N, N, N)), "f32")
    psi, u = plan(x)
    gf = plan.adjoint(yp, yu)
    plan.sync()
    lhs = float((psi.double() * yp.double()).sum() + (u.double() * yu.double()).sum())
    rhs = float((x.double() * gf.double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)
    plan.close()


@pytest.mark.parametrize("dim,n,op,ncomp", [(3, (24, 20, 16), "CURL", 3), (2, (40, 30), "GRAD", 1),
                                            (3, (16, 16, 16), "NONE", 1)])
def test_adjoint_regular_grid_unbounded_vs_oracle(dim, n, op, ncomp):
    # unbounded solves on regular grids (N_c + 1 nodes, doubled length 2^p or 3 * 2^p
    # >= 2 N_c + 1): the adjoint against the oracle's literal transpose
    import paper_2301_01145_gb300 as sf
    lo, hi = (-0.5,) * dim, (0.5, 0.4, 0.45)[:dim]
    sigma = 2.0 * max((hi[a] - lo[a]) / n[a] for a in range(dim))
    d = Desc(dim, n, lo, hi, ("U",) * dim, False, op=op, ncomp=ncomp, rhs_scale=-1.0, sigma=sigma)
    rng = np.random.default_rng(31)
    gp = rng.normal(size=(ncomp,) + d.shape())
    nop = d.op_components() if op != "NONE" else 0
    go = rng.normal(size=(nop,) + d.shape()) if nop else None
    ref = oracle.adjoint_solve(d, gp, go)
    for prec, tol in (("f32", 1e-5), ("f64", 1e-12)):
        plan = sf.Plan(dim, n, lo, hi, "U" * dim, grid="regular", op=op, ncomp=ncomp, sigma=sigma, rhs_scale=-1.0,
                       prec=prec)
        gf = plan.adjoint(to_dev(gp, prec), to_dev(go, prec) if go is not None else None)
        plan.sync()
        for c in range(ncomp):
            assert rel_l2(to_np(gf)[c], ref[c]) <= tol, (prec, c)
        plan.close()
