"""Shared helpers of the GPU tests: plan construction for both sides and error norms.

The CUDA side is reached only through the C ABI (paper_2301_01145_gb300 is a
ctypes binding); the reference side is the CPU oracle.
"""
import numpy as np

from oracle.desc import Desc

TOL = {"f32": 1e-5, "f64": 1e-12}  # relative L2 per output field (the stated targets)


def rel_l2(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.linalg.norm(ref)
    return np.linalg.norm(got - ref) / (den if den > 0 else 1.0)


def oracle_desc(dim, n, lo, hi, bc, grid="staggered", eig="PS", op="NONE", sigma=0.0, ncomp=1, rhs_scale=1.0):
    return Desc(dim, tuple(n[:dim]), tuple(lo[:dim]), tuple(hi[:dim]), tuple(bc[:dim]), grid == "staggered", eig, op,
                ncomp, rhs_scale, sigma)


def gpu_plan(dim, n, lo, hi, bc, grid="staggered", eig="PS", op="NONE", sigma=0.0, ncomp=1, prec="f32",
             rhs_scale=1.0, fused=True):
    import paper_2301_01145_gb300 as sf
    return sf.Plan(dim, tuple(n[:dim]), tuple(lo[:dim]), tuple(hi[:dim]), list(bc[:dim]), grid=grid, eig=eig, op=op,
                   sigma=sigma, ncomp=ncomp, prec=prec, rhs_scale=rhs_scale, fused=fused)


def to_dev(a, prec):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32 if prec == "f32" else torch.float64,
                        device="cuda")


def to_np(t):
    return t.detach().double().cpu().numpy()
