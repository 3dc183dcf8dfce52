"""GB300-native fast Poisson solver (spectral method of SailFFish, arXiv 2301.01145).

The compute path is libsailfish_gb300.so (hand-written sm_103a CUDA kernels
behind a C ABI, include/sailfish_gb300.h).  This package only marshals
arguments: device memory and streams come from PyTorch.

    import paper_2301_01145_gb300 as sf
    plan = sf.Plan(dim=3, n=(256,)*3, lo=(-.5,)*3, hi=(.5,)*3, bc="UUU",
                   op="CURL", ncomp=3, sigma=2/256, rhs_scale=-1.0)
    psi, u = plan(omega)          # omega: cuda tensor [3][256][256][256]
"""
from __future__ import annotations

from typing import Optional, Sequence

from . import _lib
from ._lib import SolverError  # noqa: F401
from ._lib import (sf_batch_create, sf_batch_solve, sf_execute, sf_get_output, sf_plan_create,  # noqa: F401
                   sf_plan_destroy, sf_plan_kernel_ms, sf_plan_launches, sf_plan_query, sf_plan_stats,
                   sf_plan_timing, sf_set_boundary, sf_set_source, sf_solve,
                   sf_solve_adjoint, sf_solve_host, sf_sync, sf_version)


def _torch():
    import torch
    return torch


class Plan:
    """A solver plan: lap(psi) = rhs_scale * f on one grid (Sec. 2.4 options)."""

    def __init__(self, dim: int, n: Sequence[int], lo: Sequence[float], hi: Sequence[float], bc,
                 grid: str = "staggered", eig: str = "PS", op: str = "NONE", sigma: float = 0.0, ncomp: int = 1,
                 prec: str = "f32", rhs_scale: float = 1.0, fused: bool = True, generic: bool = False, stream=None,
                 tune_radix: int = 0, tune_tile: int = 0, tune_slab: int = 0, tune_lag: int = 0,
                 kernel: str = "G2", debug_checks: bool = False):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("paper_2301_01145_gb300 needs a CUDA device")
        bc = list(bc) if isinstance(bc, str) else list(bc)
        flags = (0 if fused else _lib.FLAG_UNFUSED) | (_lib.FLAG_GENERIC if generic else 0) | \
            (_lib.FLAG_DEBUG_CHECKS if debug_checks else 0)
        self.desc = _lib.make_desc(dim, n, lo, hi, bc, grid, eig, op, sigma, ncomp, prec, rhs_scale, flags,
                                   tune_radix, tune_tile, tune_slab, tune_lag, kernel)
        self.dim, self.ncomp, self.op = dim, ncomp, op
        self.dtype = torch.float32 if prec == "f32" else torch.float64
        self.handle = sf_plan_create(self.desc, stream)
        ins, outs, ops, ws = sf_plan_query(self.handle)
        trim = (lambda s: (s[0],) + tuple(s[4 - dim:]))  # [ncomp] + the dim spatial extents
        self.in_shape = trim(tuple(ins))
        self.out_shape = trim(tuple(outs))
        self.op_shape = trim(tuple(ops)) if ops[0] else None
        self.workspace_bytes = ws
        self._faces = {}

    # -- paper's execution sequence (Sec. 2.4.5) --
    def set_source(self, f):
        self._src = f
        sf_set_source(self.handle, f)

    def set_boundary(self, axis: int, side: int, face):
        self._faces[(axis, side)] = face
        sf_set_boundary(self.handle, axis, side, face)

    def solve(self):
        sf_solve(self.handle)

    def get_output(self, psi, op_out=None):
        sf_get_output(self.handle, psi, op_out)

    # -- convenience --
    def empty_outputs(self):
        torch = _torch()
        psi = torch.empty(self.out_shape, dtype=self.dtype, device="cuda")
        opo = torch.empty(self.op_shape, dtype=self.dtype, device="cuda") if self.op_shape else None
        return psi, opo

    def execute(self, f, psi, op_out=None):
        sf_execute(self.handle, f, psi, op_out)

    def __call__(self, f):
        self._check_input(f)
        psi, opo = self.empty_outputs()
        sf_execute(self.handle, f, psi, opo)
        return (psi, opo) if opo is not None else psi

    def solve_host(self, f_host, psi_host, op_host=None):
        sf_solve_host(self.handle, f_host, psi_host, op_host)

    def solve_host_many(self, f_hosts, psi_hosts, op_hosts=None):
        """Pipelined host solves: uploads and downloads overlap the neighbouring solves."""
        _lib.sf_solve_host_many(self.handle, f_hosts, psi_hosts, op_hosts)

    def adjoint(self, g_psi=None, g_op=None, g_f=None):
        torch = _torch()
        if g_f is None:
            g_f = torch.empty(self.in_shape, dtype=self.dtype, device="cuda")
        sf_solve_adjoint(self.handle, g_psi, g_op, g_f)
        return g_f

    def sync(self):
        sf_sync(self.handle)

    def launches(self) -> int:
        return sf_plan_launches(self.handle)

    def stats(self):
        return sf_plan_stats(self.handle)

    def timing(self, enable: bool = True):
        """Start (and clear) or stop per-kernel CUDA-event timing of full solves."""
        sf_plan_timing(self.handle, enable)

    def kernel_ms(self):
        """(mean device ms of each kernel slot, number of solves averaged)."""
        return sf_plan_kernel_ms(self.handle)

    def _check_input(self, f):
        if tuple(f.shape) != tuple(self.in_shape) or f.dtype != self.dtype or not f.is_cuda or not f.is_contiguous():
            raise ValueError(f"source must be a contiguous cuda {self.dtype} tensor of shape {self.in_shape}")

    def close(self):
        if getattr(self, "handle", None) is not None:
            sf_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Independent plans solved together in one CUDA graph: one persistent launch
    for the general-engine members, plus the own launches of members on the
    register fast path."""

    def __init__(self, plans: Sequence[Plan], stream=None):
        self.plans = list(plans)
        self.handle = sf_batch_create([p.handle for p in self.plans], stream)

    def solve(self, fs, psis, ops: Optional[Sequence] = None):
        sf_batch_solve(self.handle, fs, psis, ops)

    def launches(self) -> int:
        return sf_plan_launches(self.handle)

    def sync(self):
        sf_sync(self.handle)

    def close(self):
        if getattr(self, "handle", None) is not None:
            sf_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lib_path() -> str:
    return _lib.LIB_PATH
