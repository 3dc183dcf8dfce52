"""ctypes binding of libsailfish_gb300.so (argument marshalling only).

Every function here has the name of the C entry point it wraps
(include/sailfish_gb300.h) and raises SolverError on a non-zero status.
Device buffers are passed as raw pointers taken from torch tensors; the CUDA
stream is torch's current stream unless one is given.  No computation happens
in Python: the library must be built (``__graft_entry__.build()``) and a
missing library is an error, never a fallback.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int, c_int32, c_size_t, c_uint32, c_void_p

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libsailfish_gb300.so")

SF_OK = 0
STATUS = {0: "SF_OK", -1: "SF_ERR_ARG", -2: "SF_ERR_UNSUPPORTED", -3: "SF_ERR_CUDA", -4: "SF_ERR_OOM",
          -5: "SF_ERR_STATE", -6: "SF_ERR_TIMEOUT", -7: "SF_ERR_CORRUPT"}

BC = {"P": 0, "D": 1, "N": 2, "U": 3}
GRID = {"regular": 0, "staggered": 1}
OP = {"NONE": 0, "GRAD": 1, "DIV": 2, "CURL": 3, "NABLA": 4}
EIG = {"PS": 0, "FD2": 1}
PREC = {"f32": 0, "f64": 1}
FLAG_UNFUSED = 1
FLAG_GENERIC = 2
FLAG_DEBUG_CHECKS = 4


class SolverError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {detail}")
        self.status = status


class sf_plan_desc(ctypes.Structure):
    _fields_ = [
        ("dim", c_int32),
        ("n", c_int32 * 3),
        ("lo", c_double * 3),
        ("hi", c_double * 3),
        ("bc", (c_int32 * 2) * 3),
        ("grid", c_int32),
        ("eig", c_int32),
        ("op", c_int32),
        ("green", c_int32),
        ("green_sigma", c_double),
        ("ncomp", c_int32),
        ("prec", c_int32),
        ("rhs_scale", c_double),
        ("flags", c_uint32),
        ("tune_radix", c_int32),
        ("tune_tile", c_int32),
        ("tune_slab", c_int32),
        ("tune_lag", c_int32),
    ]


_lib = None

# name -> (restype, argtypes)
SIGNATURES = {
    "sf_plan_create": (c_int, [POINTER(c_void_p), POINTER(sf_plan_desc), c_void_p]),
    "sf_plan_set_stream": (c_int, [c_void_p, c_void_p]),
    "sf_plan_query": (c_int, [c_void_p, POINTER(c_size_t), POINTER(c_size_t), POINTER(c_size_t), POINTER(c_size_t)]),
    "sf_set_source": (c_int, [c_void_p, c_void_p]),
    "sf_set_boundary": (c_int, [c_void_p, c_int, c_int, c_void_p]),
    "sf_solve": (c_int, [c_void_p]),
    "sf_get_output": (c_int, [c_void_p, c_void_p, c_void_p]),
    "sf_execute": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "sf_solve_host": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "sf_solve_adjoint": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "sf_batch_create": (c_int, [POINTER(c_void_p), POINTER(c_void_p), c_int, c_void_p]),
    "sf_batch_solve": (c_int, [c_void_p, POINTER(c_void_p), POINTER(c_void_p), POINTER(c_void_p)]),
    "sf_sync": (c_int, [c_void_p]),
    "sf_plan_launches": (c_int, [c_void_p]),
    "sf_selftest_timeout": (c_int, [c_int, c_void_p]),
    "sf_solve_static": (c_int, [POINTER(sf_plan_desc), c_void_p, c_void_p, c_void_p]),
    "sf_plan_stats": (c_int, [c_void_p, POINTER(c_double)]),
    "sf_plan_timing": (c_int, [c_void_p, c_int]),
    "sf_debug_fail_alloc": (c_int, [c_int]),
    "sf_debug_corrupt_guard": (c_int, [c_void_p]),
    "sf_solve_host_many": (c_int, [c_void_p, c_int, POINTER(c_void_p), POINTER(c_void_p), POINTER(c_void_p)]),
    "sf_probe_fp32_fma": (c_int, [POINTER(c_double), c_void_p]),
    "sf_eval_special": (c_int, [c_int, c_int, POINTER(c_double), POINTER(c_double)]),
    "sf_plan_kernel_ms": (c_int, [c_void_p, POINTER(c_double), POINTER(c_int), POINTER(c_int)]),
    "sf_plan_destroy": (c_int, [c_void_p]),
    "sf_status_string": (c_char_p, [c_int]),
    "sf_last_error": (c_char_p, []),
    "sf_version": (c_char_p, []),
}


def load(path: str = LIB_PATH):
    """Load the library (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"the CUDA library {path} is not built; run __graft_entry__.build() first")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int, where: str):
    if status != SF_OK:
        detail = _lib.sf_last_error().decode(errors="replace")
        raise SolverError(status, where, detail)


KERNEL = {"G2": 0, "G4": 1, "G6": 2, "G8": 3, "G10": 4, "SPECT": 5}


def make_desc(dim, n, lo, hi, bc, grid="staggered", eig="PS", op="NONE", sigma=0.0, ncomp=1, prec="f32",
              rhs_scale=1.0, flags=0, tune_radix=0, tune_tile=0, tune_slab=0, tune_lag=0,
              kernel="G2") -> sf_plan_desc:
    d = sf_plan_desc()
    d.dim = dim
    for a in range(3):
        d.n[a] = int(n[a]) if a < len(n) else 1
        d.lo[a] = float(lo[a]) if a < len(lo) else 0.0
        d.hi[a] = float(hi[a]) if a < len(hi) else 1.0
        b = bc[a] if a < len(bc) else "P"
        # one letter: both faces; two letters ("DN", "ND") or a pair: (lower face, upper face)
        pair = ((b, b) if len(b) == 1 else (b[0], b[1])) if isinstance(b, str) else tuple(b)
        d.bc[a][0] = BC[pair[0]]
        d.bc[a][1] = BC[pair[1]]
    d.grid = GRID[grid]
    d.eig = EIG[eig]
    d.op = OP[op]
    d.green = KERNEL[kernel]
    d.green_sigma = float(sigma)
    d.ncomp = int(ncomp)
    d.prec = PREC[prec]
    d.rhs_scale = float(rhs_scale)
    d.flags = int(flags)
    d.tune_radix = int(tune_radix)
    d.tune_tile = int(tune_tile)
    d.tune_slab = int(tune_slab)
    d.tune_lag = int(tune_lag)
    return d


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(stream)
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


# ---- thin wrappers with the C names ---------------------------------------

def sf_plan_create(desc: sf_plan_desc, stream=None) -> ctypes.c_void_p:
    lib = load()
    h = ctypes.c_void_p()
    _check(lib.sf_plan_create(ctypes.byref(h), ctypes.byref(desc), _stream(stream)), "sf_plan_create")
    return h


def sf_plan_set_stream(plan, stream):
    _check(load().sf_plan_set_stream(plan, _stream(stream)), "sf_plan_set_stream")


def sf_plan_query(plan):
    lib = load()
    a, b, c = (c_size_t * 4)(), (c_size_t * 4)(), (c_size_t * 4)()
    ws = c_size_t()
    _check(lib.sf_plan_query(plan, a, b, c, ctypes.byref(ws)), "sf_plan_query")
    return tuple(a), tuple(b), tuple(c), ws.value


def sf_set_source(plan, f):
    _check(load().sf_set_source(plan, _ptr(f)), "sf_set_source")


def sf_set_boundary(plan, axis, side, face):
    _check(load().sf_set_boundary(plan, axis, side, _ptr(face)), "sf_set_boundary")


def sf_solve(plan):
    _check(load().sf_solve(plan), "sf_solve")


def sf_get_output(plan, psi, op=None):
    _check(load().sf_get_output(plan, _ptr(psi), _ptr(op)), "sf_get_output")


def sf_execute(plan, f, psi, op=None):
    _check(load().sf_execute(plan, _ptr(f), _ptr(psi), _ptr(op)), "sf_execute")


def sf_solve_host(plan, f_host, psi_host, op_host=None):
    _check(load().sf_solve_host(plan, _ptr(f_host), _ptr(psi_host), _ptr(op_host)), "sf_solve_host")


def sf_solve_host_many(plan, f_hosts, psi_hosts, op_hosts=None):
    n = len(f_hosts)
    if len(psi_hosts) != n or (op_hosts is not None and len(op_hosts) != n):
        raise ValueError("buffer tables differ in length")
    tf = (c_void_p * n)(*[x.data_ptr() for x in f_hosts])
    tp = (c_void_p * n)(*[x.data_ptr() for x in psi_hosts])
    to = (c_void_p * n)(*[x.data_ptr() for x in op_hosts]) if op_hosts is not None else None
    _check(load().sf_solve_host_many(plan, n, tf, tp, to), "sf_solve_host_many")


def sf_solve_adjoint(plan, g_psi, g_op, g_f):
    _check(load().sf_solve_adjoint(plan, _ptr(g_psi), _ptr(g_op), _ptr(g_f)), "sf_solve_adjoint")


def sf_batch_create(plans, stream=None):
    lib = load()
    arr = (c_void_p * len(plans))(*[p.value for p in plans])
    h = ctypes.c_void_p()
    _check(lib.sf_batch_create(ctypes.byref(h), arr, len(plans), _stream(stream)), "sf_batch_create")
    return h


def sf_batch_solve(batch, fs, psis, ops=None):
    lib = load()
    n = len(fs)
    fa = (c_void_p * n)(*[t.data_ptr() for t in fs])
    pa = (c_void_p * n)(*[t.data_ptr() for t in psis])
    oa = None
    if ops is not None:
        oa = (c_void_p * n)(*[(t.data_ptr() if t is not None else None) for t in ops])
    _check(lib.sf_batch_solve(batch, fa, pa, oa), "sf_batch_solve")


def sf_sync(plan):
    _check(load().sf_sync(plan), "sf_sync")


def sf_plan_launches(plan) -> int:
    return int(load().sf_plan_launches(plan))


def sf_plan_stats(plan):
    """Per pass kind: (busy ns, dependency-wait ns, tiles) of the last executor launch."""
    out = (c_double * 24)()
    _check(load().sf_plan_stats(plan, out), "sf_plan_stats")
    return [(out[3 * k], out[3 * k + 1], int(out[3 * k + 2])) for k in range(8)]


def sf_plan_timing(plan, enable: bool):
    _check(load().sf_plan_timing(plan, 1 if enable else 0), "sf_plan_timing")


def sf_plan_kernel_ms(plan):
    """(mean ms per kernel slot, solves averaged) since timing was enabled."""
    ms = (c_double * 4)()
    ns, nsol = c_int(0), c_int(0)
    _check(load().sf_plan_kernel_ms(plan, ms, ctypes.byref(ns), ctypes.byref(nsol)), "sf_plan_kernel_ms")
    return [ms[k] for k in range(ns.value)], nsol.value


def sf_probe_fp32_fma(stream=None) -> float:
    """Measured FP32 FMA throughput of the current device (TFLOP/s)."""
    out = c_double(0.0)
    _check(load().sf_probe_fp32_fma(ctypes.byref(out), _stream(stream)), "sf_probe_fp32_fma")
    return out.value


def sf_debug_fail_alloc(after: int):
    _check(load().sf_debug_fail_alloc(int(after)), "sf_debug_fail_alloc")


def sf_debug_corrupt_guard(plan):
    _check(load().sf_debug_corrupt_guard(plan), "sf_debug_corrupt_guard")


def sf_plan_destroy(plan):
    _check(load().sf_plan_destroy(plan), "sf_plan_destroy")


def sf_solve_static(desc: sf_plan_desc, f, psi, stream=None):
    """Allocation-free solve into the library's fixed device workspace (see the header)."""
    _check(int(load().sf_solve_static(ctypes.byref(desc), _ptr(f), _ptr(psi), _stream(stream))), "sf_solve_static")


def sf_selftest_timeout(timeout_ms: int, stream=None) -> int:
    """Status of the scheduler's bounded-wait self-test (SF_ERR_TIMEOUT = -6 expected)."""
    return int(load().sf_selftest_timeout(int(timeout_ms), _stream(stream)))


def sf_eval_special(which: int, x) -> list:
    """Host evaluation of the FP64 set-up special functions (0: Si, 1: int_0^x (1 - J0)/t, 2: E1)."""
    xs = [float(v) for v in x]
    n = len(xs)
    xa = (c_double * max(n, 1))(*xs)
    out = (c_double * max(n, 1))()
    _check(load().sf_eval_special(int(which), n, xa, out), "sf_eval_special")
    return [out[i] for i in range(n)]


def sf_version() -> str:
    return load().sf_version().decode()
