"""Host-side checks of the C ABI: the library builds, loads without a GPU and
exports every entry point declared in include/*.h; the Python binding's
descriptor layout matches the header; argument errors are reported without
touching a device."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2301_01145_gb300 import _lib
    return _lib.load()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_\s\*]*?\b(sf_[a-z0-9_]+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sf_plan_create", "sf_set_source", "sf_set_boundary", "sf_solve", "sf_get_output",
                     "sf_solve_adjoint", "sf_batch_create", "sf_batch_solve", "sf_plan_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    from paper_2301_01145_gb300 import _lib
    assert set(declared_functions()) <= set(_lib.SIGNATURES)


def test_descriptor_layout_matches_header(tmp_path):
    # offsets and size of sf_plan_desc as the C compiler lays it out vs the ctypes mirror
    import shutil
    import subprocess
    from paper_2301_01145_gb300._lib import sf_plan_desc
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = [f for f, _ in sf_plan_desc._fields_]
    src = tmp_path / "layout.c"
    body = "".join(f'printf("%zu\\n", offsetof(sf_plan_desc, {f}));' for f in fields)
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "sailfish_gb300.h"\n'
                   'int main(void){' + body + 'printf("%zu\\n", sizeof(sf_plan_desc)); return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert out[:-1] == [getattr(sf_plan_desc, f).offset for f in fields]
    assert out[-1] == ctypes.sizeof(sf_plan_desc)


def test_status_strings_and_version(lib):
    assert lib.sf_status_string(0) == b"SF_OK"
    assert lib.sf_status_string(-6) == b"SF_ERR_TIMEOUT"
    assert lib.sf_version().startswith(b"sailfish-gb300")


@pytest.mark.parametrize("mutate,expect", [
    (dict(dim=4), -1),
    (dict(ncomp=0), -1),
    (dict(n=(10, 10, 10)), -2),        # FFT length 20 is not 2^p or 3*2^p
    (dict(bc=("P", "D", "P")), -2),    # periodic mixed with Dirichlet
    (dict(bc=(("D", "P"), "D", "D")), -2),  # unequal faces other than a Dirichlet / Neumann pair
    (dict(bc=(("U", "N"), "D", "D")), -2),
    (dict(bc=(("D", "N"), "P", "P")), -2),  # a Dirichlet / Neumann axis mixed with periodic axes
    (dict(rhs_scale=0.0), -1),
    (dict(bc="UUU", grid="regular", n=(1100, 16, 16)), -2),  # regular unbounded: pad 2n+1 > 2048
    (dict(bc="UUU", sigma=0.0), -1),
    (dict(op="CURL", ncomp=1), -1),
    (dict(op="CURL", bc="DDD", ncomp=1), -1),  # curl in 3D needs three components
    (dict(tune_radix=3), -1),
    (dict(tune_tile=3), -1),
    (dict(tune_slab=-1), -1),
    (dict(tune_lag=9), -1),
    (dict(n=(0, 16, 16)), -1),         # empty axis
    (dict(n=(16, -4, 16)), -1),        # negative size
    (dict(n=(1, 16, 16)), -1),         # one cell
    (dict(n=(2, 16, 16), bc="DDD", grid="regular"), -1),  # regular Dirichlet needs >= 3 cells
    (dict(n=(4096, 16, 16)), -2),      # FFT length above 2048
    (dict(n=(2, 16, 16)), -2),         # periodic FFT length 2 is below 4
    (dict(n=(17, 16, 16)), -2),        # odd periodic x length
    (dict(dim=2, bc="UD"), -2),        # unbounded mixed with a Dirichlet axis
    (dict(dim=1, bc="U", kernel="G2", sigma=0.1), -2),  # 1D unbounded: the spectral kernel only
    (dict(dim=1, op="CURL", ncomp=1), -1),       # no curl in 1D
    (dict(dim=0), -1),
    (dict(bc="UUU", sigma=0.0, kernel="G6"), -1),  # Gaussian kernels need sigma > 0
    (dict(bc="UUU", sigma=float("inf")), -1),    # ... and finite
    (dict(hi=(float("inf"), 1, 1)), -1),         # infinite extent
    (dict(lo=(-1.7e308, 0, 0), hi=(1.7e308, 1, 1)), -1),  # extent overflows
    (dict(lo=(float("nan"), 0, 0)), -1),
    (dict(n=(1 << 30, 16, 16), bc="UUU", grid="regular"), -2),  # huge n rejected before 2n + 1 is formed
    (dict(n=(1 << 29, 16, 16), bc=(("D", "N"), "D", "D")), -2),  # ... and before 4n
    (dict(flags=8), -1),                         # unknown flag bit
])
def test_descriptor_validation_without_gpu(lib, mutate, expect):
    from paper_2301_01145_gb300 import _lib
    args = dict(dim=3, n=(16, 16, 16), lo=(0, 0, 0), hi=(1, 1, 1), bc="PPP", grid="staggered", eig="PS",
                op="NONE", sigma=0.1, ncomp=1, prec="f32", rhs_scale=1.0)
    args.update(mutate)
    bc = args.pop("bc")
    bc = list(bc) if isinstance(bc, str) else list(bc)
    d = _lib.make_desc(args.pop("dim"), args.pop("n"), args.pop("lo"), args.pop("hi"), bc, **args)
    h = ctypes.c_void_p()
    st = lib.sf_plan_create(ctypes.byref(h), ctypes.byref(d), None)
    assert st == expect, lib.sf_last_error()
    assert not h.value
    assert lib.sf_last_error()


def test_null_arguments(lib):
    assert lib.sf_plan_create(None, None, None) == -1
    assert lib.sf_solve(None) == -1
    assert lib.sf_plan_destroy(None) == 0


def test_descriptor_fuzz_without_gpu(lib):
    # seeded random descriptors, most of them invalid: every call returns a defined
    # status and no handle (validation rejects, or the valid ones fail at the first
    # CUDA call on a host without a GPU); none crashes or hangs the host
    from paper_2301_01145_gb300 import _lib
    rng = np.random.default_rng(2301)
    specials = [0.0, -1.0, 1.0, 1e-300, 1e300, float("inf"), float("-inf"), float("nan")]
    nvals = [-5, 0, 1, 2, 3, 4, 6, 8, 12, 16, 24, 31, 32, 64, 127, 128, 256, 512, 1024, 1025, 2048, 4096,
             1 << 29, (1 << 31) - 1, -(1 << 31)]
    seen = set()
    for _ in range(3000):
        d = _lib.sf_plan_desc()
        d.dim = int(rng.choice([-1, 0, 1, 2, 3, 4, 3, 3, 2]))
        for a in range(3):
            d.n[a] = int(rng.choice(nvals))
            d.lo[a] = float(rng.choice(specials)) if rng.random() < 0.2 else 0.0
            d.hi[a] = float(rng.choice(specials)) if rng.random() < 0.2 else 1.0
            f0 = int(rng.integers(-1, 6))
            d.bc[a][0] = f0
            d.bc[a][1] = f0 if rng.random() < 0.7 else int(rng.integers(-1, 6))
        d.grid = int(rng.integers(-1, 3))
        d.eig = int(rng.integers(-1, 3))
        d.op = int(rng.integers(-1, 7))
        d.green = int(rng.integers(-1, 8))
        d.green_sigma = float(rng.choice(specials + [0.05]))
        d.ncomp = int(rng.integers(-1, 5))
        d.prec = int(rng.integers(-1, 3))
        d.rhs_scale = float(rng.choice(specials))
        d.flags = int(rng.choice([0, 1, 2, 3, 4, 7, 8, 1 << 31]))
        d.tune_radix = int(rng.choice([0, 2, 3, 4, 16, 32]))
        d.tune_tile = int(rng.choice([0, 1, 3, 8, 32]))
        d.tune_slab = int(rng.choice([-1, 0, 1, 2, 1 << 30]))
        d.tune_lag = int(rng.choice([-1, 0, 1, 8, 9]))
        h = ctypes.c_void_p()
        st = lib.sf_plan_create(ctypes.byref(h), ctypes.byref(d), None)
        assert st in (-1, -2, -3, -4), st
        assert not h.value
        assert lib.sf_last_error()
        seen.add(st)
    assert {-1, -2} <= seen


def test_setup_special_functions_match_independent_implementations(lib):
    # the FP64 special functions that plan set-up runs on the GPU to tabulate the
    # kernels, evaluated on the host through the ABI: Si and E1 against scipy, and
    # F(x) = int_0^x (1 - J0)/t dt (2D spectral kernel) against the oracle's
    # quadrature, across both branches of each (series / continued fraction,
    # double-double series / asymptotic expansion at x = 40)
    from scipy import special
    from oracle import green
    from paper_2301_01145_gb300 import _lib
    x = np.concatenate([np.linspace(0.0, 60.0, 601), [39.999, 40.0, 40.001, 123.4, 777.7, 2345.6, 9000.0]])
    si = np.array(_lib.sf_eval_special(0, x))
    np.testing.assert_allclose(si, special.sici(x)[0], rtol=2e-15, atol=1e-300)
    F = np.array(_lib.sf_eval_special(1, x))
    ref = green.int_one_minus_j0(x)
    np.testing.assert_allclose(F, ref, rtol=1e-14, atol=1e-18)
    xe = x[x > 0]
    e1 = np.array(_lib.sf_eval_special(2, xe))
    np.testing.assert_allclose(e1, special.exp1(xe), rtol=1e-14, atol=1e-300)
    with pytest.raises(_lib.SolverError):
        _lib.sf_eval_special(7, [1.0])
