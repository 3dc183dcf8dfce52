"""Benchmark: 3D unbounded vector Poisson solve (Hockney-Eastwood, G2 kernel) with curl.

Workload: lap(psi) = -omega on a 256^3 cell-centred grid of [-0.5, 0.5]^3,
3 components, doubled to 512^3 by zero padding, sigma = 2h, outputs psi and
u = curl(psi) (FP32 bulk arithmetic, FP64-built tables).  omega is a seeded
Gaussian vortex ring (radius 0.25, core 0.05, random axis).

One step = one full solve (forward transforms, Green's multiply, curl,
inverse transforms, extraction) through the C ABI on device-resident buffers.
The metric is grid points per second (256^3 output points per solve).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank solves its own copy (independent replicas,
no collective in the data path); the reported value is the total over ranks
divided by the slowest rank's time.  --impl reference times the FP64 CPU
oracle on a reduced grid of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "grid points/s per solve (3D unbounded 256^3 vector, FP32 vs FP64) and % HBM roofline"
UNIT = "grid points/s"
N = 256
NCOMP = 3
HBM_FALLBACK = 6800.0


def algorithmic_bytes(n: int, elem: int = 4):
    """Bytes per solve of the method (see the roofline model of the design notes).

    B_io:     read omega (3 fields), write psi and u (6 fields), read the Green's octant once.
    B_method: B_io plus one HBM round trip of the half-spectrum after the x
              transform (3 fields forward, 6 fields inverse): [n+1][n][n] complex each.
    """
    field = n ** 3 * elem
    green = (n + 1) ** 3 * elem
    b_io = 3 * field + 6 * field + green
    half = (n + 1) * n * n * 2 * elem
    b_method = b_io + 2 * 3 * half + 2 * 6 * half
    return b_io, b_method


# FP32 lanes per SM of Blackwell (GB300); one FMA = 2 flops.  The SM count is
# read from the device at run time.
FP32_LANES_PER_SM = 128


def transform_flops(n: int):
    """Algorithmic transform flops of the three kernels of one solve.

    Split-radix count S(L) = 4 L log2 L - 6 L + 8 per complex line of length L;
    every line of the doubled axes is pruned (half of its input zero, or half
    of its output discarded), counted as one radix-2 stage of L/2 twiddle
    products plus two half-length transforms, P(L) = 2 S(L/2) + 3 L; a real
    line counts half.  One field-direction (one 3D transform of one field)
    is n^2 real x lines + (n+1) n y lines + (n+1) L z lines, 3.42 GFLOP at
    n = 256, and a solve is 9 field-directions (3 forward, 6 inverse: psi and
    u = curl psi), whatever the kernels do to save work.  x forward: 3 x parts;
    y/z executor: 9 y and z parts; x inverse: 6 x parts.
    """
    L = 2 * n

    def S(m):
        return 4 * m * math.log2(m) - 6 * m + 8

    P = 2 * S(L // 2) + 3 * L
    x_part = n * n * P / 2
    yz_part = ((n + 1) * n + (n + 1) * L) * P
    return {"x_forward": 3 * x_part, "yz_executor": 9 * yz_part, "x_inverse": 6 * x_part}


def kernel_bytes(n: int, elem: int = 4):
    """Algorithmic HBM bytes of each kernel of one solve (FP32).

    x forward reads omega (3 n^3) and writes the x half-spectrum A
    (3 x (n+1) x n x n complex); the y/z executor reads A and the Green's
    octant ((n+1)^3 real) and writes B (6 x (n+1) x n x n complex); x inverse
    reads B and writes psi and u (6 n^3).
    """
    half = (n + 1) * n * n * 2 * elem
    field = n ** 3 * elem
    return {"x_forward": 3 * field + 3 * half,
            "yz_executor": 3 * half + (n + 1) ** 3 * elem + 6 * half,
            "x_inverse": 6 * half + 6 * field}


# dram__bytes_read.sum + dram__bytes_write.sum of one k_fyz launch of this
# workload (256^3 curl, parity-split y / z stages), from the ncu capture
# summarised in profiles/k_fyz_c3_256.md; None when the kernel has changed since.
K_FYZ_TRAFFIC_256 = 472_694_784 + 1_097_557_760


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured", float(d.get("sm_max_mhz", 2070.0))
    except Exception:
        return HBM_FALLBACK, "fallback", 2070.0


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self, t0: float, t1: float):
        if self.proc is None:
            return None
        time.sleep(0.12)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for ts, line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            rows.append((ts, parts))
        inside = [r for ts, r in rows if t0 - 0.06 <= ts <= t1 + 0.06] or [r for _, r in rows[-3:]]
        if not inside:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in inside if num(r[1]) is not None]
        mx = [num(r[2]) for r in inside if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in inside for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(inside)}


def dist_info():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x: float) -> float:
    """Maximum of a per-rank number over the job (the slowest rank's time); x when not distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float) -> float:
    """Sum of a per-rank number over the job (units processed by all ranks); x when not distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def lpt_partition(costs, nranks: int):
    """Longest-processing-time-first: each item, largest estimated cost first, goes to the least loaded rank."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    loads = [0.0] * nranks
    parts = [[] for _ in range(nranks)]
    for i in order:
        r = min(range(nranks), key=lambda k: (loads[k], k))
        parts[r].append(i)
        loads[r] += costs[i]
    return [sorted(p) for p in parts]


def problem_cost(bp) -> float:
    """Estimated cost of one batch problem: its transform points times log2 of the FFT size."""
    pts = 1
    for n in bp.n_cells:
        pts *= 2 * n if bp.bc in ("U", "D", "N") else n
    return pts * math.log2(max(pts, 2))


def c3_config(n: int, world: int, unfused: bool = False):
    return {"workload": "3D unbounded vector Poisson lap(psi) = -omega, 256^3 cell-centred on "
                        "[-0.5,0.5]^3 padded to 512^3, G2 kernel sigma=2h, outputs psi and "
                        "u = curl(psi); seeded Gaussian vortex ring",
            "grid": n, "ncomp": NCOMP, "precision": "fp32 bulk, fp64-built tables",
            "mode": "unfused passes" if unfused else "one persistent launch",
            "l2": "inputs larger than L2 (201 MB source, 403 MB outputs, 2.4 GB workspace)",
            "parallelism": f"replicas x{world}"}


def cpu_model() -> str:
    """CPU model name of this host (lscpu, else /proc/cpuinfo, else the platform string)."""
    try:
        out = subprocess.run(["lscpu"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def _single_thread():
    # one numerical thread per worker process: the pool supplies the parallelism
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"


def _oracle_solves(job):
    """Worker: `reps` oracle solves of the headline workload at n^3 (set-up untimed); returns seconds."""
    n, reps = job
    import oracle
    import workloads
    from oracle.desc import Desc
    d = Desc(3, (n,) * 3, (-0.5,) * 3, (0.5,) * 3, ("U",) * 3, True, op="CURL", ncomp=3, rhs_scale=-1.0,
             sigma=2.0 / n)
    omega = workloads.vortex_ring(n)["omega"]
    g_hat = oracle.green_hat(d)  # plan set-up (Sec. 2.4.4)
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.solve_unbounded(d, omega, g_hat)
    return time.perf_counter() - t0


class OraclePool:
    """The FP64 oracle on every host core: one single-threaded worker process per core.

    Started with the spawn method (workers share nothing with a CUDA context).
    A step is one oracle solve per worker; throughput = cores x n^3 / wall time.
    """

    def __init__(self, cores: int = 0):
        import multiprocessing as mp
        self.cores = cores or os.cpu_count() or 1
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_single_thread)

    def step_seconds(self, n: int, reps: int = 1) -> float:
        t0 = time.perf_counter()
        self.pool.map(_oracle_solves, [(n, reps)] * self.cores, chunksize=1)
        return time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def run_reference(args):
    """FP64 CPU oracle of the same workload on every host core (reduced grid)."""
    world, rank, _ = dist_info()
    if rank != 0:
        return 0
    n = args.ref_n
    pool = OraclePool()
    try:
        for _ in range(args.warmup):
            pool.step_seconds(n)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            pool.step_seconds(n)
        dt = time.perf_counter() - t0
    finally:
        pool.close()
    value = pool.cores * n ** 3 * args.steps / dt
    sample = (f"each step {pool.cores} oracle solves (one per worker process, one per host core) of the same "
              f"workload on a {n}^3 grid (padded {2 * n}^3), psi + curl, FP64; CPU {cpu_model()}; value in the "
              f"workload's unit (grid points/s)")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": c3_config(N, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(n: int, pool=None, target_s: float = 15.0):
    """The oracle on every host core: about target_s of solves at n^3 per worker."""
    own = pool is None
    pool = pool or OraclePool()
    try:
        pool.step_seconds(n)  # warm-up: imports and one solve per worker
        t1 = pool.step_seconds(n)  # calibration: one solve per worker
        reps = max(1, min(200, int(target_s / max(t1, 1e-3))))
        dt = pool.step_seconds(n, reps)
    finally:
        if own:
            pool.close()
    return {"value": pool.cores * reps * n ** 3 / dt, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
            "sample": f"{pool.cores} x {reps} oracle solve(s) of the same workload at {n}^3 (padded {2 * n}^3), "
                      f"psi + curl, FP64, one single-threaded worker process per host core, {dt:.1f} s wall; "
                      f"CPU {cpu_model()}"}


def cpu_fast_baseline(n: int, gpu_psi=None, gpu_u=None):
    """The same unbounded curl solve with scipy.fft on all host cores (FP32 and FP64).

    A fast CPU comparison beside the oracle: zero-padded real FFTs of length
    2n on every axis (the Green's table and its transform are set-up, outside
    the timed region), psi_hat = g_hat * omega_hat (g_hat = h^3 FFT of
    G(r) = erf(r / (sigma sqrt 2)) / (4 pi r), the wrap offset n taken as +n),
    u_hat = i k x psi_hat on the doubled grid's wavenumbers (Nyquist zero),
    inverse FFTs, crop to [0, n).  Its relative L2 difference from the GPU
    result is reported as a cross-check.
    """
    import numpy as np
    import scipy.fft as sfft
    import scipy.special as ssp

    import workloads

    cores = os.cpu_count() or 1
    h = 1.0 / n
    L = 2 * n
    sigma = 2.0 * h
    omega64 = workloads.vortex_ring(n)["omega"]
    d = np.arange(L, dtype=np.float64)
    d = np.where(d <= n, d, d - L) * h
    r = np.sqrt(d[:, None, None] ** 2 + d[None, :, None] ** 2 + d[None, None, :] ** 2)
    with np.errstate(invalid="ignore", divide="ignore"):
        G = ssp.erf(r / (sigma * math.sqrt(2.0))) / (4.0 * math.pi * r)
    G[0, 0, 0] = math.sqrt(2.0) / (4.0 * math.pi ** 1.5 * sigma)
    ghat64 = sfft.rfftn(G * h ** 3, workers=cores).real
    del G, r
    k = np.fft.fftfreq(L, d=2.0 / L) * 2.0 * math.pi  # period 2 (doubled unit domain)
    k[L // 2] = 0.0
    kr = np.fft.rfftfreq(L, d=2.0 / L) * 2.0 * math.pi
    kr[-1] = 0.0
    out = {"kind": "scipy.fft", "cores": cores, "sample": f"one full {n}^3 solve (padded {L}^3), psi + curl"}
    for prec, rdt in (("f32", np.float32), ("f64", np.float64)):
        om = omega64.astype(rdt)
        ghat = ghat64.astype(rdt)
        kz = k.astype(rdt)[:, None, None]
        ky = k.astype(rdt)[None, :, None]
        kx = kr.astype(rdt)[None, None, :]
        t0 = time.perf_counter()
        ph = [sfft.rfftn(om[c], s=(L, L, L), workers=cores) * ghat for c in range(3)]
        uh = [1j * (ky * ph[2] - kz * ph[1]), 1j * (kz * ph[0] - kx * ph[2]), 1j * (kx * ph[1] - ky * ph[0])]
        psi = [sfft.irfftn(a, s=(L, L, L), workers=cores)[:n, :n, :n] for a in ph]
        u = [sfft.irfftn(a, s=(L, L, L), workers=cores)[:n, :n, :n] for a in uh]
        dt = time.perf_counter() - t0
        out[prec] = {"value": n ** 3 / dt, "unit": UNIT, "ms_per_solve": dt * 1e3}
        if gpu_psi is not None and prec == "f32":
            num = sum(float(np.sum((psi[c] - gpu_psi[c]) ** 2)) for c in range(3))
            den = sum(float(np.sum(gpu_psi[c].astype(np.float64) ** 2)) for c in range(3))
            numu = sum(float(np.sum((u[c] - gpu_u[c]) ** 2)) for c in range(3))
            denu = sum(float(np.sum(gpu_u[c].astype(np.float64) ** 2)) for c in range(3))
            out["rel_l2_vs_gpu"] = {"psi": math.sqrt(num / den), "u": math.sqrt(numu / denu)}
        del ph, uh, psi, u
    return out


def cufft_context(n: int, omega, psi_ref, u_ref, steps: int = 10):
    """The same unbounded curl solve as one library call chain on this GPU (context only).

    torch.fft (cuFFT) in FP32: zero-padded real transforms of length 2n on every
    axis (the padded arrays are materialised), psi_hat = g_hat * omega_hat with
    g_hat = the real transform of h^3 G(r), G = erf(r / (sigma sqrt 2)) / (4 pi r)
    sampled on the doubled grid (offset n taken as +n; the table is set-up,
    outside the timed region), u_hat = i k x psi_hat on the doubled grid's
    wavenumbers (Nyquist zero), inverse transforms, crop to [0, n).  Timed with
    CUDA events after one warm-up; its relative L2 difference from the
    library's own result is reported as a cross-check.
    """
    import torch
    dev = omega.device
    L, h = 2 * n, 1.0 / n
    sigma = 2.0 * h
    d = torch.arange(L, dtype=torch.float64, device=dev)
    d = torch.where(d <= n, d, d - L) * h
    r = torch.sqrt(d[:, None, None] ** 2 + d[None, :, None] ** 2 + d[None, None, :] ** 2)
    G = torch.special.erf(r / (sigma * math.sqrt(2.0))) / (4.0 * math.pi * r)
    G[0, 0, 0] = math.sqrt(2.0) / (4.0 * math.pi ** 1.5 * sigma)
    ghat = torch.fft.rfftn(G * h ** 3).real.float()
    del G, r
    k = torch.fft.fftfreq(L, d=2.0 / L, device=dev, dtype=torch.float64) * 2.0 * math.pi
    k[L // 2] = 0.0
    kr = torch.fft.rfftfreq(L, d=2.0 / L, device=dev, dtype=torch.float64) * 2.0 * math.pi
    kr[-1] = 0.0
    kz, ky, kx = k.float()[:, None, None], k.float()[None, :, None], kr.float()[None, None, :]

    def solve():
        ph = [torch.fft.rfftn(omega[c], s=(L, L, L)) * ghat for c in range(3)]
        uh = [1j * (ky * ph[2] - kz * ph[1]), 1j * (kz * ph[0] - kx * ph[2]), 1j * (kx * ph[1] - ky * ph[0])]
        psi = [torch.fft.irfftn(a, s=(L, L, L))[:n, :n, :n] for a in ph]
        u = [torch.fft.irfftn(a, s=(L, L, L))[:n, :n, :n] for a in uh]
        return psi, u

    psi, u = solve()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        solve()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps

    def rel(a, b):
        num = sum(float((a[c].double() - b[c].double()).norm() ** 2) for c in range(3))
        den = sum(float(b[c].double().norm() ** 2) for c in range(3))
        return math.sqrt(num / den)

    out = {"kind": "torch.fft (cuFFT), FP32, padded arrays materialised", "ms_per_step": ms,
           "value": n ** 3 / (ms * 1e-3), "unit": UNIT, "steps": steps,
           "rel_l2_vs_library": {"psi": rel(psi, psi_ref), "u": rel(u, u_ref)}}
    del psi, u, ghat
    torch.cuda.empty_cache()
    return out


def _events_time(fn, steps, stream):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _rel_l2(got, ref):
    import numpy as np
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = float(np.linalg.norm(ref))
    return float(np.linalg.norm(got - ref)) / (den if den > 0 else 1.0)


def _batch_kwargs(bp):
    dim = bp.dim
    return dict(dim=dim, n=bp.n_cells, lo=(-0.5,) * dim, hi=(0.5,) * dim, bc=bp.bc * dim,
                grid="staggered" if bp.staggered else "regular", eig="PS",
                sigma=2.0 / max(bp.n_cells) if bp.bc == "U" else 0.0, rhs_scale=-1.0 if bp.bc == "U" else 1.0)


def config_case(name: str, world: int = 1, rank: int = 0):
    """Plans, buffers and one step of a configuration other than the headline one.

    Returns a dict: step (one step on device-resident buffers), points (output
    grid points per step), dtype, cfg (the config description), check (a
    function that compares the last step's result with the oracle and returns
    the errors), close.
    """
    import numpy as np
    import torch

    import oracle
    import paper_2301_01145_gb300 as sf
    import workloads
    from oracle.desc import Desc

    dev = lambda a, dt=torch.float32: torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    host = lambda t: t.detach().double().cpu().numpy()
    plans = []
    extra = {}
    if name == "c1":
        pm = workloads.periodic_modes(64)
        plan = sf.Plan(3, (64,) * 3, (0,) * 3, (2 * math.pi,) * 3, "PPP", eig="PS", prec="f64")
        plans.append(plan)
        f = dev(pm.f[None], torch.float64)
        psi, _ = plan.empty_outputs()
        step = lambda: plan.execute(f, psi)
        points, dtype = 64 ** 3, "f64"
        cfg = {"workload": "3D periodic scalar Poisson 64^3 cell-centred on [0,2pi)^3, pseudo-spectral, "
                           "sum of 8 seeded sine modes", "grid": 64}

        def check():
            d = Desc(3, (64,) * 3, (0,) * 3, (2 * math.pi,) * 3, ("P",) * 3, True, "PS")
            ref, _ = oracle.solve(d, pm.f[None])
            got = host(psi)[0]
            return {"psi": _rel_l2(got, ref[0]), "psi_vs_closed_form": _rel_l2(got, pm.psi_exact), "tol": 1e-12}
    elif name in ("c2", "c6"):
        n = 256
        man = workloads.manufactured(seed_index=1)
        case = workloads.bounded_case(man, (n, n, n), ("D", "N", "D"), False)
        op = "GRAD" if name == "c6" else "NONE"
        plan = sf.Plan(3, (n,) * 3, (0,) * 3, (1,) * 3, "DND", grid="regular", eig="FD2", op=op, prec="f32")
        plans.append(plan)
        for (ax, side), g in case["faces"].items():
            plan.set_boundary(ax, side, dev(g))
        f = dev(case["f"][None])
        psi, grad = plan.empty_outputs()
        step = lambda: plan.execute(f, psi, grad)
        points, dtype = n ** 3, "f32"
        if name == "c2":
            cfg = {"workload": "3D Dirichlet/Neumann/Dirichlet Poisson, 256^3 cells regular grid on the unit cube, "
                               "FD2 eigenvalues, inhomogeneous faces (manufactured sin/cos solution)", "grid": n}
        else:
            cfg = {"workload": "3D Dirichlet/Neumann/Dirichlet Poisson 256^3 regular grid, FD2, inhomogeneous "
                               "faces, plus the gradient on the bounded axes (each term formed where its axis is still spectral)",
                   "grid": n}

        def check():
            d = Desc(3, (n,) * 3, (0,) * 3, (1,) * 3, ("D", "N", "D"), False, "FD2", op=op)
            ref, ref_g = oracle.solve(d, case["f"], case["faces"])
            out = {"psi": _rel_l2(host(psi)[0], ref[0]), "tol": 1e-5}
            if grad is not None:
                g = host(grad)
                out["grad"] = max(_rel_l2(g[a], ref_g[a]) for a in range(3))
            return out
    elif name == "c7":
        rng = np.random.default_rng(7)
        kinds = ["P", "D", "N", "DN", "ND", "U"]
        fs, ps, descs = [], [], []
        for i in range(1024):
            bc = kinds[i % len(kinds)]
            n1 = int(rng.choice([256, 384, 512])) if len(bc) == 1 else int(rng.choice([128, 256]))
            grid = "staggered" if i % 2 == 0 or bc == "P" else "regular"
            kw = dict(kernel="SPECT" if bc == "U" else "G2", rhs_scale=-1.0 if bc == "U" else 1.0)
            plans.append(sf.Plan(1, (n1,), (-0.5,), (0.5,), [bc], grid=grid, eig="PS", **kw))
            fs.append(dev(rng.normal(size=plans[-1].in_shape)))
            ps.append(plans[-1].empty_outputs()[0])
            descs.append((n1, bc, grid, kw["rhs_scale"]))
        batch = sf.Batch(plans)
        extra["batch"] = batch
        step = lambda: batch.solve(fs, ps)
        points, dtype = sum(int(np.prod(p.out_shape[1:])) for p in plans), "f32"
        cfg = {"workload": "1024 uneven 1D problems (periodic, Dirichlet, Neumann, D-N, N-D, unbounded with the "
                           "1D spectral kernel; 128..512 cells; both grids) in one persistent launch",
               "problems": 1024, "points_per_step": points}

        def check():
            errs = []
            for i in range(12):  # two of each boundary kind, both grids
                n1, bc, grid, rs = descs[i]
                d = Desc(1, (n1,), (-0.5,), (0.5,), (bc,), grid == "staggered", "PS", rhs_scale=rs,
                         kernel="SPECT" if bc == "U" else "G2")
                ref, _ = oracle.solve(d, host(fs[i]))
                errs.append(_rel_l2(host(ps[i])[0], ref[0]))
            return {"psi_max_over_sample": max(errs), "sample": "12 problems, two of each boundary kind", "tol": 1e-5}
    elif name == "c5":
        from paper_2301_01145_gb300.autograd import poisson_solve
        from oracle import unbounded
        n = 128
        data = workloads.gaussian_blobs(n)
        plan = sf.Plan(3, (n,) * 3, (-0.5,) * 3, (0.5,) * 3, "UUU", op="CURL", ncomp=3, sigma=2.0 / n,
                       rhs_scale=-1.0)
        plans.append(plan)
        om = dev(data["omega"])
        w = dev(data["w"])
        last = {}

        def step():
            x = om.detach().requires_grad_(True)
            psi, u = poisson_solve(x, plan)
            L = (w[None] * u * u).sum()
            L.backward()
            last["psi"], last["u"] = psi, u

        points, dtype = n ** 3, "f32"
        cfg = {"workload": "differentiable 3D unbounded curl solve 128^3 (padded 256^3), loss sum w|u|^2, "
                           "forward + adjoint backward per step", "grid": n}

        def check():
            d = Desc(3, (n,) * 3, (-0.5,) * 3, (0.5,) * 3, ("U",) * 3, True, op="CURL", ncomp=3, rhs_scale=-1.0,
                     sigma=2.0 / n)
            rng = np.random.default_rng(3)
            pts = [tuple(int(v) for v in rng.integers(0, n, size=3)) for _ in range(12)]
            ref_psi, ref_u = unbounded.sample_points(d, data["omega"], pts)
            worst = 0.0
            for got, ref in ((host(last["psi"]), ref_psi), (host(last["u"]), ref_u)):
                for c in range(3):
                    rms = float(np.sqrt(np.mean(got[c] ** 2)))
                    for i, p in enumerate(pts):
                        worst = max(worst, abs(got[c][p[2], p[1], p[0]] - ref[i][c]) / rms)
            return {"psi_u_max_pointwise_over_rms": worst, "sample": "forward psi and u at 12 seeded points",
                    "tol": 1e-5}
    elif name == "c4":
        from paper_2301_01145_gb300 import autotune
        probs = workloads.batch_problems(512)
        total_points = sum(bp.out_points() for bp in probs)
        parallelism = None
        if world > 1:
            # independent problems: each rank solves its longest-processing-time share, no collective
            mine = lpt_partition([problem_cost(bp) for bp in probs], world)[rank]
            probs = [probs[i] for i in mine]
            parallelism = f"problem shards x{world} (LPT by estimated cost)"
        kwargs = [_batch_kwargs(bp) for bp in probs]
        knobs = autotune.batch_knobs(kwargs)
        fs, ps = [], []
        for kw, bp, kn in zip(kwargs, probs, knobs):
            plans.append(sf.Plan(**kw, **kn))
            fs.append(dev(workloads.lowpass_noise(tuple(reversed(bp.node_counts())), bp.seed)[None]))
            ps.append(plans[-1].empty_outputs()[0])
        batch = sf.Batch(plans)
        extra["batch"] = batch
        step = lambda: batch.solve(fs, ps)
        points, dtype = sum(bp.out_points() for bp in probs), "f32"
        cfg = {"workload": "512 uneven problems in one persistent launch (CUDA graph): 2D 64^2..1024^2, 3D "
                           "32^3..128^3, periodic/Dirichlet/Neumann/unbounded, regular/staggered, low-pass "
                           "N(0,1) sources", "problems": 512, "points_per_step": total_points,
               "knobs": autotune.describe_knobs(kwargs, knobs)}
        if parallelism:
            extra["parallelism"] = parallelism

        def buckets():
            # each size class (dimension, largest FFT length) of the batch timed as its own batch
            groups = {}
            for i, kw in enumerate(kwargs):
                groups.setdefault(autotune.size_class(kw), []).append(i)
            out = {}
            for cls, idx in sorted(groups.items()):
                sub = sf.Batch([plans[i] for i in idx])
                fsub, psub = [fs[i] for i in idx], [ps[i] for i in idx]
                for _ in range(3):
                    sub.solve(fsub, psub)
                ms = _events_time(lambda: sub.solve(fsub, psub), 5, torch.cuda.current_stream())
                pts = sum(probs[i].out_points() for i in idx)
                out[cls] = {"problems": len(idx), "points": pts, "ms": ms, "points_per_s": pts / (ms * 1e-3)}
                sub.close()
            return out
        extra["buckets"] = buckets

        def check():
            picked, seen = [], set()
            for i, bp in enumerate(probs):
                key = (bp.dim, bp.bc, bp.staggered)
                if key not in seen and bp.out_points() <= 300_000:
                    seen.add(key)
                    picked.append(i)
            errs = []
            for i in picked:
                kw = kwargs[i]
                dim = kw["dim"]
                d = Desc(dim, tuple(kw["n"]), kw["lo"], kw["hi"], tuple(kw["bc"]), kw["grid"] == "staggered", "PS",
                         rhs_scale=kw["rhs_scale"], sigma=kw["sigma"])
                ref, _ = oracle.solve(d, host(fs[i]))
                errs.append(_rel_l2(host(ps[i])[0], ref[0]))
            return {"psi_max_over_sample": max(errs), "sample": f"{len(picked)} problems, one per (dimension, "
                    "boundary type, grid)", "tol": 1e-5}
    else:
        raise ValueError(name)

    def close():
        if "batch" in extra:
            extra["batch"].close()
        for p in plans:
            p.close()
        torch.cuda.empty_cache()

    return {"step": step, "points": points, "dtype": dtype, "cfg": cfg, "check": check, "close": close,
            "parallelism": extra.get("parallelism"), "buckets": extra.get("buckets")}


def measure_config(name: str, steps: int, warmup: int, check: bool = True):
    """Device time of one configuration (CUDA events, after warm-up) and its oracle errors."""
    import torch
    case = config_case(name)
    try:
        for _ in range(warmup):
            case["step"]()
        torch.cuda.synchronize()
        ms = _events_time(case["step"], steps, torch.cuda.current_stream())
        out = {"workload": case["cfg"]["workload"], "ms_per_step": ms, "value": case["points"] / (ms * 1e-3),
               "unit": UNIT, "dtype": case["dtype"], "steps": steps}
        if "knobs" in case["cfg"]:
            out["knobs"] = case["cfg"]["knobs"]
        if case["buckets"]:
            out["per_class"] = case["buckets"]()
        if check:
            out["oracle"] = case["check"]()
        return out
    finally:
        case["close"]()


def run_other(args):
    """Timing line for the configurations other than the headline one."""
    import torch

    import __graft_entry__ as ge

    world, rank, local = dist_info()
    torch.cuda.set_device(local)
    if world > 1:
        torch.distributed.init_process_group("nccl")
    ge.build()
    stream = torch.cuda.current_stream()
    line = {"unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "data": "synthetic"}
    case = config_case(args.workload, world, rank)
    step, points, dtype, cfg = case["step"], case["points"], case["dtype"], case["cfg"]
    cfg["parallelism"] = case["parallelism"] or f"replicas x{world}"
    if case["parallelism"]:
        line["scaling"] = "strong"
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = max_over_ranks(_events_time(step, args.steps, stream))
    points_all = sum_over_ranks(float(points))  # units every rank processed in one step
    line.update({"metric": f"grid points/s ({args.workload})", "value": points_all / (ms * 1e-3), "ms_per_step": ms,
                 "dtype": dtype, "config": cfg})
    if rank == 0 and world == 1 and case["buckets"]:
        line["per_class"] = case["buckets"]()
    if rank == 0 and world == 1 and not args.no_cpu:
        line["oracle"] = case["check"]()
    case["close"]()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--ref-n", type=int, default=32)
    ap.add_argument("--cpu-n", type=int, default=48)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--unfused", action="store_true")
    ap.add_argument("--no-cufft", action="store_true")
    ap.add_argument("--no-others", action="store_true")
    ap.add_argument("--n", type=int, default=N)
    ap.add_argument("--workload", default="c3", choices=["c1", "c2", "c3", "c4", "c5", "c6", "c7"],
                    help="c3 (default): the headline 256^3 unbounded curl solve; the others time the remaining "
                         "configurations (64^3 periodic FP64, 256^3 mixed D/N FD2, 512-problem batch, "
                         "differentiable 128^3, 256^3 D/N FD2 with the gradient, 1024 batched 1D problems) "
                         "and print their own line")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "c3":
        return run_other(args)

    import numpy as np
    import torch

    import __graft_entry__ as ge
    import paper_2301_01145_gb300 as sf
    import workloads

    world, rank, local = dist_info()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    ge.build()
    n = args.n
    h = 1.0 / n
    ring = workloads.vortex_ring(n)
    omega = torch.tensor(ring["omega"], dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    plan = sf.Plan(3, (n,) * 3, (-0.5,) * 3, (0.5,) * 3, "UUU", op="CURL", ncomp=3, sigma=2 * h, rhs_scale=-1.0,
                   prec="f32", fused=not args.unfused)
    psi, u = plan.empty_outputs()
    for _ in range(args.warmup):
        plan.execute(omega, psi, u)
    plan.sync()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.15)
    plan.timing(True)  # CUDA events between this plan's kernels, on its launch stream
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_wall0 = time.time()
    ev0.record(stream)
    for _ in range(args.steps):
        plan.execute(omega, psi, u)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_wall1 = time.time()
    barrier()
    clocks = sampler.stop(t_wall0, t_wall1)
    plan.sync()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps)
    points = n ** 3
    value = sum_over_ranks(float(points)) / (ms * 1e-3)  # every rank solves its own replica
    launches = plan.launches() * args.steps

    kms, ksolves = plan.kernel_ms()
    plan.timing(False)
    fma_tflops = sf._lib.sf_probe_fp32_fma()  # measured FP32 FMA stream, after the timed region

    # roofline of the dominant kernel (the y/z executor, bound by FP32 issue),
    # timed per launch by the events above; the other kernels and the whole
    # step against HBM for context
    hbm_peak, peak_kind, sm_mhz = read_peaks()
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    alu_peak = n_sm * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12  # TFLOP/s
    b_io, b_method = algorithmic_bytes(n)
    kb, kf = kernel_bytes(n), transform_flops(n)
    names = ["x_forward", "yz_executor", "x_inverse"]
    kernels = {}
    if len(kms) == 3 and not args.unfused:
        for k, name in enumerate(names):
            t = kms[k] * 1e-3
            kernels[name] = {"ms": kms[k], "share": kms[k] / sum(kms), "GB/s": kb[name] / t / 1e9,
                             "hbm_frac": kb[name] / t / 1e9 / hbm_peak, "TFLOP/s": kf[name] / t / 1e12,
                             "alu_frac": kf[name] / t / 1e12 / alu_peak, "bytes": kb[name], "flops": kf[name]}
        dom = kernels["yz_executor"]
        roof = {"bound": "alu", "kernel": "k_fyz (y/z executor)", "achieved": dom["TFLOP/s"], "peak": alu_peak,
                "unit": "TFLOP/s", "frac": dom["alu_frac"],
                "traffic": K_FYZ_TRAFFIC_256 if n == 256 else None, "algorithmic_bytes": kb["yz_executor"],
                "algorithmic_flops": kf["yz_executor"],
                "peak_source": f"derived: {n_sm} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 (FMA) x {sm_mhz:.0f} MHz",
                "peak_fma_measured": fma_tflops, "frac_of_fma_measured": dom["TFLOP/s"] / fma_tflops,
                "kernels": kernels, "solves_timed": ksolves,
                "step_hbm": {"achieved": b_method / (ms * 1e-3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                             "frac": b_method / (ms * 1e-3) / 1e9 / hbm_peak, "bytes_model": "B_method",
                             "algorithmic_bytes": b_method, "b_io_bytes": b_io,
                             "b_io_frac": b_io / (ms * 1e-3) / 1e9 / hbm_peak, "peak_source": peak_kind}}
    else:
        achieved = b_method / (ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": "whole step", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": None, "bytes_model": "B_method", "algorithmic_bytes": b_method,
                "b_io_bytes": b_io, "b_io_frac": b_io / (ms * 1e-3) / 1e9 / hbm_peak, "peak_source": peak_kind}

    # end to end through the C ABI with pinned host buffers (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        hf = omega.cpu().pin_memory()
        hpsi = [torch.empty(psi.shape, dtype=psi.dtype).pin_memory() for _ in range(2)]
        hu = [torch.empty(u.shape, dtype=u.dtype).pin_memory() for _ in range(2)]
        ksteps = max(3, min(args.steps, 30))

        def host_many(k):
            plan.solve_host_many([hf] * k, [hpsi[i & 1] for i in range(k)], [hu[i & 1] for i in range(k)])

        reduce_max = max_over_ranks

        # serial: one call per step (upload, solve, download, wait)
        plan.solve_host(hf, hpsi[0], hu[0])
        barrier()
        t0 = time.perf_counter()
        for _ in range(ksteps):
            plan.solve_host(hf, hpsi[0], hu[0])
        dt_serial = reduce_max(time.perf_counter() - t0)
        # pipelined: the next step's upload and the previous step's download overlap each solve
        host_many(3)
        barrier()
        t0 = time.perf_counter()
        host_many(ksteps)
        dt = reduce_max(time.perf_counter() - t0)
        e2e = {"value": sum_over_ranks(float(points)) * ksteps / dt, "unit": UNIT, "h2d_bytes_per_step": hf.numel() * 4,
               "d2h_bytes_per_step": (hpsi[0].numel() + hu[0].numel()) * 4, "steps": ksteps,
               "mode": "sf_solve_host_many: pinned host buffers, every step uploads its source and downloads "
                       "psi and u; copies of neighbouring steps overlap the solve",
               "serial": {"value": sum_over_ranks(float(points)) * ksteps / dt_serial, "unit": UNIT,
                          "mode": "sf_solve_host per step (upload, solve, download, wait)"}}

    # FP64 plain GPU solve of the same workload (comparison the metric names)
    fp64 = None
    if not args.no_fp64:
        p64 = sf.Plan(3, (n,) * 3, (-0.5,) * 3, (0.5,) * 3, "UUU", op="CURL", ncomp=3, sigma=2 * h, rhs_scale=-1.0,
                      prec="f64")
        o64 = omega.double()
        psi64, u64 = p64.empty_outputs()
        p64.execute(o64, psi64, u64)
        p64.sync()
        k64 = 5
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k64):
            p64.execute(o64, psi64, u64)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1) / k64
        rel = float(((psi.double() - psi64).norm() / psi64.norm()).item())
        relu = float(((u.double() - u64).norm() / u64.norm()).item())
        fp64 = {"value": points / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64,
                "f32_rel_l2_vs_f64": {"psi": rel, "u": relu}}
        p64.close()

    # the same solve as a cuFFT library call chain on this GPU (context for the hand-written transforms)
    ctx = None
    if rank == 0 and not args.no_cufft:
        try:
            ctx = cufft_context(n, omega, psi, u)
        except Exception as exc:  # noqa: BLE001 - reported, not fatal
            ctx = {"unavailable": f"{type(exc).__name__}: {exc}"}

    cpu = cpu_fast = None
    psi_h, u_h = psi.cpu().numpy(), u.cpu().numpy()
    plan.close()
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(args.cpu_n)
        try:
            cpu_fast = cpu_fast_baseline(n, psi_h, u_h)
        except ImportError as exc:  # scipy missing on the host
            cpu_fast = {"unavailable": str(exc)}

    # the other configurations: device time and errors against the oracle
    others = None
    if rank == 0 and world == 1 and not args.no_others:
        others = {}
        for name in ("c1", "c2", "c4", "c5", "c6", "c7"):
            try:
                others[name] = measure_config(name, steps=10, warmup=3, check=not args.no_cpu)
            except Exception as exc:  # noqa: BLE001 - reported per configuration
                others[name] = {"error": f"{type(exc).__name__}: {exc}"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": c3_config(n, world, args.unfused),
                "gpu_launches": launches, "roofline": roof, "clocks": clocks, "e2e": e2e, "fp64": fp64,
                "cpu_baseline": cpu, "cpu_fast": cpu_fast, "cufft_context": ctx, "other_configs": others}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
