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


# FP32 lanes per SM and SM count of a GB300 (Blackwell Ultra); one FMA = 2 flops
FP32_LANES_PER_SM = 128
N_SM = 152


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
# workload (256^3 curl, split z stage), from the ncu capture summarised in
# profiles/k_fyz_c3_256.md; None when the kernel has changed since.
K_FYZ_TRAFFIC_256 = 474_517_504 + 987_640_832


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


def run_reference(args):
    """FP64 CPU oracle on a reduced grid of the same workload (host cores)."""
    world, rank, _ = dist_info()
    if rank != 0:
        return 0
    import numpy as np

    import oracle
    import workloads
    from oracle.desc import Desc

    n = args.ref_n
    d = Desc(3, (n,) * 3, (-0.5,) * 3, (0.5,) * 3, ("U",) * 3, True, op="CURL", ncomp=3, rhs_scale=-1.0,
             sigma=2.0 / n)
    omega = workloads.vortex_ring(n)["omega"]
    g_hat = oracle.green_hat(d)  # plan set-up, outside the timed region (Sec. 2.4.4)
    for _ in range(args.warmup):
        oracle.solve_unbounded(d, omega, g_hat)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.solve_unbounded(d, omega, g_hat)
    dt = time.perf_counter() - t0
    value = n ** 3 * args.steps / dt
    sample = (f"each step one oracle solve of the same workload on a {n}^3 grid (padded {2 * n}^3), psi + curl, "
              f"FP64, one single-threaded process; value in the workload's unit (grid points/s)")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": c3_config(N, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(n: int):
    import numpy as np

    import oracle
    import workloads
    from oracle.desc import Desc

    d = Desc(3, (n,) * 3, (-0.5,) * 3, (0.5,) * 3, ("U",) * 3, True, op="CURL", ncomp=3, rhs_scale=-1.0,
             sigma=2.0 / n)
    omega = workloads.vortex_ring(n)["omega"]
    g_hat = oracle.green_hat(d)
    reps = 0
    t0 = time.perf_counter()
    while True:
        oracle.solve_unbounded(d, omega, g_hat)
        reps += 1
        el = time.perf_counter() - t0
        if (el > 10.0 and reps >= 3) or reps >= 100:
            break
    dt = time.perf_counter() - t0
    return {"value": n ** 3 * reps / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{reps} oracle solve(s) of the same workload at {n}^3 (padded {2 * n}^3), psi + curl, "
                      f"FP64, single-threaded numpy, {dt:.1f} s"}


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


def run_other(args):
    """Timing line for the configurations other than the headline one."""
    import numpy as np
    import torch

    import __graft_entry__ as ge
    import paper_2301_01145_gb300 as sf
    import workloads

    world, rank, local = dist_info()
    torch.cuda.set_device(local)
    if world > 1:
        torch.distributed.init_process_group("nccl")
    ge.build()
    stream = torch.cuda.current_stream()
    dev = lambda a, dt=torch.float32: torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    line = {"unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "data": "synthetic"}
    parallelism = f"replicas x{world}"
    if args.workload == "c1":
        pm = workloads.periodic_modes(64)
        plan = sf.Plan(3, (64,) * 3, (0,) * 3, (2 * math.pi,) * 3, "PPP", eig="PS", prec="f64")
        f = dev(pm.f[None], torch.float64)
        psi, _ = plan.empty_outputs()
        step = lambda: plan.execute(f, psi)
        points, dtype = 64 ** 3, "f64"
        cfg = {"workload": "3D periodic scalar Poisson 64^3 cell-centred on [0,2pi)^3, pseudo-spectral, "
                           "sum of 8 seeded sine modes", "grid": 64}
    elif args.workload == "c2":
        n = 256
        man = workloads.manufactured(seed_index=1)
        case = workloads.bounded_case(man, (n, n, n), ("D", "N", "D"), False)
        plan = sf.Plan(3, (n,) * 3, (0,) * 3, (1,) * 3, "DND", grid="regular", eig="FD2", prec="f32")
        faces = {k: dev(v) for k, v in case["faces"].items()}
        for (ax, side), g in faces.items():
            plan.set_boundary(ax, side, g)
        f = dev(case["f"][None])
        psi, _ = plan.empty_outputs()
        step = lambda: plan.execute(f, psi)
        points, dtype = n ** 3, "f32"
        cfg = {"workload": "3D Dirichlet/Neumann/Dirichlet Poisson, 256^3 cells regular grid on the unit cube, "
                           "FD2 eigenvalues, inhomogeneous faces (manufactured sin/cos solution)", "grid": n}
    elif args.workload == "c6":
        n = 256
        man = workloads.manufactured(seed_index=1)
        case = workloads.bounded_case(man, (n, n, n), ("D", "N", "D"), False)
        plan = sf.Plan(3, (n,) * 3, (0,) * 3, (1,) * 3, "DND", grid="regular", eig="FD2", op="GRAD", prec="f32")
        for (ax, side), g in case["faces"].items():
            plan.set_boundary(ax, side, dev(g))
        f = dev(case["f"][None])
        psi, grad = plan.empty_outputs()
        step = lambda: plan.execute(f, psi, grad)
        points, dtype = n ** 3, "f32"
        cfg = {"workload": "3D Dirichlet/Neumann/Dirichlet Poisson 256^3 regular grid, FD2, inhomogeneous faces, "
                           "plus the gradient on the bounded axes (three derivative passes over psi)", "grid": n}
    elif args.workload == "c7":
        rng = np.random.default_rng(7)
        kinds = ["P", "D", "N", "DN", "ND", "U"]
        plans, fs, ps = [], [], []
        for i in range(1024):
            bc = kinds[i % len(kinds)]
            n1 = int(rng.choice([256, 384, 512])) if len(bc) == 1 else int(rng.choice([128, 256]))
            grid = "staggered" if i % 2 == 0 or bc == "P" else "regular"
            plans.append(sf.Plan(1, (n1,), (-0.5,), (0.5,), [bc], grid=grid, eig="PS",
                                 kernel="SPECT" if bc == "U" else "G2", rhs_scale=-1.0 if bc == "U" else 1.0))
            fs.append(dev(rng.normal(size=plans[-1].in_shape)))
            ps.append(plans[-1].empty_outputs()[0])
        batch = sf.Batch(plans)
        step = lambda: batch.solve(fs, ps)
        points, dtype = sum(int(np.prod(p.out_shape[1:])) for p in plans), "f32"
        cfg = {"workload": "1024 uneven 1D problems (periodic, Dirichlet, Neumann, D-N, N-D, unbounded with the "
                           "1D spectral kernel; 128..512 cells; both grids) in one persistent launch",
               "problems": 1024, "points_per_step": points}
    elif args.workload == "c5":
        from paper_2301_01145_gb300.autograd import poisson_solve
        n = 128
        data = workloads.gaussian_blobs(n)
        plan = sf.Plan(3, (n,) * 3, (-0.5,) * 3, (0.5,) * 3, "UUU", op="CURL", ncomp=3, sigma=2.0 / n,
                       rhs_scale=-1.0)
        om = dev(data["omega"])
        w = dev(data["w"])

        def step():
            x = om.detach().requires_grad_(True)
            psi, u = poisson_solve(x, plan)
            L = (w[None] * u * u).sum()
            L.backward()

        points, dtype = n ** 3, "f32"
        cfg = {"workload": "differentiable 3D unbounded curl solve 128^3 (padded 256^3), loss sum w|u|^2, "
                           "forward + adjoint backward per step", "grid": n}
    else:  # c4
        probs = workloads.batch_problems(512)
        total_points = sum(bp.out_points() for bp in probs)
        if world > 1:
            # independent problems: each rank solves its longest-processing-time share, no collective
            mine = lpt_partition([problem_cost(bp) for bp in probs], world)[rank]
            probs = [probs[i] for i in mine]
            parallelism = f"problem shards x{world} (LPT by estimated cost)"
            line["scaling"] = "strong"
        plans, fs, ps = [], [], []
        for bp in probs:
            dim = bp.dim
            plans.append(sf.Plan(dim, bp.n_cells, (-0.5,) * dim, (0.5,) * dim, bp.bc * dim,
                                 grid="staggered" if bp.staggered else "regular", eig="PS",
                                 sigma=2.0 / max(bp.n_cells) if bp.bc == "U" else 0.0,
                                 rhs_scale=-1.0 if bp.bc == "U" else 1.0, generic=True))
            fs.append(dev(workloads.lowpass_noise(tuple(reversed(bp.node_counts())), bp.seed)[None]))
            ps.append(plans[-1].empty_outputs()[0])
        batch = sf.Batch(plans)
        step = lambda: batch.solve(fs, ps)
        points, dtype = sum(bp.out_points() for bp in probs), "f32"
        cfg = {"workload": "512 uneven problems in one persistent launch (CUDA graph): 2D 64^2..1024^2, 3D "
                           "32^3..128^3, periodic/Dirichlet/Neumann/unbounded, regular/staggered, low-pass "
                           "N(0,1) sources", "problems": 512, "points_per_step": total_points}
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = max_over_ranks(_events_time(step, args.steps, stream))
    points_all = sum_over_ranks(float(points))  # units every rank processed in one step
    cfg["parallelism"] = parallelism
    line.update({"metric": f"grid points/s ({args.workload})", "value": points_all / (ms * 1e-3), "ms_per_step": ms,
                 "dtype": dtype, "config": cfg})
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
    ap.add_argument("--ref-n", type=int, default=24)
    ap.add_argument("--cpu-n", type=int, default=48)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--unfused", action="store_true")
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
    alu_peak = N_SM * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12  # TFLOP/s
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
                "peak_source": f"derived: {N_SM} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 (FMA) x {sm_mhz:.0f} MHz",
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

    cpu = cpu_fast = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(args.cpu_n)
        try:
            cpu_fast = cpu_fast_baseline(n, psi.cpu().numpy(), u.cpu().numpy())
        except ImportError as exc:  # scipy missing on the host
            cpu_fast = {"unavailable": str(exc)}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": c3_config(n, world, args.unfused),
                "gpu_launches": launches, "roofline": roof, "clocks": clocks, "e2e": e2e, "fp64": fp64,
                "cpu_baseline": cpu, "cpu_fast": cpu_fast}
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
