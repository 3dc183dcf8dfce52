"""Autotuner for radix, tile (pencil) and slab choices.

A configuration is the set of tuning knobs of sf_plan_desc (tune_radix,
tune_tile, tune_slab) plus the execution mode (one persistent launch or one
launch per pass).  The tuner builds a plan per candidate, times a few solves
with CUDA events on the current stream and keeps the fastest.  Results are
cached in a JSON file keyed by the problem description, so a later run with
the same problem reuses the choice without timing.

    best = autotune(dict(dim=3, n=(256,)*3, lo=..., hi=..., bc="UUU", op="CURL", ncomp=3, sigma=..., rhs_scale=-1))
    plan = Plan(**problem, **best)

For a batch of uneven problems, batch_knobs() groups the problems into size
classes (dimension, boundary types, largest FFT length), times the radix
choices on a small batch of each class and one tile cap for the whole batch
(the batch's executor uses a single cap), and returns the knobs per problem.

The cache lives at $SF_TUNE_CACHE, or ~/.cache/sailfish_gb300/tune.json.
"""
from __future__ import annotations

import itertools
import json
import os
from typing import Dict, Iterable, List, Optional

from . import Batch, Plan

KNOBS = ("tune_radix", "tune_tile", "tune_slab", "tune_lag", "fused")


def cache_path() -> str:
    return os.environ.get("SF_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "sailfish_gb300",
                                                        "tune.json"))


def _key(problem: Dict) -> str:
    items = {k: (list(v) if isinstance(v, (tuple, list)) else v) for k, v in sorted(problem.items())}
    return json.dumps(items, sort_keys=True)


def _load() -> Dict:
    try:
        with open(cache_path()) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(db: Dict) -> None:
    path = cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(db, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def candidates(problem: Dict) -> List[Dict]:
    """Knob settings worth timing for this problem."""
    cands = [dict(tune_radix=0, tune_tile=0, tune_slab=0, fused=True)]
    for r, t in itertools.product((16, 8, 4), (16, 8, 4)):
        cands.append(dict(tune_radix=r, tune_tile=t, tune_slab=0, fused=True))
    for sl, lag in itertools.product((1, 2, 3, 4, 8), (1, 2)):
        cands.append(dict(tune_radix=0, tune_tile=0, tune_slab=sl, tune_lag=lag, fused=True))
    cands.append(dict(tune_radix=0, tune_tile=0, tune_slab=0, fused=False))
    uniq, seen = [], set()
    for c in cands:
        k = json.dumps(c, sort_keys=True)
        if k not in seen:
            seen.add(k)
            uniq.append(c)
    return uniq


def _time(fn, reps: int) -> float:
    import torch
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def autotune(problem: Dict, reps: int = 3, cands: Optional[Iterable[Dict]] = None, use_cache: bool = True) -> Dict:
    """Best knob setting for a single plan (timed on random sources)."""
    import torch
    db = _load() if use_cache else {}
    key = "plan:" + _key(problem)
    if use_cache and key in db:
        return db[key]["best"]
    best, best_ms, results = None, float("inf"), []
    for c in (cands or candidates(problem)):
        try:
            plan = Plan(**problem, **c)
        except Exception:
            continue
        f = torch.randn(plan.in_shape, dtype=plan.dtype, device="cuda")
        psi, opo = plan.empty_outputs()
        ms = _time(lambda: plan.execute(f, psi, opo), reps)
        plan.sync()
        plan.close()
        results.append((c, ms))
        if ms < best_ms:
            best, best_ms = c, ms
    if use_cache and best is not None:
        db[key] = {"best": best, "ms": best_ms, "tried": len(results)}
        _store(db)
    return best


def autotune_batch(problems: List[Dict], reps: int = 2, use_cache: bool = True) -> Dict:
    """Best (radix, tile) setting for a batch of problems solved in one launch."""
    import torch
    db = _load() if use_cache else {}
    key = "batch:" + _key({"problems": [_key(p) for p in problems]})
    if use_cache and key in db:
        return db[key]["best"]
    best, best_ms = None, float("inf")
    for r, t in itertools.product((16, 8), (16, 8, 4)):
        knobs = dict(tune_radix=r, tune_tile=t)
        plans = [Plan(**p, **knobs, generic=True) for p in problems]
        fs = [torch.randn(pl.in_shape, dtype=pl.dtype, device="cuda") for pl in plans]
        ps = [pl.empty_outputs()[0] for pl in plans]
        batch = Batch(plans)
        ms = _time(lambda: batch.solve(fs, ps), reps)
        batch.sync()
        batch.close()
        for pl in plans:
            pl.close()
        if ms < best_ms:
            best, best_ms = knobs, ms
    if use_cache:
        db[key] = {"best": best, "ms": best_ms}
        _store(db)
    return best


def _fft_len(bc: str, n: int, grid: str) -> int:
    """FFT length of one axis (periodic N, Dirichlet/Neumann 2N, unbounded the padded 2N or more)."""
    if bc == "P":
        return n
    if bc == "U" and grid != "staggered":
        m, best = 2 * n + 1, None
        for base in (1, 3):
            v = base
            while v < m:
                v *= 2
            best = v if best is None else min(best, v)
        return best
    return 2 * n


def size_class(problem: Dict) -> str:
    """Class key of a problem for batch tuning: dimension and the power-of-two bucket of its largest FFT length."""
    dim = problem["dim"]
    bc = problem["bc"]
    bcs = list(bc) if isinstance(bc, str) else list(bc)
    grid = problem.get("grid", "staggered")
    lmax = max(_fft_len(bcs[a], problem["n"][a], grid) for a in range(dim))
    bucket = 256
    while bucket < lmax:
        bucket *= 2
    return f"{dim}D-L{bucket}"


def batch_knobs(problems: List[Dict], reps: int = 2, per_class: int = 6, use_cache: bool = True) -> List[Dict]:
    """Knobs (tune_radix per size class, one tile cap for the batch) for a batch of plans.

    Classes are (dimension, largest FFT length rounded up to a power of two).
    Each class is timed on a small batch of up to per_class of its problems
    for every (radix, tile) pair; the radix with the best time at its best
    tile is kept per class, and the tile cap that minimises the class times
    weighted by class size is used for the whole batch.  Batches run the
    general engine, so every plan is built with generic=True.
    """
    import torch
    db = _load() if use_cache else {}
    key = "batchclasses:" + _key({"problems": [_key(p) for p in problems]})
    if use_cache and key in db:
        choice = db[key]
    else:
        classes: Dict[str, List[int]] = {}
        for i, p in enumerate(problems):
            classes.setdefault(size_class(p), []).append(i)
        radices, tiles = (16, 8), (16, 8)
        times: Dict[str, Dict[str, float]] = {}
        for cls, idx in classes.items():
            sample = [problems[i] for i in idx[:per_class]]
            times[cls] = {}
            for r, t in itertools.product(radices, tiles):
                try:
                    plans = [Plan(**p, tune_radix=r, tune_tile=t, generic=True) for p in sample]
                except Exception:
                    continue
                fs = [torch.randn(pl.in_shape, dtype=pl.dtype, device="cuda") for pl in plans]
                ps = [pl.empty_outputs()[0] for pl in plans]
                batch = Batch(plans)
                ms = _time(lambda: batch.solve(fs, ps), reps)
                batch.sync()
                batch.close()
                for pl in plans:
                    pl.close()
                times[cls][f"{r},{t}"] = ms * len(idx) / len(sample)
        radix = {}
        for cls, tt in times.items():
            best = min(tt.items(), key=lambda kv: kv[1])[0] if tt else "0,0"
            radix[cls] = int(best.split(",")[0])
        tile_cost = {}
        for t in tiles:
            tot = 0.0
            for cls, tt in times.items():
                tot += tt.get(f"{radix[cls]},{t}", min(tt.values()) if tt else 0.0)
            tile_cost[t] = tot
        tile = min(tile_cost.items(), key=lambda kv: kv[1])[0]
        choice = {"radix": radix, "tile": tile, "classes": len(classes)}
        if use_cache:
            db[key] = choice
            _store(db)
    return [dict(tune_radix=choice["radix"].get(size_class(p), 0), tune_tile=choice["tile"], generic=True)
            for p in problems]


def describe_knobs(problems: List[Dict], knobs: List[Dict]) -> Dict:
    """Compact summary of batch knobs: the tile cap and the radix chosen per size class."""
    per_class = {}
    for p, k in zip(problems, knobs):
        per_class[size_class(p)] = k["tune_radix"]
    return {"tile": knobs[0]["tune_tile"] if knobs else 0, "radix_per_class": per_class,
            "classes": len(per_class)}
