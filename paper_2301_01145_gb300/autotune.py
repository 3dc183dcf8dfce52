"""Autotuner for radix, tile (pencil) and slab choices.

A configuration is the set of tuning knobs of sf_plan_desc (tune_radix,
tune_tile, tune_slab) plus the execution mode (one persistent launch or one
launch per pass).  The tuner builds a plan per candidate, times a few solves
with CUDA events on the current stream and keeps the fastest.  Results are
cached in a JSON file keyed by the problem description, so a later run with
the same problem reuses the choice without timing.

    best = autotune(dict(dim=3, n=(256,)*3, lo=..., hi=..., bc="UUU", op="CURL", ncomp=3, sigma=..., rhs_scale=-1))
    plan = Plan(**problem, **best)

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
