"""The autotuner on the GPU: it returns one of its candidates, caches the
choice (a second call times nothing), and the tuned plans compute what the
default plans compute.  The cache is a file under the test's tmp_path.
"""
import json

import numpy as np
import pytest

from tests.gpu_helpers import rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built(gpu_available):
    import __graft_entry__ as g
    g.build()


@pytest.fixture()
def cache(tmp_path, monkeypatch):
    path = tmp_path / "tune.json"
    monkeypatch.setenv("SF_TUNE_CACHE", str(path))
    return path


PROBLEM = dict(dim=3, n=(64, 64, 64), lo=(-0.5,) * 3, hi=(0.5,) * 3, bc="UUU", op="CURL", ncomp=3,
               sigma=2.0 / 64, rhs_scale=-1.0)


def _outputs(plan, f):
    out = plan(f)
    plan.sync()
    return [to_np(o) for o in (out if isinstance(out, tuple) else (out,))]


def test_autotune_picks_a_candidate_caches_it_and_matches_the_default(cache, monkeypatch):
    import paper_2301_01145_gb300 as sf
    from paper_2301_01145_gb300 import autotune
    cands = autotune.candidates(PROBLEM)[:6]
    best = autotune.autotune(PROBLEM, reps=2, cands=cands)
    assert best in cands
    db = json.loads(cache.read_text())
    assert any(k.startswith("plan:") and v["best"] == best for k, v in db.items())
    # the cached choice is returned without timing anything
    monkeypatch.setattr(autotune, "_time", lambda *a, **k: pytest.fail("timed a cached problem"))
    assert autotune.autotune(PROBLEM, reps=2, cands=cands) == best
    f = to_dev(np.random.default_rng(3).normal(size=(3, 64, 64, 64)), "f32")
    base = sf.Plan(**PROBLEM)
    tuned = sf.Plan(**PROBLEM, **best)
    for a, b in zip(_outputs(base, f), _outputs(tuned, f)):
        for c in range(a.shape[0]):
            assert rel_l2(b[c], a[c]) <= 1e-5
    base.close()
    tuned.close()


def test_batch_knobs_per_size_class_match_single_solves(cache):
    import torch
    import paper_2301_01145_gb300 as sf
    from paper_2301_01145_gb300 import autotune
    problems = [dict(dim=2, n=(96, 64), lo=(0.0, 0.0), hi=(1.0, 1.0), bc="PP"),
                dict(dim=2, n=(384, 256), lo=(0.0, 0.0), hi=(1.0, 1.0), bc="DN"),
                dict(dim=3, n=(32, 32, 32), lo=(0.0,) * 3, hi=(1.0,) * 3, bc="NNN"),
                dict(dim=3, n=(24, 48, 32), lo=(-0.5,) * 3, hi=(0.5,) * 3, bc="UUU", sigma=1.0 / 20, rhs_scale=-1.0)]
    knobs = autotune.batch_knobs(problems, reps=1, per_class=2)
    assert len(knobs) == len(problems)
    desc = autotune.describe_knobs(problems, knobs)
    assert desc["classes"] == len({autotune.size_class(p) for p in problems})
    assert all(k["tune_radix"] in (8, 16) and k["tune_tile"] in (8, 16) for k in knobs)
    assert any(k.startswith("batchclasses:") for k in json.loads(cache.read_text()))
    plans = [sf.Plan(**p, **k) for p, k in zip(problems, knobs)]
    rng = np.random.default_rng(8)
    fs = [to_dev(rng.normal(size=pl.in_shape), "f32") for pl in plans]
    psis = [torch.empty(pl.out_shape, dtype=torch.float32, device="cuda") for pl in plans]
    batch = sf.Batch(plans)
    batch.solve(fs, psis)
    batch.sync()
    for p, f, psi in zip(problems, fs, psis):
        ref = sf.Plan(**p)
        want = _outputs(ref, f)[0]
        ref.close()
        assert rel_l2(to_np(psi), want) <= 1e-5, p
    batch.close()
    for pl in plans:
        pl.close()
