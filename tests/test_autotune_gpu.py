"""The autotuner times real runs over the launch-shape space, caches the
winner, and every candidate gives bitwise the same result."""
import json

import pytest

from paper_1309_1720_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_tune_batch_and_cache(cuda_ok, tmp_path, monkeypatch):
    import torch
    from paper_1309_1720_gb300 import Plan, Problem, FHN, RK4, autotune
    monkeypatch.setenv("CG_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    sizes, states, dus = I.batch_workload(n_inst=16, lo=40, hi=200, seed=3)
    probs = [Problem(model=FHN, nx=int(n), ny=int(n), dx=0.04, D=(float(d), 1.5), scheme=RK4, dt=2.5e-4)
             for n, d in zip(sizes, dus)]
    base = Plan(probs)
    zin = base.pack(states)
    best = autotune.tune(probs, zin, n_steps=10)
    data = json.load(open(tmp_path / "tune.json"))
    key = autotune.cache_key(probs)
    assert data[key]["best"] == best and len(data[key]["tried"]) >= 4
    # cached on the second call
    assert autotune.tune(probs, zin, n_steps=10) == best
    tp = autotune.tuned_plan(probs, zin, n_steps=10)
    assert torch.equal(tp.run(zin, 15), base.run(zin, 15))
