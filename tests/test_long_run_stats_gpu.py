"""Long chaotic runs compared by statistics (the paper's reason for double
precision, Sect. 1: such runs diverge pointwise from any perturbation).

The Karma model of Eq. (karma) with M = 10 on 512^2 cells, RK4, dt 0.05 ms,
S1-S2 initiation, 8000 ms after S2 (tests/karma_long_run.py): 172,000 steps
on the GPU through the C ABI, against the CPU oracle's run of the same
protocol (stored by tests/golden/make_karma_long_run.py, oracle only).

Checks:
* right after S2 the two agree pointwise (the S1 plane wave is stable), and
  at the end they have decorrelated (max |du| above 1e-3 on the sampled
  cells: the dynamics are chaotic);
* the action-potential-duration restitution over 3000-8000 ms after S2
  (threshold u = u_v = 1: the mean APD of the beats whose preceding
  diastolic interval falls in each 5 ms bin) agrees within 1% in every bin
  holding at least 2.5% of the beats;
* the distributions of APD and activation interval (count, mean, 10/50/90%
  quantiles) and the activations per cell agree within 10% (15% for the
  90% quantiles): the same dynamical regime.

Why these two levels: the whole-domain distributions of one 5 s run on a
13 cm domain depend on where the chaotic trajectory happens to go; runs
that differ only by rounding (GPU runs whose u differs by one ulp after S2,
and the oracle) spread by up to 3% in the means and 8% in the 90%
quantiles over this window.  The restitution relation is a property of the
dynamics rather than of the trajectory: the same runs agree within 0.63%
in its well-populated bins."""
import json
import os

import numpy as np
import pytest

import karma_long_run as K
from activation_stats import ActivationStats, compare, compare_restitution

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
WINDOW = "3000-8000"


def test_karma_long_chaotic_run_statistics(cuda_ok):
    import torch
    from paper_1309_1720_gb300 import Plan, Problem, KARMA, RK4
    with open(os.path.join(HERE, "golden", "karma_long_run_512.json")) as fh:
        gold = json.load(fh)
    plan = Plan(Problem(model=KARMA, nx=K.N, ny=K.N, dx=K.DX, D=(K.GAMMA,), scheme=RK4, dt=K.DT,
                        params=K.PARAMS))
    bufs = [torch.empty((2, K.N, K.N), dtype=torch.float64, device="cuda") for _ in range(2)]
    turn = [0]

    def advance(z, n):
        out = bufs[turn[0]]
        turn[0] ^= 1
        return plan.run(z, n, out=out)

    z0 = torch.from_numpy(K.initial_state(np)).cuda()
    stats, snaps = K.run(advance, lambda z: z[0].cpu().numpy(), z0,
                         lambda u, t, w: ActivationStats(u, t, K.THETA, w))
    plan.status()
    ref = {int(k): np.asarray(v) for k, v in gold["snapshots_ms"].items()}
    scale = max(float(np.abs(v).max()) for v in ref.values())
    early = float(np.abs(snaps[0] - ref[0]).max())
    late = float(np.abs(snaps[K.CHECKPOINTS_MS[-1]] - ref[K.CHECKPOINTS_MS[-1]]).max())
    g, o = stats[WINDOW], gold["stats"][WINDOW]
    rg, ro = g["restitution"], o["restitution"]
    tot = sum(ro["n"])
    rel_bins = {k: rg["mean_apd"][k] / ro["mean_apd"][k] - 1.0 for k in range(len(ro["n"]))
                if ro["n"][k] >= 0.025 * tot and rg["mean_apd"][k] is not None}
    rel = {k + "." + q: (g[k][q] - o[k][q]) / o[k]["p50"] for k in ("apd", "interval")
           for q in ("mean", "p10", "p50", "p90")}
    rel["activations_per_cell"] = g["activations_per_cell"] / o["activations_per_cell"] - 1.0
    print("long run: max |du| %.3g after S2, %.3g at the end; restitution by bin %s; distributions %s"
          % (early, late, rel_bins, rel))
    assert early <= 1e-9 * scale, early
    assert late >= 1e-3, late
    assert len(rel_bins) >= 5, rel_bins
    assert not compare_restitution(ro, rg, rel=0.01, min_share=0.025), rel_bins
    bad = compare(o, g, rel=0.10, rel_mean=0.10, rel_tail=0.15)
    assert not bad, (bad, rel)
