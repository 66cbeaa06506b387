"""Launch-shape autotuner for the stepper.

Searches the plan's tuning space (``cg_tuning`` plus the synchronisation
flag) by timing short runs of the actual workload, and remembers the winner
in a JSON cache keyed by GPU, model, stencil, scheme and size class.  The
knobs:

* ``cells_x``: cells per lane along x (tile width 32 or 64 columns);
* ``threads``, ``blocks_per_sm``: warps per SM of the persistent grid;
* ``schedule``: static balanced segments, the atomic tile queue with
  ``rows`` rows per tile, or temporal blocking (2) with ``rows`` steps per
  grid barrier;
* synchronisation depth between stages: a grid-wide barrier (default),
  neighbour-only waits, or one kernel launch per RK stage (the shallowest
  fusion: one stage per pass instead of every stage of the run in one pass).

Every candidate computes each cell with the same arithmetic, so results are
bitwise identical across the search space; the tuner checks that.
"""
from __future__ import annotations

import json
import os
import time
from typing import Dict, List, Optional

import torch

from . import api

FLAG_NEIGHBOR_SYNC = 1 << 2

DEFAULT_CANDIDATES: List[Dict] = [
    dict(cells_x=2, threads=512, blocks_per_sm=1, schedule=0),
    dict(cells_x=1, threads=512, blocks_per_sm=1, schedule=0),
    dict(cells_x=2, threads=256, blocks_per_sm=2, schedule=0),
    dict(cells_x=2, threads=512, blocks_per_sm=1, schedule=0, sync="neighbor"),
    dict(cells_x=2, threads=256, blocks_per_sm=2, schedule=0, sync="neighbor"),
    dict(cells_x=2, threads=512, blocks_per_sm=1, schedule=1, rows=4),
    dict(cells_x=1, threads=128, blocks_per_sm=4, schedule=1, rows=2),
    dict(cells_x=1, threads=512, blocks_per_sm=1, schedule=1, rows=2),
    dict(cells_x=2, threads=256, blocks_per_sm=2, schedule=1, rows=8),
    dict(cells_x=1, threads=512, blocks_per_sm=1, schedule=1, rows=4),
    # taller queue tiles: fewer window start-up rows per tile (row sums of
    # the 9-point stencil are formed for 2 extra rows per tile)
    dict(cells_x=1, threads=512, blocks_per_sm=1, schedule=1, rows=8),
    dict(cells_x=1, threads=512, blocks_per_sm=1, schedule=1, rows=16),
    dict(cells_x=1, threads=256, blocks_per_sm=2, schedule=1, rows=8),
    dict(cells_x=2, threads=512, blocks_per_sm=1, schedule=0, sync="per_stage"),
    # fewer, longer warp shares: the 9-point window's start-up rows are
    # amortised over more rows, at lower occupancy
    dict(cells_x=2, threads=256, blocks_per_sm=1, schedule=0),
    dict(cells_x=1, threads=256, blocks_per_sm=1, schedule=0),
    dict(cells_x=2, threads=384, blocks_per_sm=1, schedule=0),
    # temporal blocking (small grids): k steps per grid barrier in shared
    # memory; plan creation fails, and the candidate is skipped, where a
    # tile and its halo do not fit
    dict(schedule=2, rows=2, threads=256),
    dict(schedule=2, rows=4, threads=256),
    dict(schedule=2, rows=8, threads=256),
    dict(schedule=2, rows=1, threads=512),
    dict(schedule=2, rows=2, threads=512),
    dict(schedule=2, rows=4, threads=512),
    dict(schedule=2, rows=8, threads=512),
]


def cache_path() -> str:
    return os.environ.get("CG_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "cardiac_gb300", "autotune.json"))


def _size_class(problems) -> str:
    cells = sum(int(p.nx) * int(p.ny) for p in problems)
    return "n%d_c2^%d" % (len(problems), max(0, cells - 1).bit_length())


def cache_key(problems) -> str:
    p = problems[0]
    name = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    return "|".join([name, "m%d" % p.model, "st%d" % p.stencil, "sc%d" % p.scheme, "bc%d" % p.bc,
                     _size_class(problems)])


def _with_flags(problems, cand):
    out = []
    extra = 0
    if cand.get("sync") == "neighbor":
        extra = FLAG_NEIGHBOR_SYNC
    elif cand.get("sync") == "per_stage":
        extra = api.FLAG_PER_STAGE_LAUNCH
    for p in problems:
        q = api.Problem(**{k: getattr(p, k) for k in ("model", "nx", "ny", "dx", "dy", "D", "Dyy", "stencil", "bc",
                                                         "scheme", "alpha_d", "dt", "params", "barrier_timeout_s")})
        q.flags = p.flags | extra
        out.append(q)
    return out


def _tuning(cand):
    return {k: v for k, v in cand.items() if k in ("cells_x", "rows", "threads", "blocks_per_sm", "schedule")}


def tune(problems, z_in: torch.Tensor, n_steps: int = 50, candidates: Optional[List[Dict]] = None,
         reps: int = 3, use_cache: bool = True, verbose: bool = False) -> Dict:
    """Return the fastest candidate (a dict with the tuning and an optional
    ``sync`` entry) for these problems, timing ``n_steps`` steps from
    ``z_in`` (packed layout)."""
    if isinstance(problems, api.Problem):
        problems = [problems]
    key = cache_key(problems)
    path = cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            cache = json.load(open(path))
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            return cache[key]["best"]
    cands = candidates or DEFAULT_CANDIDATES
    results = []
    reference = None
    for cand in cands:
        try:
            plan = api.Plan(_with_flags(problems, cand), tuning=_tuning(cand))
        except Exception as exc:          # a shape the device cannot co-schedule
            if verbose:
                print("skip", cand, exc)
            continue
        out = plan.run(z_in, n_steps)
        plan.status()
        if reference is None:
            reference = out.clone()
        elif not torch.equal(out, reference):
            raise RuntimeError("autotune candidate %r changed the result" % (cand,))
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            plan.run(z_in, n_steps, out=out)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        plan.close()
        results.append((min(ts), cand))
        if verbose:
            print("%.3f ms  %r" % (1e3 * min(ts), cand))
    if not results:
        raise RuntimeError("no autotune candidate could run")
    results.sort(key=lambda r: r[0])
    best = results[0][1]
    if use_cache:
        cache[key] = {"best": best, "seconds": results[0][0], "when": time.time(),
                      "tried": [{"seconds": t, "cand": c} for t, c in results]}
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp%d" % os.getpid()
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1)
        os.replace(tmp, path)
    return best


def cached(problems) -> Optional[Dict]:
    """The cached winner for these problems, or None (no timing runs)."""
    if isinstance(problems, api.Problem):
        problems = [problems]
    try:
        return json.load(open(cache_path()))[cache_key(problems)]["best"]
    except (OSError, ValueError, KeyError):
        return None


def plan_for(problems, cand: Optional[Dict]) -> api.Plan:
    """Plan with a given candidate (None: library defaults)."""
    if isinstance(problems, api.Problem):
        problems = [problems]
    if cand is None:
        return api.Plan(problems)
    return api.Plan(_with_flags(problems, cand), tuning=_tuning(cand))


def tuned_plan(problems, z_in: torch.Tensor, **kw) -> api.Plan:
    """Plan built with the tuned launch shape."""
    if isinstance(problems, api.Problem):
        problems = [problems]
    best = tune(problems, z_in, **kw)
    return api.Plan(_with_flags(problems, best), tuning=_tuning(best))
