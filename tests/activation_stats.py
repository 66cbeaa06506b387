"""Activation and action-potential-duration statistics of a voltage field
sampled in time (test infrastructure, no model arithmetic).

A cell activates when its voltage crosses the threshold upward and
repolarises when it crosses it downward; crossing times are interpolated
linearly between samples.  Over a time window the statistics are: the
activation intervals (time between successive activations of a cell), the
action-potential durations (activation to the next repolarisation), the
mean number of activations per cell and the fraction of cells that
activate.  Long chaotic runs are compared through these numbers rather than
pointwise (the paper's reason for double precision is that such runs
diverge pointwise, Sect. 1)."""
from __future__ import annotations

import numpy as np


class ActivationStats:
    """Streaming accumulation over frames u(t).  Beats are counted when
    their activation time lies in ``window``; ``t0`` is the time of the
    first frame u0."""

    def __init__(self, u0: np.ndarray, t0: float, theta: float, window=(0.0, np.inf)):
        self.theta = float(theta)
        self.win = window
        self.t_prev = float(t0)
        self.u_prev = np.array(u0, dtype=np.float64, copy=True)
        self.above = self.u_prev > self.theta
        self.last_up = np.full(self.u_prev.shape, np.nan)
        self.n_up = np.zeros(self.u_prev.shape, dtype=np.int64)
        self.apd, self.cl = [], []

    def add(self, u: np.ndarray, t: float) -> None:
        u = np.asarray(u, dtype=np.float64)
        th, up_prev, t_prev = self.theta, self.u_prev, self.t_prev
        dts = float(t) - t_prev
        lo, hi = self.win
        now_above = u > th
        dn = self.above & ~now_above
        if dn.any():
            t_dn = t_prev + (up_prev[dn] - th) / (up_prev[dn] - u[dn]) * dts
            t_a = self.last_up[dn]
            ok = np.isfinite(t_a) & (t_a >= lo) & (t_a <= hi)
            self.apd.append((t_dn - t_a)[ok])
        up = ~self.above & now_above
        if up.any():
            t_up = t_prev + (th - up_prev[up]) / (u[up] - up_prev[up]) * dts
            t_a = self.last_up[up]
            ok = np.isfinite(t_a) & (t_up >= lo) & (t_up <= hi)
            self.cl.append((t_up - t_a)[ok])
            inwin = (t_up >= lo) & (t_up <= hi)
            idx = np.flatnonzero(up)
            self.n_up.flat[idx[inwin]] += 1
            self.last_up[up] = t_up
        self.above = now_above
        self.u_prev = u.copy()
        self.t_prev = float(t)

    def summary(self) -> dict:
        def q(x):
            x = np.concatenate(x) if x else np.zeros(0)
            if x.size == 0:
                return {"n": 0}
            return {"n": int(x.size), "mean": float(x.mean()), "p10": float(np.percentile(x, 10)),
                    "p50": float(np.percentile(x, 50)), "p90": float(np.percentile(x, 90))}
        return {"apd": q(self.apd), "interval": q(self.cl),
                "activations_per_cell": float(self.n_up.mean()),
                "active_fraction": float((self.n_up > 0).mean())}


def compare(a: dict, b: dict, rel: float = 0.01, rel_tail: float = None) -> list:
    """Names of the statistics of b that differ from a's by more than rel
    (relative to a's; percentiles relative to a's median); the 90%
    quantiles by more than rel_tail (default rel)."""
    tail = rel if rel_tail is None else rel_tail
    bad = []
    for key in ("apd", "interval"):
        sa, sb = a[key], b[key]
        if sa["n"] == 0 or sb["n"] == 0:
            bad.append(key + ".n")
            continue
        if abs(sb["n"] - sa["n"]) > rel * sa["n"]:
            bad.append(key + ".n")
        if abs(sb["mean"] - sa["mean"]) > rel * abs(sa["mean"]):
            bad.append(key + ".mean")
        for p, r in (("p10", rel), ("p50", rel), ("p90", tail)):
            if abs(sb[p] - sa[p]) > r * abs(sa["p50"]):
                bad.append(key + "." + p)
    for key in ("activations_per_cell", "active_fraction"):
        if abs(b[key] - a[key]) > rel * abs(a[key]):
            bad.append(key)
    return bad
