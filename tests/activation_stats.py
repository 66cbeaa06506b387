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
        self.last_dn = np.full(self.u_prev.shape, np.nan)
        self.di_up = np.full(self.u_prev.shape, np.nan)     # diastolic interval before the current beat
        self.n_up = np.zeros(self.u_prev.shape, dtype=np.int64)
        self.apd, self.cl, self.di = [], [], []

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
            self.di.append(self.di_up[dn][ok])
            self.last_dn[dn] = t_dn
        up = ~self.above & now_above
        if up.any():
            t_up = t_prev + (th - up_prev[up]) / (u[up] - up_prev[up]) * dts
            t_a = self.last_up[up]
            ok = np.isfinite(t_a) & (t_up >= lo) & (t_up <= hi)
            self.cl.append((t_up - t_a)[ok])
            inwin = (t_up >= lo) & (t_up <= hi)
            idx = np.flatnonzero(up)
            self.n_up.flat[idx[inwin]] += 1
            self.di_up[up] = t_up - self.last_dn[up]
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
                "active_fraction": float((self.n_up > 0).mean()),
                "restitution": self.restitution()}

    def restitution(self, width: float = 5.0, n_bins: int = 40) -> dict:
        """APD restitution: the mean action-potential duration of the beats
        whose preceding diastolic interval (the previous repolarisation to
        this activation) falls in [k width, (k + 1) width), with the beat
        count per bin (beats with a known interval only)."""
        apd = np.concatenate(self.apd) if self.apd else np.zeros(0)
        di = np.concatenate(self.di) if self.di else np.zeros(0)
        ok = np.isfinite(di)
        apd, di = apd[ok], di[ok]
        k = np.floor(di / width).astype(np.int64)
        out = {"width": width, "n": [], "mean_apd": []}
        for b in range(n_bins):
            m = k == b
            out["n"].append(int(m.sum()))
            out["mean_apd"].append(float(apd[m].mean()) if m.any() else None)
        return out


def compare_restitution(a: dict, b: dict, rel: float = 0.01, min_share: float = 0.01) -> list:
    """Bins (by index) whose mean APD differs by more than rel between a and
    b, among the bins holding at least min_share of a's beats."""
    tot = sum(a["n"])
    bad = []
    for k, (na, ma, mb) in enumerate(zip(a["n"], a["mean_apd"], b["mean_apd"])):
        if tot == 0 or na < min_share * tot:
            continue
        if mb is None or abs(mb - ma) > rel * abs(ma):
            bad.append(k)
    return bad


def compare(a: dict, b: dict, rel: float = 0.01, rel_mean: float = None, rel_tail: float = None) -> list:
    """Names of the statistics of b that differ from a's by more than their
    tolerance, relative to a's value (quantiles relative to a's median):
    rel for the 10% and 50% quantiles, rel_mean (default rel) for the means,
    the counts and the activations per cell, rel_tail (default rel) for the
    90% quantiles."""
    mean_tol = rel if rel_mean is None else rel_mean
    tail = rel if rel_tail is None else rel_tail
    bad = []
    for key in ("apd", "interval"):
        sa, sb = a[key], b[key]
        if sa["n"] == 0 or sb["n"] == 0:
            bad.append(key + ".n")
            continue
        if abs(sb["n"] - sa["n"]) > mean_tol * sa["n"]:
            bad.append(key + ".n")
        if abs(sb["mean"] - sa["mean"]) > mean_tol * abs(sa["mean"]):
            bad.append(key + ".mean")
        for p, r in (("p10", rel), ("p50", rel), ("p90", tail)):
            if abs(sb[p] - sa[p]) > r * abs(sa["p50"]):
                bad.append(key + "." + p)
    if abs(b["activations_per_cell"] - a["activations_per_cell"]) > mean_tol * abs(a["activations_per_cell"]):
        bad.append("activations_per_cell")
    if abs(b["active_fraction"] - a["active_fraction"]) > rel * abs(a["active_fraction"]):
        bad.append("active_fraction")
    return bad
