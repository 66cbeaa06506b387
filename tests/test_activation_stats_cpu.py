"""The activation statistics used to compare long runs, on signals whose
threshold crossings are known in closed form (piecewise-linear voltage, so
linear interpolation between samples is exact)."""
import numpy as np

from activation_stats import ActivationStats, compare, compare_restitution


def _tri(t, period, phase, lo=0.0, hi=2.0):
    """Triangle wave between lo and hi (rises for the first half period)."""
    x = np.mod(t - phase, period) / period
    return lo + (hi - lo) * np.where(x < 0.5, 2.0 * x, 2.0 - 2.0 * x)


def test_closed_form_triangle_waves():
    # each cell a triangle wave of its own period; threshold 1 is crossed
    # upward at phase + period/4 and downward at phase + 3 period/4, so
    # APD = period/2 and the activation interval = period
    periods = np.array([[8.0, 10.0], [12.5, 20.0]])
    phases = np.array([[0.0, 1.0], [2.5, 3.0]])
    dt = 0.25
    win = (30.0, 90.0)
    st = ActivationStats(_tri(0.0, periods, phases), 0.0, 1.0, window=win)
    for k in range(1, 481):
        st.add(_tri(k * dt, periods, phases), k * dt)
    s = st.summary()
    ups = []
    for p, ph in zip(periods.ravel(), phases.ravel()):
        t_up = ph + p / 4 + p * np.arange(0, 20)
        ups.append(t_up[(t_up >= win[0]) & (t_up <= win[1])])
    n_up = sum(len(u) for u in ups)
    assert s["activations_per_cell"] == n_up / 4
    assert s["active_fraction"] == 1.0
    apd = np.concatenate([np.full(len(u), p / 2) for u, p in zip(ups, periods.ravel())])
    assert s["apd"]["n"] == len(apd)
    assert abs(s["apd"]["mean"] - apd.mean()) <= 1e-12
    cl = np.concatenate([np.full(len(u), p) for u, p in zip(ups, periods.ravel())])
    assert s["interval"]["n"] == len(cl)
    assert abs(s["interval"]["mean"] - cl.mean()) <= 1e-12
    assert abs(s["interval"]["p50"] - np.percentile(cl, 50)) <= 1e-12


def test_compare_flags_each_statistic():
    a = {"apd": {"n": 1000, "mean": 50.0, "p10": 35.0, "p50": 47.0, "p90": 70.0},
         "interval": {"n": 1000, "mean": 80.0, "p10": 64.0, "p50": 77.0, "p90": 110.0},
         "activations_per_cell": 20.0, "active_fraction": 1.0}
    assert compare(a, a) == []
    b = {k: (dict(v) if isinstance(v, dict) else v) for k, v in a.items()}
    b["apd"]["mean"] = 50.6
    b["interval"]["p90"] = 112.0
    assert compare(a, b) == ["apd.mean", "interval.p90"]
    assert compare(a, b, rel_tail=0.05) == ["apd.mean"]
    assert compare(a, b, rel_mean=0.02, rel_tail=0.05) == []
    b["activations_per_cell"] = 20.3
    assert "activations_per_cell" in compare(a, b)
    assert "activations_per_cell" not in compare(a, b, rel_mean=0.02)
    b["apd"]["p50"] = 47.6
    assert "apd.p50" in compare(a, b, rel_mean=0.05, rel_tail=0.05)


def test_restitution_bins():
    """Beats with a known diastolic interval: each cell alternates
    repolarisation and activation at fixed offsets, so every beat's DI and
    APD are known; the per-bin means and counts follow."""
    # two cells: period 40 ms with APD 30 (DI 10) and period 50 with APD 20 (DI 30)
    periods = np.array([40.0, 50.0])
    apds = np.array([30.0, 20.0])

    def u_at(t):
        x = np.mod(t, periods)
        # piecewise linear: up through 1 at x = 5, down through 1 at x = 5 + apd
        up = np.clip((x - 4.5) * 2.0, 0.0, 2.0)
        dn = np.clip((x - (4.5 + apds)) * 2.0, 0.0, 2.0)
        return up - dn
    dt = 0.25
    st = ActivationStats(u_at(0.0), 0.0, 1.0, window=(60.0, 400.0))
    for k in range(1, 1601):
        st.add(u_at(k * dt), k * dt)
    r = st.restitution(width=5.0, n_bins=10)
    assert r["n"][2] > 0 and r["n"][6] > 0 and sum(r["n"]) == r["n"][2] + r["n"][6]
    assert abs(r["mean_apd"][2] - 30.0) <= 1e-12 and abs(r["mean_apd"][6] - 20.0) <= 1e-12
    b = {"n": list(r["n"]), "mean_apd": list(r["mean_apd"])}
    assert compare_restitution(r, b) == []
    b["mean_apd"][6] = 20.3
    assert compare_restitution(r, b) == [6]
    assert compare_restitution(r, b, rel=0.02) == []
