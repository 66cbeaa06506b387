"""The long chaotic run of the Karma model (Eq. karma) whose activation
statistics the GPU path must reproduce (test infrastructure: the protocol
only; the stepping is passed in, so this module holds none of the method's
arithmetic).

Why this workload: the paper argues for double precision because long
chaotic runs diverge pointwise from any perturbation (Sect. 1), so such
runs can only be compared statistically.  With the paper's Karma
constants (Re, M) = (1, 6) and with the four-field model's epicardial set
the spirals these protocols make are stable: a rounding-level perturbation
stays below 1e-11 over a second.  With M = 10 (the steep v^M of Karma's own
spiral-breakup study) the same S1-S2 protocol on 512^2 cells gives
irregular reentry in which a one-ulp perturbation of u grows by about a
decade every 180 ms and reaches O(1) after 3.6 s.

Protocol: rest (u = v = 0); S1: u = 3 in the 10 leftmost columns; after
600 ms, S2: u = 3 on the lower half (rows y < 256), unconditionally, so
the edit is the same on every path; then 8000 ms more.  Frames every
10 steps (0.5 ms) feed the activation statistics (threshold u = u_v = 1)
of the windows below, in ms after S2."""
from __future__ import annotations

N = 512
DX = 0.0262              # cm, Sect. 2
GAMMA = 1.1e-3           # cm^2/ms, Sect. 2
DT = 0.05                # ms
# tau_u, tau_v, u*, u_h, u_v, Re, M, k (cg_default_params order) with M = 10
PARAMS = [2.5, 250.0, 1.5415, 3.0, 1.0, 1.0, 10.0, 28.4]
S1_COLS = 10
STIM_U = 3.0
S2_STEP = 12000          # 600 ms
AFTER_S2 = 160000        # 8000 ms
SAMPLE = 10              # steps between frames
THETA = 1.0
WINDOWS = {"3000-8000": (3000.0, 8000.0), "4000-8000": (4000.0, 8000.0)}
CHECKPOINTS_MS = (0, 1000, 2000, 3000, 4000, 5000, 6000, 7000, 8000)
SUB = 32                 # pointwise samples: u at every 32nd row and column


def initial_state(np):
    z = np.zeros((2, N, N), dtype=np.float64)
    z[0, :, :S1_COLS] = STIM_U
    return z


def apply_s2(z):
    z[0, : N // 2, :] = STIM_U
    return z


LEAD_MS = 500.0          # frames start this long before a window opens


def run(advance, to_numpy, z, stats_factory):
    """Drive the protocol.  advance(z, n) returns the state n steps later;
    to_numpy(z) gives u as a numpy array; stats_factory(u0, t0, window)
    makes a statistics accumulator (ActivationStats).  Returns (summary per
    window, {ms after S2: u[::SUB, ::SUB]})."""
    z = advance(z, S2_STEP)
    z = apply_s2(z)
    u = to_numpy(z)
    snaps = {0: u[::SUB, ::SUB].copy()}
    stats = {}
    start = {k: w[0] - LEAD_MS for k, w in WINDOWS.items()}
    steps_per_ms = int(round(1.0 / DT))
    for k in range(1, AFTER_S2 // SAMPLE + 1):
        z = advance(z, SAMPLE)
        n = k * SAMPLE
        t = n * DT
        ms = n // steps_per_ms if n % steps_per_ms == 0 else None
        is_cp = ms is not None and ms in CHECKPOINTS_MS
        live = [key for key in WINDOWS if t >= start[key]]
        if not live and not is_cp:
            continue
        u = to_numpy(z)
        if is_cp:
            snaps[ms] = u[::SUB, ::SUB].copy()
        for key in live:
            if key not in stats:
                stats[key] = stats_factory(u, t, WINDOWS[key])
            else:
                stats[key].add(u, t)
    return {key: st.summary() for key, st in stats.items()}, snaps
