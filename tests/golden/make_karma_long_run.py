"""Writes karma_long_run_512.json: the CPU oracle's activation statistics
and sampled voltages for the long chaotic Karma run of
tests/karma_long_run.py (the Karma model of Eq. karma with M = 10 on 512^2
cells, RK4, dt 0.05 ms, S1-S2 initiation, 8000 ms after S2).  Calls only
the oracle (about 2.5 hours on one x86 core):

    python tests/golden/make_karma_long_run.py
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

import oracle as O  # noqa: E402
import karma_long_run as K  # noqa: E402
from activation_stats import ActivationStats  # noqa: E402


def main():
    p = O.problem(O.KARMA, nx=K.N, ny=K.N, dx=K.DX, Dxx=[K.GAMMA, 0.0], scheme=O.RK4, dt=K.DT,
                  params=K.PARAMS)
    t0 = time.time()
    stats, snaps = K.run(lambda z, n: O.step(p, z, n), lambda z: z[0], K.initial_state(np),
                         lambda u0, t, w: ActivationStats(u0, t, K.THETA, w))
    out = {
        "what": "oracle activation statistics and sampled u of the long Karma run (tests/karma_long_run.py)",
        "writer": "tests/golden/make_karma_long_run.py (oracle only)",
        "seconds": time.time() - t0,
        "stats": stats,
        "snapshots_ms": {str(k): v.tolist() for k, v in sorted(snaps.items())},
    }
    with open(os.path.join(HERE, "karma_long_run_512.json"), "w") as fh:
        json.dump(out, fh, indent=0)
    print("wrote karma_long_run_512.json in %.0f s" % out["seconds"])


if __name__ == "__main__":
    main()
