#!/usr/bin/env python3
"""Benchmark of the fused FP64 cardiac stepper on GB300.

Workload (one bench step): the paper's four-field Bueno-Orovio-Cherry-Fenton
model (Sect. 2, Eq. bochfe; voltage u and gates v, w, s) on a 2048 x 2048
grid (dx = 0.03 cm), anisotropic diagonal diffusion Dxx = 1.171e-3 cm^2/ms =
4 Dyy on the 9-point stencil (alpha_d = 1/6), no-flux mirror ghosts, classic
RK4 with dt = 0.05 ms, 5000 time steps from the seeded eight-core spiral
state; one persistent kernel launch per bench step.
Metric: FP64 giga cell-updates per second (GCUPS) and the fraction of the
FP64 roofline.  Also reported: the same metric end to end through the public
API with host buffers, the other workloads (the 1024^2 two-field RK4 run,
the small grid, the gate integrators, Karma, the batch, the tangent-linear
and adjoint runs), and the CPU oracle on a bounded sample of the workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FP64 GCUPS & % of HBM/FP64 roofline; batched and adjoint/JVP vs plain stepper"

# ---------------------------------------------------------------- workload
NX = NY = 2048
DX = 0.03                      # cm (Sect. 2)
D_XX = 1.171e-3                # cm^2/ms (Sect. 2: D = 1.171 cm^2/s)
D_YY = D_XX / 4.0
DT = 0.05                      # ms
STEPS_PER_RUN = 5000
# Algorithmic HBM bytes per cell-update of a fused step: four fields read
# and written once (4 x 8 B x 2).
BYTES_PER_CELL_UPDATE = 64

# Algorithmic FP64 flops of one cell and one RK stage (FMA = 2, add = 1,
# multiply = 1), per branch of the local terms, including the anisotropic
# 9-point stencil on u (row-sum form) and the stage combine of the four
# fields.  A branch is the switch state of the cell's own voltage:
#   rest     u <= theta_w - 1/(2k): the v and w switches H_k are exactly 0,
#            so every term they multiply is exactly 0 and is not evaluated;
#   excited  u >= theta_v + 1/(2k): every switch is exactly 1;
#   general  in between: the whole of Eq. (bochfe).
# The sigmoid, exponential and reciprocal count at the flops of the
# library's own evaluations as they stood when the count was frozen
# (Tang's table-driven exponential with a 256-entry table: 7 FMA, 1 add,
# 1 multiply; a cubic Newton reciprocal: 3 FMA), which take the place of
# the tanh and division costs T and R; later changes that evaluate the same
# functions with fewer operations show as speed, not as a lower count.
# Frozen from ncu's per-opcode counters (DFMA x 2 + DADD + DMUL thread
# instructions per cell and stage) on uniform states where every warp takes
# one branch, in the workload's tuned launch shape:
#   rest     DFMA 48.5, DADD 14.5, DMUL 13.0 -> 124.5
#   excited  DFMA 34.5, DADD 13.5, DMUL 13.0 ->  95.5
#   general  DFMA 71.5, DADD 23.5, DMUL 31.0 -> 197.5
# A cell is charged its own branch, so a warp whose lanes straddle a switch
# (it runs the general path for all 32) does more than this count.
BOCF_STAGE_FLOPS = {"rest": 124.5, "excited": 95.5, "general": 197.5}
# DRAM bytes per cell-update measured by ncu (dram__bytes_read.sum +
# dram__bytes_write.sum) on a 2-step launch of this workload in its tuned
# shape: every RK stage streams the state, the accumulator and the stage
# buffers of the four fields (640 MB, more than L2) through HBM, so the
# traffic grows in proportion to the steps of a launch.
MEASURED_DRAM_BYTES_PER_CELL_UPDATE = 508.8

# the 1024^2 two-field row (the FitzHugh-Nagumo model, 9-point isotropic,
# RK4): per stage 9-point Laplacian 2 x 11, local terms 8, D scaling 2 x 2,
# combine 2 x 4; x 4 stages
FHN_FLOPS_PER_CELL_UPDATE = 168


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-rows", action="store_true", help="skip the secondary workloads")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--profile-case", nargs="?", const="bocf", default=None,
                    choices=["fhn", "bocf", "bocf-branches", "fp64-probe", "karma", "tlm", "adj", "c1"],
                    help="run a short case and exit (for ncu captures): 2 steps of the 2048^2 four-field "
                         "workload in its tuned launch shape (bocf); 2 steps of the same plan on three "
                         "uniform states, one per branch of the local terms (bocf-branches); the FP64 "
                         "DFMA, DADD and DMUL rate probes and the one-lane DFMA probe (fp64-probe); 20 "
                         "steps of the 1024^2 two-field "
                         "RK4 workload (fhn); 10 steps of the 2048^2 Karma model (karma); on the 512^2 "
                         "two-field RK4 problem 4 steps of 64 tangents (tlm) or the adjoint of 16 steps "
                         "(adj); or 200 steps of the 128^2 Euler problem with 4 steps per grid barrier (c1)")
    ap.add_argument("--experiment", default=None,
                    choices=["all", "timing", "grid", "convergence", "orbit", "snapshots", "small-grid"],
                    help="run the paper's timing / grid-size / accuracy experiments instead of the bench")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, ws: int) -> float:
    """Largest value of x over all ranks (the slowest replica's time)."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(cell_updates_per_rank: float, ws: int, seconds: float) -> float:
    """Whole-job GCUPS: every rank steps its own replica of the workload (the
    path runs one instance per GPU; replicas share nothing), so the job's
    cell-updates are ws times one rank's, over the slowest rank's time."""
    return ws * cell_updates_per_rank / seconds / 1e9


def bocf_flops_per_cell_update(mix) -> float:
    """Algorithmic FP64 flops of one RK4 cell-update of the four-field model
    for a branch mix {branch: fraction of cell-stages}."""
    return 4.0 * sum(BOCF_STAGE_FLOPS[b] * f for b, f in mix.items())


def bocf_branch_bounds(params):
    """Voltage bounds of the rest and excited branches: u <= theta_w - 1/(2k)
    puts the v and w switches at exactly 0, u >= max(thresholds) + 1/(2k)
    puts all four at exactly 1 (params in cg_default_params order)."""
    th_v, th_w, th_vm, th_o, k = params[2], params[3], params[4], params[5], params[28]
    return min(th_v, th_w) - 0.5 / k, max(th_v, th_w, th_vm, th_o) + 0.5 / k


def headline_problem(api):
    return api.Problem(model=api.BOCF, nx=NX, ny=NY, dx=DX, D=(D_XX,), Dyy=(D_YY,), stencil=api.STENCIL9,
                       alpha_d=1 / 6, scheme=api.RK4, dt=DT)


def headline_state(I):
    return I.bocf_spiral_cores(NX, NY, seed=0)


def oracle_headline_problem(O):
    return O.problem(O.BOCF, nx=NX, ny=NY, dx=DX, Dxx=[D_XX, 0, 0, 0], Dyy=[D_YY, 0, 0, 0], stencil=O.ST9,
                     alpha_d=1 / 6, scheme=O.RK4, dt=DT)


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        out_dir = os.environ.get("CG_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, "clocks_%d.csv" % os.getpid())

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        except OSError:
            return None
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measure_fp64_peak():
    """FP64 DFMA throughput of this GPU (TFLOP/s, FMA = 2) from the library's
    probe, best of three."""
    import ctypes
    from paper_1309_1720_gb300 import _lib
    L = _lib.lib()
    rate = ctypes.c_double()
    best = 0.0
    for _ in range(3):
        _lib.check(L.cg_measure_fp64_rate(0, 0, ctypes.byref(rate), None))
        best = max(best, rate.value)
    return 2.0 * best / 1e12, best


def cpu_baseline(seconds_target=12.0):
    """The oracle as it stands (single thread) on a bounded sample of the
    workload: the same 2048^2 four-field RK4 problem for a few steps."""
    import oracle as O
    from paper_1309_1720_gb300 import inputs as I
    z = headline_state(I)
    p = oracle_headline_problem(O)
    t = time.perf_counter()
    z1 = O.step(p, z, 1)
    per = time.perf_counter() - t
    n = int(max(2, min(50, seconds_target / max(per, 1e-6))))
    t = time.perf_counter()
    O.step(p, z1, n)
    dt = time.perf_counter() - t
    out = {"value": NX * NY * n / dt / 1e9, "unit": "GCUPS", "cores": 1, "kind": "oracle",
           "sample": "%d RK4 steps of the 2048x2048 four-field anisotropic 9-point workload, single-threaded C "
                     "oracle (-O2 -ffp-contract=off), rate extrapolated to the full run" % n,
           "seconds": dt}
    # every host core: one independent single-threaded copy of the same
    # oracle per core on the same sample (ctypes releases the GIL during the
    # call, so the copies run in parallel; the oracle itself is unchanged)
    import threading
    cores = os.cpu_count() or 1
    m = 2
    copies = [z1.copy() for _ in range(cores)]
    threads = [threading.Thread(target=O.step, args=(p, c, m)) for c in copies]
    t = time.perf_counter()
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    dt_all = time.perf_counter() - t
    out["all_cores"] = {"value": cores * NX * NY * m / dt_all / 1e9, "unit": "GCUPS", "cores": cores,
                        "kind": "oracle, one independent single-threaded copy per core",
                        "sample": "%d RK4 steps per copy of the same workload" % m, "seconds": dt_all}
    return out


def run_reference(args):
    """The reference arm: the CPU oracle, single-threaded, on the headline
    workload; each bench step is a bounded sample of one RK4 time step of
    the 2048^2 four-field problem (the rate is per cell-update)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle as O
    from paper_1309_1720_gb300 import inputs as I
    z = headline_state(I)
    p = oracle_headline_problem(O)
    sample_steps = 1
    for _ in range(args.warmup):
        z = O.step(p, z, sample_steps)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        z = O.step(p, z, sample_steps)
        times.append(time.perf_counter() - t)
    tot = sum(times)
    val = NX * NY * sample_steps * args.steps / tot / 1e9
    line = {
        "metric": METRIC, "value": val, "unit": "GCUPS", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": workload_config(),
        "cpu_baseline": {"value": val, "unit": "GCUPS", "cores": 1, "kind": "oracle",
                         "sample": "each step: %d RK4 time step of the 2048x2048 four-field anisotropic 9-point "
                                   "workload on the single-threaded C oracle" % sample_steps},
        "e2e": {"value": val, "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config():
    return {"workload": "bocf-2048x2048-aniso9pt-rk4-5000steps",
            "system": "Bueno-Orovio-Cherry-Fenton four-field equations (Eq. bochfe), epicardial constants, H_k "
                      "with k = 28.4",
            "grid": [NX, NY], "dx_cm": DX, "D_cm2_per_ms": {"xx": D_XX, "yy": D_YY},
            "stencil": "9-point anisotropic diagonal tensor, alpha_d = 1/6", "bc": "no-flux mirror",
            "scheme": "RK4", "dt_ms": DT, "time_steps_per_bench_step": STEPS_PER_RUN,
            "ic": "seeded eight-core spiral state (seed 0) plus 1e-3 noise",
            "l2": "inputs larger than L2: the 128 MiB state and 512 MiB of stage buffers are streamed from HBM "
                  "each stage; L2 also flushed (256 MB write) between timed bench steps"}


def secondary_rows(torch, plan_cls, I, api, peak_tflops, head_tuning):
    """Short rate measurements of the other workloads (rate-based; truncated
    step counts are stated)."""
    rows = {}

    def timed(plan, z, n, reps=3):
        out = torch.empty_like(z)
        plan.run(z, n, out=out)
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            plan.run(z, n, out=out)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        plan.status()
        return min(ts)

    # 128^2 explicit Euler, 5-point, 1000 steps (launch/latency-bound size)
    from paper_1309_1720_gb300 import autotune
    p = api.Problem(model=api.FHN, nx=128, ny=128, dx=0.04, scheme=api.EULER, dt=2e-4)
    z = torch.from_numpy(I.fhn_broken_wave(128, 128, seed=0)).cuda()
    tun = autotune.tune([p], z, n_steps=200)
    plan = autotune.tuned_plan([p], z, n_steps=200)
    t = timed(plan, z, 1000)
    rows["fhn-128x128-5pt-euler-1000steps"] = {"gcups": 128 * 128 * 1000 / t / 1e9, "seconds": t, "tuning": tun}
    plan.close()

    # the 1024^2 two-field workload: FitzHugh-Nagumo, 9-point isotropic,
    # RK4, dt = 4e-4, 10000 steps from the seeded broken wave (whole runs,
    # L2 flushed between them; the 80 MB working set is L2-resident within a
    # run by design)
    n, steps = 1024, 10000
    p2 = api.Problem(model=api.FHN, nx=n, ny=n, dx=0.04, stencil=api.STENCIL9, alpha_d=1 / 6, scheme=api.RK4,
                     dt=4e-4)
    z = torch.from_numpy(I.fhn_broken_wave(n, n, seed=0)).cuda()
    tun2 = autotune.tune([p2], z, n_steps=200)
    plan = autotune.tuned_plan([p2], z, n_steps=200)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    out = torch.empty_like(z)
    plan.run(z, steps, out=out)
    ts = []
    for _ in range(3):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        plan.run(z, steps, out=out)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) / 1e3)
    plan.status()
    t = statistics.median(ts)
    ach = FHN_FLOPS_PER_CELL_UPDATE * n * n * steps / t / 1e12
    rows["fhn-1024x1024-9pt-rk4-10000steps"] = {
        "gcups": n * n * steps / t / 1e9, "seconds": t, "tuning": tun2,
        "roofline": {"bound": "alu", "achieved": ach, "peak": peak_tflops, "unit": "TFLOP/s",
                     "frac": ach / peak_tflops, "flops_per_cell_update": FHN_FLOPS_PER_CELL_UPDATE},
        "note": "median of 3 whole runs, L2 flushed between them"}
    plan.close()
    del flush, out, z

    # the gate integrators and the tanh variant on the headline workload
    n, steps = NX, 500
    p = headline_problem(api)
    z = torch.from_numpy(headline_state(I)).cuda()
    tun = head_tuning
    for name, kw in [("bocf-2048x2048-aniso9pt-rk4-tanh-as-hk", dict(flags=api.FLAG_TANH_AS_HK)),
                     ("bocf-2048x2048-aniso9pt-rush-larsen", dict(scheme=api.RUSH_LARSEN)),
                     ("bocf-2048x2048-aniso9pt-implicit-euler", dict(scheme=api.IMPLICIT_EULER))]:
        q = api.Problem(**{**{k: getattr(p, k) for k in ("model", "nx", "ny", "dx", "D", "Dyy", "stencil",
                                                            "scheme", "dt", "flags")}, **kw})
        plan = autotune.plan_for([q], tun)
        t = timed(plan, z, steps, reps=2)
        rows[name] = {"gcups": n * n * steps / t / 1e9, "seconds": t, "steps_timed": steps,
                      "note": "rate of 500 steps, launch shape of the headline RK4 workload"}
        plan.close()

    # the Karma model (Eq. karma): the 256^2 grid of the paper's timing
    # figures (autotuned, temporal blocking allowed) and a 2048^2 grid
    for n, steps in ((256, 2000), (2048, 500)):
        p = api.Problem(model=api.KARMA, nx=n, ny=n, dx=I.KARMA_DX, D=(I.KARMA_GAMMA,), scheme=api.RK4,
                        dt=0.05)
        z = torch.from_numpy(I.karma_broken_wave(n, n, seed=0)).cuda()
        tun = autotune.tune([p], z, n_steps=200 if n <= 256 else 10)
        plan = autotune.plan_for([p], tun)
        t = timed(plan, z, steps, reps=2)
        rows["karma-%dx%d-5pt-rk4" % (n, n)] = {"gcups": n * n * steps / t / 1e9, "seconds": t, "tuning": tun,
                                               "steps_timed": steps, "us_per_step": 1e6 * t / steps}
        plan.close()
        del z

    # 256 uneven instances (64..512, seed 1), 5-point RK4: one persistent
    # launch replayed from a CUDA graph vs 256 sequential single-instance runs
    steps = 200
    sizes, states, dus = I.batch_workload(n_inst=256, seed=1)
    probs = [api.Problem(model=api.FHN, nx=int(n), ny=int(n), dx=0.04, D=(float(d), 1.5),
                         scheme=api.RK4, dt=2.5e-4) for n, d in zip(sizes, dus)]
    cells = int(np.sum(sizes.astype(np.int64) ** 2))
    from paper_1309_1720_gb300 import autotune
    zin = plan_cls(probs).pack(states)
    batch_tuning = autotune.tune(probs, zin, n_steps=20)
    bp = autotune.tuned_plan(probs, zin, n_steps=20)
    zout = torch.empty_like(zin)
    bp.run(zin, steps, out=zout)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        bp.run(zin, steps, out=zout, stream=torch.cuda.current_stream())
    g.replay()
    torch.cuda.synchronize()
    tb = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.replay()
        e1.record()
        torch.cuda.synchronize()
        tb.append(e0.elapsed_time(e1) / 1e3)
    bp.status()
    seq_plans = [plan_cls(p) for p in probs]
    parts_in = bp.unpack(zin)
    outs = [torch.empty_like(x) for x in parts_in]
    for sp, zi, zo in zip(seq_plans, parts_in, outs):
        sp.run(zi, steps, out=zo)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for sp, zi, zo in zip(seq_plans, parts_in, outs):
        sp.run(zi, steps, out=zo)
    e1.record()
    torch.cuda.synchronize()
    ts = e0.elapsed_time(e1) / 1e3
    same = all(torch.equal(a, b) for a, b in zip(outs, bp.unpack(zout)))
    rows["batch-256x(64..512)^2-5pt-rk4"] = {
        "gcups_batched": cells * steps / min(tb) / 1e9, "gcups_sequential": cells * steps / ts / 1e9,
        "speedup": ts / min(tb), "cells": cells, "steps_timed": steps, "bitwise_equal_to_sequential": same,
        "tuning": batch_tuning,
        "note": "rate of 200 of the 2000 steps; batched = one graph-replayed persistent launch, launch shape "
                "from the autotuner"}
    for sp in seq_plans:
        sp.close()
    bp.close()

    # differentiation workload: 512^2 two-field RK4 5-point.  Plain stepper,
    # 64 tangents in one tangent-linear run, and the checkpointed adjoint of
    # the full T = 2000 horizon, all in cell-updates per second.
    n = 512
    p = api.Problem(model=api.FHN, nx=n, ny=n, dx=0.04, scheme=api.RK4, dt=2.5e-4)
    plan = plan_cls(p)
    z = torch.from_numpy(I.fhn_broken_wave(n, n, seed=0)).cuda()
    T = 2000
    t_plain = timed(plan, z, T, reps=2)
    dz0 = torch.from_numpy(np.stack([I.unit_direction(z.shape, 2, offset=i * z.numel()) for i in range(64)])).cuda()
    steps_t = 200
    plan.tlm(z, dz0, steps_t)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    plan.tlm(z, dz0, steps_t)
    e1.record()
    torch.cuda.synchronize()
    t_tlm = e0.elapsed_time(e1) / 1e3
    plan.status()
    zT = plan.run(z, T)
    lamT = torch.zeros_like(zT)
    lamT[0] = 2.0 * zT[0]
    plan.adjoint(z, lamT, T)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    plan.adjoint(z, lamT, T)
    e1.record()
    torch.cuda.synchronize()
    t_adj = e0.elapsed_time(e1) / 1e3
    plan.status()
    # the same gradient split at the end of the forward run: the forward
    # keeps its checkpoints (cg_adjoint_forward), the backward sweeps back
    # from them (cg_adjoint_reverse) with no forward sweep of its own
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record()
    zT_ck, ck = plan.forward_checkpointed(z, T)
    e1.record()
    lam_ck, dd_ck = ck.adjoint(lamT)
    e2.record()
    torch.cuda.synchronize()
    t_fwd_ck, t_rev_ck = e0.elapsed_time(e1) / 1e3, e1.elapsed_time(e2) / 1e3
    lam_ref, dd_ref = plan.adjoint(z, lamT, T)
    split_same = bool(torch.equal(zT_ck, zT) and torch.equal(lam_ck, lam_ref) and torch.equal(dd_ck, dd_ref))
    plan.status()
    del ck, zT_ck, lam_ck, dd_ck, lam_ref, dd_ref
    # dL/dz0 alone (no dL/dD accumulation)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    plan.adjoint(z, lamT, T, with_dD=False)
    e1.record()
    torch.cuda.synchronize()
    t_adj_state = e0.elapsed_time(e1) / 1e3
    plan.status()
    # the same gradient keeping every stage input of the whole horizon in
    # HBM (one segment: no checkpoint sweep, no recomputation)
    import ctypes
    from paper_1309_1720_gb300 import _lib
    sz = ctypes.c_size_t()
    _lib.check(_lib.lib().cg_adjoint_workspace_size(plan.handle, T, T, ctypes.byref(sz)))
    plan.adjoint(z, lamT, T, checkpoint_every=T)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    plan.adjoint(z, lamT, T, checkpoint_every=T)
    e1.record()
    torch.cuda.synchronize()
    t_adj_all = e0.elapsed_time(e1) / 1e3
    plan.status()
    plan._ws = None
    torch.cuda.empty_cache()
    # one Newton step on the period-T flow map: GMRES(30), one restart cycle,
    # every Jacobian-vector product an exact tangent-linear run of T steps
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    dz_a, hist = plan.newton_step(z, T, restart=30, max_restarts=1, rtol=1e-10)
    torch.cuda.synchronize()
    t_newton = time.perf_counter() - t0
    # the same step with the stage Jacobians of the base trajectory stored
    # once (2000 x 4 stages x 1 plane) and every JVP a tangent-only run
    t0 = time.perf_counter()
    dz_b, hist_b = plan.newton_step(z, T, restart=30, max_restarts=1, rtol=1e-10, linearized=True)
    torch.cuda.synchronize()
    t_newton_lin = time.perf_counter() - t0
    newton_same = bool(torch.equal(dz_a, dz_b)) and hist == hist_b
    del dz_a, dz_b
    torch.cuda.empty_cache()
    g_plain = n * n * T / t_plain / 1e9
    rows["grad-512x512-5pt-rk4"] = {
        "gcups_plain": g_plain,
        "tlm_gcups_tangent_cells": 64 * n * n * steps_t / t_tlm / 1e9,
        "tlm_vs_plain": (64 * n * n * steps_t / t_tlm / 1e9) / g_plain,
        "adjoint_gcups": n * n * T / t_adj / 1e9,
        "adjoint_seconds_T2000": t_adj,
        "adjoint_vs_plain": (n * n * T / t_adj / 1e9) / g_plain,
        "adjoint_state_only_seconds_T2000": t_adj_state,
        "forward_checkpointed_seconds_T2000": t_fwd_ck,
        "adjoint_reverse_from_checkpoints_seconds_T2000": t_rev_ck,
        "forward_plus_reverse_seconds_T2000": t_fwd_ck + t_rev_ck,
        "split_bitwise_equal_to_adjoint_run": split_same,
        "adjoint_seconds_T2000_all_stages_stored": t_adj_all,
        "adjoint_all_stages_workspace_gb": sz.value / 1e9,
        "adjoint_all_stages_vs_plain": (n * n * T / t_adj_all / 1e9) / g_plain,
        "newton_gmres30_seconds": t_newton,
        "newton_gmres30_iterations": len(hist) - 1,
        "newton_gmres30_residual_reduction": hist[-1] / hist[0],
        "newton_gmres30_linearized_seconds": t_newton_lin,
        "newton_gmres30_linearized_bitwise_equal": newton_same,
        "note": "tlm: 64 tangents x 200 steps (rate); adjoint: full T = 2000 with ceil(sqrt(T)) checkpoints "
                "(forward + segment recompute + reverse sweep; state_only: dL/dz0 without dL/dD); split: a "
                "forward run keeping the checkpoints, then the segment recompute + reverse sweep from them "
                "(what an autograd backward costs), and with every stage input of the horizon "
                "kept in HBM (forward with stores + reverse sweep); newton: one GMRES(30) cycle on the "
                "T = 2000 flow map (wall time, 30 exact JVPs of 2000 steps each; linearized: stage "
                "Jacobians stored by one primal run, JVPs advance the tangent alone)"}
    plan.close()
    return rows


def _fit_slope(xs, ys):
    """Least-squares slope of log(ys) against log(xs)."""
    lx, ly = np.log(np.asarray(xs, float)), np.log(np.asarray(ys, float))
    return float(np.polyfit(lx, ly, 1)[0])


def paper_experiments(which):
    """The measurements of the paper's Sect. 5 on the GB300 stepper, for the
    three models of Sect. 2: wall time per unit of simulated time against dt
    (Fig. 3), against the grid size N (Fig. 4, with the crossover N0 of the
    fit tau = a max(1, b N^2)), relative L2 accuracy against dt with the
    observed orders (Fig. 5, Table 2), and cost against accuracy (Fig. 6).
    Prints one JSON line per experiment."""
    import torch
    from paper_1309_1720_gb300 import Plan, api, inputs as I

    def timed_step(plan, z, n, reps=3):
        out = torch.empty_like(z)
        plan.run(z, n, out=out)
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            plan.run(z, n, out=out)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        plan.status()
        return best / n

    names = {api.EULER: "euler", api.HEUN: "heun", api.RK4: "rk4", api.RUSH_LARSEN: "rush_larsen",
             api.IMPLICIT_EULER: "implicit_euler"}
    models = {
        "fhn": dict(prob=dict(model=api.FHN, dx=0.04), T=0.2, dts=[2e-4, 1e-4, 5e-5, 2.5e-5, 1.25e-5],
                    schemes=[api.EULER, api.HEUN, api.RK4],
                    ic=lambda n: I.fhn_broken_wave(n, n, seed=0)),
        "bocf": dict(prob=dict(model=api.BOCF, dx=0.03, D=(1.171e-3,)), T=10.0,
                     dts=[0.1, 0.05, 0.025, 0.0125, 0.00625],
                     schemes=[api.EULER, api.RUSH_LARSEN, api.IMPLICIT_EULER, api.HEUN, api.RK4],
                     ic=lambda n: I.bocf_spiral_cores(n, n, seed=0)),
        "karma": dict(prob=dict(model=api.KARMA, dx=I.KARMA_DX, D=(I.KARMA_GAMMA,)), T=10.0,
                      dts=[0.1, 0.05, 0.025, 0.0125, 0.00625],
                      schemes=[api.EULER, api.HEUN, api.RK4],
                      ic=lambda n: I.karma_broken_wave(n, n, seed=0)),
    }
    n = 256
    step_time = {}
    if which in ("all", "timing", "efficiency", "convergence"):
        res = {}
        for mname, m in models.items():
            z = torch.from_numpy(m["ic"](n)).cuda()
            res[mname] = {}
            for sc in m["schemes"]:
                plan = Plan(api.Problem(nx=n, ny=n, scheme=sc, dt=m["dts"][0], **m["prob"]))
                t = timed_step(plan, z, 2000)
                plan.close()
                step_time[(mname, sc)] = t
                res[mname][names[sc]] = {"us_per_step": 1e6 * t,
                                         "tau_at_dt": {str(dt): t / dt for dt in m["dts"]}}
            r = res[mname]
            r["heun_over_euler"] = r["heun"]["us_per_step"] / r["euler"]["us_per_step"]
            r["rk4_over_heun"] = r["rk4"]["us_per_step"] / r["heun"]["us_per_step"]
        if which in ("all", "timing"):
            print(json.dumps({"experiment": "timing_vs_dt (Fig. 3)", "grid": n, "steps_timed": 2000,
                              "tau": "device seconds per unit of simulated time = time per step / dt",
                              "results": res}), flush=True)
    grid_models = {
        "fhn 5-point": (dict(model=api.FHN, dx=0.04), 1e-4, lambda N: I.fhn_broken_wave(N, N, seed=0)),
        "karma 5-point": (dict(model=api.KARMA, dx=I.KARMA_DX, D=(I.KARMA_GAMMA,)), 0.05,
                          lambda N: I.karma_broken_wave(N, N, seed=0)),
    }
    for gname, (gprob, gdt, gic) in (grid_models.items() if which in ("all", "grid") else []):
        res = {}
        Ns = [32, 48, 64, 96, 128, 181, 256, 362, 512, 724, 1024, 1448, 2048, 2896, 4096]
        for sc in (api.EULER, api.HEUN, api.RK4):
            ts, tb = [], {}
            for N in Ns:
                prob = api.Problem(nx=N, ny=N, scheme=sc, dt=gdt, **gprob)
                plan = Plan(prob)
                z = torch.from_numpy(gic(N)).cuda()
                ts.append(timed_step(plan, z, 2000, reps=2) * 2000)
                plan.close()
                # temporally blocked (best of k = 2, 4, 8 steps per barrier) where it fits
                best = None
                if N <= 1024:
                    for k in (2, 4, 8):
                        for thr in (256, 512):
                            try:
                                tplan = Plan(prob, tuning=dict(schedule=2, rows=k, threads=thr))
                            except Exception:
                                continue
                            tk = timed_step(tplan, z, 2000, reps=2) * 2000
                            tplan.close()
                            if best is None or tk < best[0]:
                                best = (tk, k, thr)
                if best is not None:
                    tb[str(N)] = {"seconds": best[0], "k": best[1], "threads": best[2]}
                del z
            a = float(np.median(ts[:3]))
            b = float(np.median([t / N ** 2 for t, N in zip(ts, Ns) if N >= 2048]))
            a_tb = float(np.median([tb[str(N)]["seconds"] for N in Ns[:3]]))
            res[names[sc]] = {"seconds_2000_steps": dict(zip(map(str, Ns), ts)), "a_s": a, "b_s": b,
                              "N0": (a / b) ** 0.5,
                              "gcups_at_4096": 4096 ** 2 * 2000 / ts[-1] / 1e9,
                              "temporal_blocking": tb, "a_s_temporal_blocking": a_tb,
                              "N0_temporal_blocking": (a_tb / b) ** 0.5}
        print(json.dumps({"experiment": "time_vs_grid (Fig. 4)", "model": gname, "steps": 2000,
                          "fit": "t = a max(1, (N/N0)^2), a = median of N <= 64, b = a/N0^2 = median t/N^2 "
                                 "for N >= 2048", "results": res}), flush=True)
    if which in ("all", "small-grid"):
        # the 128^2 explicit-Euler workload with temporal blocking: steps per
        # pass, block size, and grid barrier or neighbour waits between
        # passes (best of five whole 1000-step runs; every shape must give
        # the stage kernel's result bit for bit)
        prob = dict(model=api.FHN, nx=128, ny=128, dx=0.04, scheme=api.EULER, dt=2e-4)
        z = torch.from_numpy(I.fhn_broken_wave(128, 128, seed=0)).cuda()
        ref = Plan(api.Problem(**prob)).run(z, 1000)
        res = []
        for flags, sync in ((0, "grid barrier"), (api.FLAG_NEIGHBOR_SYNC, "neighbour waits")):
            for k in (2, 3, 4, 6, 8):
                for thr in (128, 256, 512):
                    plan = Plan(api.Problem(flags=flags, **prob), tuning=dict(schedule=2, rows=k, threads=thr))
                    out = plan.run(z, 1000)
                    plan.status()
                    same = bool(torch.equal(out, ref))
                    t = timed_step(plan, z, 1000, reps=5)
                    plan.close()
                    res.append({"sync": sync, "steps_per_pass": k, "threads": thr, "us_per_step": 1e6 * t,
                                "bitwise_equal": same})
        res.sort(key=lambda r: r["us_per_step"])
        print(json.dumps({"experiment": "small grid: temporal blocking shapes (128^2 Euler, 1000 steps)",
                          "results": res}), flush=True)
    if which in ("all", "snapshots"):
        # Fig. 2: voltage fields of the three models on the paper's grids
        # (FHN 384^2, Karma 256^2, BOCF 768^2), RK4, reported as the range of
        # u over the run (the paper quotes about (-1, 1), (0, 3.5) and
        # (0, 1.55)) and whether activity is self-sustained at the end.  FHN
        # and BOCF start from the seeded states; Karma from an S1-S2 cross
        # field stimulus (a plane wave from the left edge, then the lower
        # half stimulated at 300 ms, exciting only recovered tissue), which
        # leaves a rotating spiral: its period is measured from the
        # upcrossings of u at the domain's centre over the last third.
        snaps = {
            "fhn": (api.Problem(model=api.FHN, nx=384, ny=384, dx=0.04, scheme=api.RK4, dt=2e-4),
                    I.fhn_broken_wave(384, 384, seed=0), 200.0, 0.0, None, 1.0),
            "karma": (api.Problem(model=api.KARMA, nx=256, ny=256, dx=I.KARMA_DX, D=(I.KARMA_GAMMA,),
                                  scheme=api.RK4, dt=0.05), np.zeros((2, 256, 256)), 3000.0, 1.0, 300.0, 1.0),
            "bocf": (api.Problem(model=api.BOCF, nx=768, ny=768, dx=0.03, D=(1.171e-3,), scheme=api.RK4,
                                 dt=0.05), I.bocf_spiral_cores(768, 768, seed=0), 2000.0, 0.5, None, 5.0),
        }
        res = {}
        for name, (prob, z0, T, thr, t_s2, every) in snaps.items():
            plan = Plan(prob)
            n = prob.nx
            z = torch.from_numpy(np.ascontiguousarray(z0)).cuda()
            if t_s2 is not None:
                z[0, :, :10] = 3.0                                   # S1
                z = plan.run(z, int(round(t_s2 / prob.dt)))
                z[0, : n // 2, :] = 3.0                              # S2
                t0 = t_s2
            else:
                t0 = 0.0
            n_chunk = int(round(every / prob.dt))                  # one sample per `every` time units
            chunks = int(round((T - t0) / prob.dt / n_chunk))
            umin, umax, excited, probe = float("inf"), -float("inf"), [], []
            for _ in range(chunks):
                z = plan.run(z, n_chunk)
                u = z[0]
                umin = min(umin, float(u.min()))
                umax = max(umax, float(u.max()))
                excited.append(float((u > thr).double().mean()))
                probe.append(float(u[n // 2, n // 2]))
            plan.status()
            last = max(2, chunks // 3)                              # the last third of the run
            tail_exc = excited[-last:]
            pr = np.array(probe[-last:])
            ups = np.nonzero((pr[:-1] <= thr) & (pr[1:] > thr))[0]
            period = float(np.mean(np.diff(ups)) * n_chunk * prob.dt) if len(ups) >= 3 else None
            res[name] = {"grid": [prob.nx, prob.ny], "T": T, "u_min": umin, "u_max": umax,
                         "excited_fraction_final": excited[-1],
                         "excited_fraction_range_last_third": [min(tail_exc), max(tail_exc)],
                         "self_sustained": bool(min(tail_exc) > 0.05),
                         "probe_upcrossings_last_third": int(len(ups)), "rotation_period": period,
                         "initial_state": "S1-S2 cross field" if t_s2 is not None else "seeded"}
            plan.close()
        print(json.dumps({"experiment": "voltage fields (Fig. 2)", "results": res}), flush=True)
    if which in ("all", "orbit"):
        # Sect. 1's use: a periodic orbit by Newton-Krylov.  A FitzHugh-Nagumo
        # pulse travelling round a periodic ring (512 x 2 cells, dx = 0.5)
        from paper_1309_1720_gb300.newton import periodic_orbit
        nx, ny, dt = 512, 2, 0.05
        base = api.Problem(model=api.FHN, nx=nx, ny=ny, dx=0.5, bc=api.PERIODIC, scheme=api.RK4, dt=dt)
        z = np.empty((2, ny, nx))
        z[0], z[1] = I.FHN_U_REST, I.FHN_V_REST
        z[0, :, 10:20] = 1.0
        z[1, :, 0:10] = 0.6
        z[1, :, -30:] = 0.6
        plan = Plan(base)
        zd = plan.run(torch.from_numpy(z).cuda(), 6000)

        def front(u):
            k = int(np.argmax(u))
            for j in range(u.size):
                a0, b0 = u[(k + j) % u.size], u[(k + j + 1) % u.size]
                if a0 >= 0.0 > b0:
                    return k + j + a0 / (a0 - b0)
            return float(k)
        x0 = front(zd[0, 0].cpu().numpy())
        zd = plan.run(zd, 2000)
        x1 = front(zd[0, 0].cpu().numpy())
        T0 = nx / (((x1 - x0) % nx) / (2000 * dt))
        n_steps = int(round(T0 / dt))
        torch.cuda.synchronize()
        t = time.perf_counter()
        _, T, hist = periodic_orbit(base, zd, T0, n_steps, tol=1e-12)
        torch.cuda.synchronize()
        print(json.dumps({"experiment": "periodic orbit by Newton-Krylov (Sect. 1)",
                          "system": "FitzHugh-Nagumo pulse on a periodic 512 x 2 ring, dx = 0.5, RK4, %d steps "
                                    "per period" % n_steps,
                          "T0": T0, "T": T, "seconds": time.perf_counter() - t, "newton": hist}), flush=True)
    if which in ("all", "convergence", "efficiency"):
        conv = {}
        for mname, m in models.items():
            z = torch.from_numpy(m["ic"](n)).cuda()
            T = m["T"]
            dref = m["dts"][-1] / 8
            ref_plan = Plan(api.Problem(nx=n, ny=n, scheme=api.RK4, dt=dref, **m["prob"]))
            ref = ref_plan.run(z, int(round(T / dref)))[0]
            ref_plan.status()
            conv[mname] = {}
            for sc in m["schemes"]:
                errs = []
                for dt in m["dts"]:
                    plan = Plan(api.Problem(nx=n, ny=n, scheme=sc, dt=dt, **m["prob"]))
                    u = plan.run(z, int(round(T / dt)))[0]
                    plan.status()
                    plan.close()
                    errs.append(float(torch.linalg.norm(u - ref) / torch.linalg.norm(ref)))
                use = [(d, e) for d, e in zip(m["dts"], errs) if e > 1e-13]
                alpha = _fit_slope(*zip(*use)) if len(use) >= 2 else None
                cost = [step_time[(mname, sc)] / d for d in m["dts"]]
                conv[mname][names[sc]] = {"dt": m["dts"], "Delta": errs, "alpha": alpha, "tau": cost}
            # cost of reaching Delta = 1e-7 from each method's power law
            target = 1e-7
            at = {}
            for sc in m["schemes"]:
                c = conv[mname][names[sc]]
                pts = [(d, e) for d, e in zip(c["dt"], c["Delta"]) if e > 1e-13]
                if c["alpha"] and len(pts) >= 2:
                    d0, e0 = pts[-1]
                    dt_t = d0 * (target / e0) ** (1.0 / c["alpha"])
                    at[names[sc]] = step_time[(mname, sc)] / dt_t
            conv[mname]["tau_at_Delta_1e-7"] = at
            if "rk4" in at:
                conv[mname]["rk4_speedup_at_1e-7"] = {k: v / at["rk4"] for k, v in at.items() if k != "rk4"}
        print(json.dumps({"experiment": "accuracy_vs_dt and cost_vs_accuracy (Figs. 5, 6, Table 2)",
                          "grid": n, "Delta": "relative L2 error of u against RK4 at dt/8 of the finest dt",
                          "T": {k: m["T"] for k, m in models.items()}, "results": conv}), flush=True)


def profile_case(args):
    """Short runs for ncu captures (run twice where a launch is captured
    after a warm one)."""
    import ctypes
    import torch
    from paper_1309_1720_gb300 import Plan, _lib, api, autotune, inputs as I
    case = args.profile_case
    if case == "fp64-probe":
        # the DFMA, DADD and DMUL rate probes at their default size (two
        # launches each: a warm-up half as long, then the timed one)
        L = _lib.lib()
        rate = ctypes.c_double()
        for op, name in ((0, "dfma"), (1, "dadd"), (2, "dmul"), (6, "dfma one lane per warp")):
            secs = ctypes.c_double()
            _lib.check(L.cg_measure_fp64_rate(op, 0, ctypes.byref(rate), ctypes.byref(secs)))
            print("%s %.4e per s (%.3f ms)" % (name, rate.value, 1e3 * secs.value))
        print("profile case done")
        return
    if case == "c1":
        cp = api.Problem(model=api.FHN, nx=128, ny=128, dx=0.04, scheme=api.EULER, dt=2e-4)
        plan = Plan(cp, tuning=dict(schedule=2, rows=4, threads=512))
        z = torch.from_numpy(I.fhn_broken_wave(128, 128, seed=0)).cuda()
        for _ in range(2):
            plan.run(z, 200)
        plan.status()
    elif case in ("tlm", "adj"):
        n = 512
        gp = api.Problem(model=api.FHN, nx=n, ny=n, dx=0.04, scheme=api.RK4, dt=2.5e-4)
        plan = Plan(gp)
        z = torch.from_numpy(I.fhn_broken_wave(n, n, seed=0)).cuda()
        for _ in range(2):
            if case == "tlm":
                dz0 = torch.from_numpy(np.stack([I.unit_direction(z.shape, 2, offset=i * z.numel())
                                                 for i in range(64)])).cuda()
                plan.tlm(z, dz0, 4)
            else:
                plan.adjoint(z, z.clone(), 16)
        plan.status()
    elif case == "fhn":
        # 1024^2 two-field 9-point RK4, 20 steps, its tuned launch shape
        n = 1024
        fp = api.Problem(model=api.FHN, nx=n, ny=n, dx=0.04, stencil=api.STENCIL9, alpha_d=1 / 6,
                         scheme=api.RK4, dt=4e-4)
        z = torch.from_numpy(I.fhn_broken_wave(n, n, seed=0)).cuda()
        plan = autotune.plan_for([fp], autotune.tune([fp], z, n_steps=200))
        out = torch.empty_like(z)
        for _ in range(2):
            plan.run(z, 20, out=out)
        plan.status()
    elif case == "karma":
        n = 2048
        kp = api.Problem(model=api.KARMA, nx=n, ny=n, dx=I.KARMA_DX, D=(I.KARMA_GAMMA,), scheme=api.RK4,
                         dt=0.05)
        z = torch.from_numpy(I.karma_broken_wave(n, n, seed=0)).cuda()
        plan = autotune.plan_for([kp], autotune.tune([kp], z, n_steps=10))
        out = torch.empty_like(z)
        for _ in range(2):
            plan.run(z, 10, out=out)
        plan.status()
    else:
        # the headline workload's plan in its tuned launch shape
        bp = headline_problem(api)
        z = torch.from_numpy(headline_state(I)).cuda()
        plan = autotune.plan_for([bp], autotune.tune([bp], z, n_steps=10))
        out = torch.empty_like(z)
        if case == "bocf":
            for _ in range(2):
                plan.run(z, 2, out=out)
        else:
            # one launch per branch of the local terms: uniform states whose
            # voltage puts every cell (so every warp) on that branch (rest:
            # u = 0; excited: u = 1; general: u = 0.2, between the w and v
            # switches), 2 steps each
            for u, v, w, s in ((0.0, 0.9, 0.8, 0.1), (1.0, 0.0, 0.5, 0.6), (0.2, 0.5, 0.6, 0.3)):
                zu = torch.empty_like(z)
                zu[0], zu[1], zu[2], zu[3] = u, v, w, s
                plan.run(zu, 2, out=out)
        plan.status()
    torch.cuda.synchronize()
    print("profile case done")


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.experiment:
        paper_experiments(args.experiment)
        return
    if args.profile_case:
        profile_case(args)
        return
    ws, rank, local = dist_env()
    import torch
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1309_1720_gb300 import Plan, api, autotune, inputs as I

    prob = headline_problem(api)
    z0_host = headline_state(I)
    z0 = torch.from_numpy(z0_host).cuda()
    # launch shape chosen by the project's autotuner on a short run of the
    # same workload (cached per GPU / model / size class)
    tuning = autotune.tune([prob], z0, n_steps=10)
    plan = autotune.plan_for([prob], tuning)
    out = torch.empty_like(z0)
    plan.workspace()

    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    cells = NX * NY * STEPS_PER_RUN

    peak_tflops, dfma_rate = measure_fp64_peak()

    for _ in range(args.warmup):
        plan.run(z0, STEPS_PER_RUN, out=out, stream=stream)
    plan.status()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    times = []
    with ClockSampler(local) as clk:
        barrier()
        t_wall = time.perf_counter()
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan.run(z0, STEPS_PER_RUN, out=out, stream=stream)
            e1.record(stream)
            times.append((e0, e1))
        barrier()
        t_wall = time.perf_counter() - t_wall
    plan.status()
    secs = [a.elapsed_time(b) / 1e3 for a, b in times]
    tot = max_over_ranks(sum(secs), ws)
    value = replica_throughput(cells * args.steps, ws, tot)
    launch_s = statistics.median(secs)

    # end to end through the C ABI with host buffers (cg_run_host): each
    # step copies the state in from pinned host memory, runs, copies the
    # result out and reads the device status word back
    e2e_steps = min(args.steps, 3)
    h_in = torch.from_numpy(z0_host).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    plan.run_host(h_in, 1, out=h_out, stream=stream)
    barrier()
    e2e_t = []
    for _ in range(e2e_steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.run_host(h_in, STEPS_PER_RUN, out=h_out, stream=stream)
        e1.record(stream)
        e2e_t.append((e0, e1))
    barrier()
    e2e_tot = max_over_ranks(sum(a.elapsed_time(b) / 1e3 for a, b in e2e_t), ws)
    nbytes = z0.numel() * 8
    del h_in, h_out

    # branch mix of the local terms over one whole run (outside the timed
    # region): the voltage of every cell every 250 steps, classified by its
    # switch state
    params = api.default_params(api.BOCF)
    lo, hi = bocf_branch_bounds(params)
    every = 250
    counts = {"rest": 0, "excited": 0}
    n_seen = 0
    zc = z0.clone()
    zn = torch.empty_like(zc)
    for _ in range(STEPS_PER_RUN // every):
        counts["rest"] += int((zc[0] <= lo).sum())
        counts["excited"] += int((zc[0] >= hi).sum())
        n_seen += zc[0].numel()
        plan.run(zc, every, out=zn, stream=stream)
        zc, zn = zn, zc
    plan.status()
    mix = {"rest": counts["rest"] / n_seen, "excited": counts["excited"] / n_seen}
    mix["general"] = 1.0 - mix["rest"] - mix["excited"]
    del zc, zn
    flops_cu = bocf_flops_per_cell_update(mix)
    achieved_tflops = flops_cu * cells / launch_s / 1e12

    rows = None
    if not args.no_rows and rank == 0:
        rows = secondary_rows(torch, Plan, I, api, peak_tflops, tuning)
    cpu = None
    if not args.no_cpu and rank == 0 and args.gpus == 1:
        cpu = cpu_baseline()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GCUPS", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(),
            "roofline": {"bound": "alu", "achieved": achieved_tflops, "peak": peak_tflops, "unit": "TFLOP/s",
                         "frac": achieved_tflops / peak_tflops,
                         "traffic": MEASURED_DRAM_BYTES_PER_CELL_UPDATE * cells,
                         "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of a 2-step launch of "
                                           "this workload in its tuned launch shape (508.8 B per cell-update), "
                                           "scaled to the 5000-step launch; the kernel is bound by the FP64 pipe, "
                                           "not HBM",
                         "peak_source": "measured FP64 DFMA throughput of this GPU (library probe, 8 chains x "
                                        "256 threads x 4 blocks/SM), FMA = 2 flops",
                         "flops_per_cell_update": flops_cu,
                         "flops_per_stage_by_branch": BOCF_STAGE_FLOPS,
                         "branch_mix": mix,
                         "branch_mix_sample": "voltage of all cells every %d steps of one whole run" % every,
                         "hbm_bytes_per_cell_update": BYTES_PER_CELL_UPDATE,
                         "hbm_achieved_gbs": BYTES_PER_CELL_UPDATE * cells / launch_s / 1e9,
                         "kernel": "k_stage<BOCF, 9-point anisotropic, RK4> (persistent)", "tuning": tuning},
            "e2e": {"value": ws * cells * e2e_steps / e2e_tot / 1e9, "unit": "GCUPS",
                    "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes + 4, "steps": e2e_steps,
                    "call": "cg_run_host (pinned host state in and out, status word read back)"},
            "gpu_launches": args.steps,
            "clocks": clk.summary(),
            "wall_s_timed": t_wall,
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
        if rows is not None:
            line["rows"] = rows
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
