#!/usr/bin/env python
"""Benchmark of the MLVS-DUGKS hot path: cell-velocity updates per second on one B300.

Workload (N = 1): the 2-D lid-driven cavity, 64 x 64 cells, Kn = 0.075, lid Mach 0.16,
Shakhov Pr = 2/3, on the 101 x 101 Boole velocity grid over [-6, 6]^2 (UVS), f stored in
FP32 with FP64 moment sums.  One step is one DUGKS step over every (cell, velocity) pair.
The distributions (2 x 334 MB) are larger than L2, so no flush is needed between steps.

value: UVS cell-velocity updates/s over K timed steps.  Beside it:
  mlvs            the same cavity with multi-level velocity spaces (criterion, grouping and
                  remap every 100 steps inside the timed region, Sec. 3.2 / Sec. 4 settings)
  time_to_steady  UVS and MLVS from rest until the residual falls below 1e-6 (at most
                  10,000 steps), their device times, and the MLVS fields' relative L2
                  difference from the UVS fields (the "same error" check)

Arms:
  (default)          the CUDA library through its C ABI
  --impl reference   the FP64 CPU oracle as it stands, on the host cores, on a bounded
                     sample of the same workload (a smaller cavity on the same velocity grid)

Multi-GPU: the path is run as independent replicas (one cavity per rank, no collective on
the data path); value = all ranks' updates / max-over-ranks time, scaling "weak".
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# the oracle baseline runs on one host thread (numpy elementwise; no threaded BLAS)
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

METRIC = "cell-velocity updates/s & time-to-steady, MLVS vs UVS on 1 B300, same error"
UNIT = "updates/s"

# DRAM bytes per launch of the dominant kernel from one ncu capture, keyed by workload, with
# the hash of the tile-kernel sources at capture time (a changed kernel reports null).
TRAFFIC = {"cavity64_uvs101_f32:face_sums": (355803648 + 657018624, "349dc532daf9")}
TILE_SOURCES = ("dugks_tile.cuh", "mlvs_common.cuh")


def kernel_source_hash():
    """Hash of the sources the tile kernels (face sums and update) are compiled from."""
    h = hashlib.sha1()
    d = os.path.join(ROOT, "paper_2609_35258_b300", "csrc")
    for f in TILE_SOURCES:
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_rate(ncell_side, nsteps, threads=1):
    """FP64 oracle on a ncell_side^2 cavity with the bench's velocity grid; updates/s."""
    from paper_2609_35258_b300 import workloads
    from tests.helpers import oracle_run, oracle_setup
    d = workloads.cavity(ncell_side, n_base=101, umax=6.0, Kn=0.075)
    o = oracle_setup(d)
    t0 = time.perf_counter()
    oracle_run(o, nsteps)
    t = time.perf_counter() - t0
    upd = ncell_side * ncell_side * 101 * 101 * nsteps
    return upd / t, t, upd


def _oracle_worker(args):
    side, nsteps = args
    return oracle_rate(side, nsteps)


def oracle_rate_all_cores(side, nsteps, procs=None):
    """The oracle as it stands on every host core: one independent oracle run per process
    (spawned, so that no CUDA state is inherited), each one thread.  Aggregate updates/s."""
    import multiprocessing as mp
    procs = procs or os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        pool.map(_oracle_worker, [(2, 1)] * procs)          # start-up (imports) outside the timing
        t0 = time.perf_counter()
        res = pool.map(_oracle_worker, [(side, nsteps)] * procs)
        t = time.perf_counter() - t0
    upd = sum(r[2] for r in res)
    return upd / t, t, upd, procs


def run_reference(args, rank):
    if rank != 0:
        return
    # sample size so that (K + W) oracle steps take about 1-2 minutes
    per_upd = 1.1e-6
    cells = 100.0 / ((args.steps + args.warmup) * 101 * 101 * per_upd)
    side = int(max(2, min(16, math.floor(math.sqrt(max(cells, 4.0))))))
    from paper_2609_35258_b300 import workloads
    from tests.helpers import oracle_run, oracle_setup
    d = workloads.cavity(side, n_base=101, umax=6.0, Kn=0.075)
    o = oracle_setup(d)
    for _ in range(args.warmup):
        g, h = oracle_run(o, 1)
        o["g"], o["h"] = g, h
    t0 = time.perf_counter()
    for _ in range(args.steps):
        g, h = oracle_run(o, 1)
        o["g"], o["h"] = g, h
    t = time.perf_counter() - t0
    upd = side * side * 101 * 101 * args.steps
    val = upd / t
    sample = f"{side}x{side}-cell cavity on the same 101^2 velocity grid, {args.steps} oracle steps"
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "cavity64_uvs101_f32", "sample": sample},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# MLVS settings of the cavity runs (Sec. 4): C_split, C_merge, eps_merge, tau_clust, the
# coarsest candidate block (level 2: the 101^2 / 51^2 / 25^2 quadtree depths), interval.
MLVS_PARAMS = (5e-3, 2.5e-3, 5e-5, 0.05, 2)
ADAPT_INTERVAL = 100
STEADY_TOL = 1e-6        # max over rho, u, v, T of |W^n - W^(n-100)|_2 / |W^n|_2
STEADY_MAX = 10000       # the paper's cavity runs stop at 10,000 steps


def _steady(desc, stream, mlvs):
    """Steps (100 at a time, as two-step CUDA graphs) until the residual falls below STEADY_TOL;
    device time."""
    from paper_2609_35258_b300 import mlvs as M
    from paper_2609_35258_b300.solver import Solver
    import numpy as np
    s = Solver(desc, stream=stream, adaptive=1)
    M.mlvs_set_graph(s.h, True)                 # both runs as two-step CUDA graphs
    if mlvs:
        M.mlvs_set_adaptation(s.h, M.adapt_params(*MLVS_PARAMS), ADAPT_INTERVAL)
    F = M.RHO | M.U | M.V | M.T
    prev = s.moments(F)
    ms, steps, res, upd = 0.0, 0, 1.0, 0
    while steps < STEADY_MAX:
        st = s.step(100)
        ms += st.ms_total
        upd += st.cell_velocity_updates
        steps += 100
        m = s.moments(F)
        res = max(float(np.linalg.norm(m[i] - prev[i]) / np.linalg.norm(m[i])) for i in range(4))
        prev = m
        if res < STEADY_TOL:
            break
    out = s.moments(M.RHO | M.U | M.V | M.T | M.QX | M.QY)
    s.close()
    return {"steps": steps, "seconds": ms / 1e3, "residual": res, "converged": res < STEADY_TOL,
            "updates": upd}, out


def _selector_leg(kns=(0.01, 0.1, 1.0), snaps=20, every=20, held=4, epochs=300, conf=0.9, warm=200,
                  interval=100):
    """The level selector on the Ma 5 cylinder (O-grid 256 x 128, base 201^2 on [-15, 15]^2, FP32,
    smooth start) with the four uniform levels 201^2 / 101^2 / 51^2 / 25^2 and the paper's
    cylinder criterion (C_split 0.01, C_merge 0.005).  Labels: the fixed-level-set rule on the
    criterion's masks for every cell of `snaps` snapshots, `every` steps apart, of one UVS run
    per Knudsen number in `kns`; features: the library's ten cell features.  The last `held`
    snapshots of every run are held out; the network trains on the rest (full batch, SGD with
    momentum, on the GPU).  In the solve: two runs at Kn 0.1 take `warm` UVS steps, then adapt
    every `interval` steps up to step snaps * every, one with the criterion, one with the
    selector (the criterion on the cells below confidence `conf`); both are compared with the
    UVS run at Kn 0.1 (the training run, which never adapts) at that step."""
    import numpy as np
    import torch
    from paper_2609_35258_b300 import mlvs as M
    from paper_2609_35258_b300 import workloads
    from paper_2609_35258_b300.solver import Solver
    nt, nr = 256, 128
    n = nt * nr
    levels = [0, 1, 2, 3]
    p = M.adapt_params(0.01, 0.005, 0.0, 0.05, 3)
    F = M.RHO | M.T
    Xtr, ytr, Xho, yho = [], [], [], []
    t_label, ref = 0.0, None
    for Kn in kns:
        s = Solver(workloads.cylinder(nt, nr, Kn=Kn, storage="f32", start="ramp"), levels=levels, adaptive=0)
        M.mlvs_set_graph(s.h, True)
        for k in range(snaps):
            s.step(every)
            t0 = time.perf_counter()
            X = M.mlvs_features(s.h, 0, n)
            y = M.mlvs_criterion_levels(s.h, 0, p, n)
            t_label += time.perf_counter() - t0
            (Xtr if k < snaps - held else Xho).append(X)
            (ytr if k < snaps - held else yho).append(y)
        if Kn == 0.1:
            ref = s.moments(F)
        s.close()
    X, y = np.concatenate(Xtr), np.concatenate(ytr)
    Xh, yh = np.concatenate(Xho), np.concatenate(yho)
    m = M.mlvs_mlp_create()
    M.mlvs_mlp_set_weights(m, workloads.selector_init())
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    first = last = M.mlvs_mlp_train_step(m, Xd, yd, len(y), 0.02, 0.9)
    for _ in range(epochs - 1):
        last = M.mlvs_mlp_train_step(m, Xd, yd, len(y), 0.02, 0.9)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    prob = torch.zeros(len(yh), 4, device="cuda")
    M.mlvs_mlp_forward(m, torch.from_numpy(Xh).cuda(), len(yh), None, prob)
    pr = prob.cpu().numpy()
    pred, top = np.argmax(pr, 1), np.max(pr, 1)
    sure = top >= conf
    out = {"workload": f"cylinder O-grid {nt}x{nr}, Ma 5, base 201^2 on [-15,15]^2, FP32, smooth start, "
                       f"uniform levels 201^2/101^2/51^2/25^2", "network": "10-64-64-4 ReLU, BF16 weights, FP32 accumulation",
           "kn": list(kns), "train_samples": int(len(y)), "heldout_samples": int(len(yh)),
           "label_counts": np.bincount(np.concatenate([y, yh]), minlength=4).tolist(),
           "label_seconds": t_label, "epochs": epochs, "train_seconds": t_train,
           "loss_first": first, "loss_last": last,
           "heldout_accuracy": float(np.mean(pred == yh)),
           "heldout_confident_fraction": float(np.mean(sure)),
           "heldout_confident_accuracy": float(np.mean(pred[sure] == yh[sure])) if sure.any() else None,
           "confidence": conf, "solve": {}}
    for mode in ("criterion", "selector"):
        s = Solver(workloads.cylinder(nt, nr, Kn=0.1, storage="f32", start="ramp"), levels=levels, adaptive=0)
        M.mlvs_set_graph(s.h, True)
        s.step(warm)
        ta, ts, fb, pts = [], 0.0, [], []
        try:
            for _ in range((snaps * every - warm) // interval):
                if mode == "criterion":
                    a = M.mlvs_adapt(s.h, p)
                else:
                    a = M.mlvs_adapt_mlp(s.h, m, p, conf)
                    fb.append(int(a.n_distinct))
                ta.append(a.ms_total)
                pts.append(a.updates_per_step / n)
                ts += s.step(interval).ms_total
            mo = s.moments(F)
            out["solve"][mode] = {"adapt_ms": ta, "mean_points_per_cell": pts,
                                  "ms_per_step": ts / (snaps * every - warm),
                                  "rel_l2_vs_uvs": {"rho": _l2(mo[0], ref[0]), "T": _l2(mo[1], ref[1])},
                                  "levels": np.bincount(s.moments(M.LEVEL)[0].astype(int), minlength=4).tolist()}
            if fb:
                out["solve"][mode]["fallback_cells"] = fb
        except M.MLVSError as e:
            out["solve"][mode] = {"error": str(e)}
        s.close()
    M.mlvs_mlp_destroy(m)
    c, q = out["solve"].get("criterion", {}), out["solve"].get("selector", {})
    if "adapt_ms" in c and "adapt_ms" in q:
        out["adapt_speedup"] = float(np.sum(c["adapt_ms"]) / np.sum(q["adapt_ms"]))
        tc = np.sum(c["adapt_ms"]) + c["ms_per_step"] * (snaps * every - warm)
        tq = np.sum(q["adapt_ms"]) + q["ms_per_step"] * (snaps * every - warm)
        out["end_to_end_speedup"] = float(tc / tq)
    return out


def _cylinder_leg(storage="f32", warm_steps=300, run_steps=300, taus=(1.0, 0.07, 0.05, 0.04, 0.035),
                  positive_mapping=0):
    """Ma 5 flow past a cylinder (O-grid 256 x 128, Kn 0.1, base 201^2 on [-15, 15]^2), from the
    smooth start of `workloads.cylinder(start="ramp")` (speed rising from the wall over two
    radii at the freestream's total enthalpy and pressure).  UVS runs first and keeps its fields
    at the comparison step.  MLVS then starts from the same initial state and, after
    `warm_steps` steps on the full space, runs the paper's setting (C_split 0.01, C_merge 0.005, tau_clust 0.05, up to four depths, spaces
    rebuilt every 100 steps) with the transport test on (eps_merge 5e-5, the cavity's value; the
    paper gives none for the cylinder) for `run_steps` steps; its fields are compared with UVS at
    the same step.  Afterwards the same state is adapted with each clustering threshold in turn and timed
    for 50 steps.  A failing MLVS step is reported in the result instead of ending the benchmark.
    positive_mapping = 1 gives the level switches the exponential fallback (Sec. 3.3.2)."""
    import numpy as np
    from paper_2609_35258_b300 import mlvs as M, workloads
    from paper_2609_35258_b300.solver import Solver
    nt, nr = 256, 128
    d = workloads.cylinder(nt, nr, storage=storage, start="ramp")
    F = M.RHO | M.U | M.V | M.T | M.QX | M.QY
    u = Solver(d)
    M.mlvs_set_graph(u.h, True)
    u.step(warm_steps)
    su = u.step(run_steps)
    uvs_ms = su.ms_total / run_steps
    nv = su.cell_velocity_updates / run_steps / (nt * nr)
    mu = u.moments(F)
    u.close()
    out = {"workload": f"cylinder O-grid {nt}x{nr}, Ma 5, Kn 0.1, base 201^2 on [-15,15]^2, {storage}, "
                       f"smooth start",
           "uvs_ms_per_step": uvs_ms, "uvs_points_per_cell": nv, "adapt_from_step": warm_steps,
           "run": None, "tau_sweep": []}
    s = Solver(d, adaptive=1, positive_mapping=positive_mapping)
    out["positive_mapping"] = positive_mapping
    M.mlvs_set_graph(s.h, True)
    try:
        s.step(warm_steps)
        p = M.adapt_params(0.01, 0.005, 5e-5, 0.05, 3)
        a = M.mlvs_adapt(s.h, p)
        M.mlvs_set_adaptation(s.h, p, 100)
        sm = s.step(run_steps)
        ms = s.moments(F)
        out["run"] = {"tau_clust": 0.05, "eps_merge": 5e-5, "adapt_interval": 100, "steps": run_steps,
                      "compared_at_step": warm_steps + run_steps, "spaces_first": a.n_levels,
                      "adapt_ms_first": a.ms_total,
                      "exp_corrected_first": a.n_exp_corrected, "exp_failed_first": a.n_exp_failed,
                      "cross_fraction_first": a.n_cross_faces / max(1, a.n_interior_faces),
                      "mean_points_per_cell_first": a.updates_per_step / (nt * nr),
                      "mlvs_ms_per_step": sm.ms_total / run_steps, "uvs_ms_per_step": uvs_ms,
                      "speedup_vs_uvs": uvs_ms / (sm.ms_total / run_steps),
                      "rel_l2_vs_uvs": {"rho": _l2(ms[0], mu[0]),
                                        "u": _l2(np.hypot(ms[1], ms[2]), np.hypot(mu[1], mu[2])),
                                        "T": _l2(ms[3], mu[3]),
                                        "q": _l2(np.hypot(ms[4], ms[5]), np.hypot(mu[4], mu[5]))}}
        M.mlvs_set_adaptation(s.h, p, 0)
        for tau in taus:
            a = M.mlvs_adapt(s.h, M.adapt_params(0.01, 0.005, 0.0, tau, 3))
            s.step(2)
            sm = s.step(50)
            out["tau_sweep"].append({"tau_clust": tau, "spaces": a.n_levels, "distinct_masks": a.n_distinct,
                                     "mean_points_per_cell": a.updates_per_step / (nt * nr),
                                     "cross_faces": a.n_cross_faces, "interior_faces": a.n_interior_faces,
                                     "ms_per_step": sm.ms_total / 50, "speedup_vs_uvs": uvs_ms / (sm.ms_total / 50),
                                     "adapt_ms": a.ms_total})
        # the paper's runtime model t/t_UVS ~ r + lambda_cross f + c, calibrated on this sweep
        from paper_2609_35258_b300 import runtime_model as RM
        sw = out["tau_sweep"]
        r = [x["mean_points_per_cell"] / nv for x in sw]
        f = [x["cross_faces"] / max(1, x["interior_faces"]) for x in sw]
        m = RM.fit(r, f, [x["ms_per_step"] / uvs_ms for x in sw])
        out["runtime_model"] = {"lambda_cross": m["lambda_cross"], "c": m["c"], "r2": m["r2"],
                                "r": r, "f": f, "t_rel": [x["ms_per_step"] / uvs_ms for x in sw],
                                "t_rel_model": [float(v) for v in m["t_rel_model"]],
                                "update_term_at_interval_100": out["run"]["adapt_ms_first"] / (100.0 * uvs_ms)}
    except M.MLVSError as e:
        out["error"] = str(e)
    s.close()
    return out


def _sod_leg(steps=500):
    """The 1-D shock tube (200 cells, 101 velocities on [-10, 10], FP64, BGK, Kn 1e-3, CFL 0.5):
    device time per step over `steps` steps replayed as two-step CUDA graphs, and launched one
    kernel at a time, with the host's wall time per step beside each."""
    import time
    from paper_2609_35258_b300 import mlvs as M, workloads
    from paper_2609_35258_b300.solver import Solver
    d = workloads.sod_1d()
    out = {"workload": "Sod shock tube, 200 cells, 101 velocities on [-10,10], FP64, BGK, Kn 1e-3, CFL 0.5",
           "steps": steps}
    for graph in (True, False):
        s = Solver(d)
        M.mlvs_set_graph(s.h, graph)
        s.step(10)                                  # warm: tables, graph capture
        t0 = time.perf_counter()
        st = s.step(steps)
        wall = (time.perf_counter() - t0) / steps
        rho = s.moments(M.RHO)[0]
        out["graph" if graph else "eager"] = {"ms_per_step": st.ms_total / steps, "wall_ms_per_step": 1e3 * wall,
                                              "launches_per_step": st.launches / steps,
                                              "updates_per_s": st.cell_velocity_updates / (st.ms_total / 1e3)}
        out["rho_range"] = [float(rho.min()), float(rho.max())]
        s.close()
    return out


def _batch_leg(n_inst=64, warm=50, steps=40):
    """Independent lid-driven cavities (Kn log-uniform in [1e-3, 10], sizes drawn from 32^2 ..
    128^2, 101^2 base grid, FP32), each adapting on its own (the cavity thresholds, up to two
    coarsening depths: spaces between 101^2 and 25^2 points, rebuilt every `warm` steps).  After
    `warm` steps and the first adaptation, `steps` steps of the whole group run as one graph per
    two steps (mlvs_step_many; every instance's tile passes are level-batched launches), then
    the same steps one handle after another."""
    import time
    import torch
    from paper_2609_35258_b300 import mlvs as M, workloads
    from paper_2609_35258_b300.solver import Solver
    descs = workloads.batched_cavities(n_inst)
    ss = [Solver(d, adaptive=1) for d in descs]
    hs = [s.h for s in ss]
    p = M.adapt_params(5e-3, 2.5e-3, 5e-5, 0.05, 2)
    for s in ss:
        M.mlvs_set_adaptation(s.h, p, warm)
    out = {"workload": f"{n_inst} cavities, Kn log-uniform [1e-3, 10], sizes 32^2..128^2, base 101^2, FP32, "
                       f"adaptive (spaces 101^2..25^2)",
           "instances": n_inst, "cells": int(sum(d["nx"] * d["ny"] for d in descs))}
    try:
        M.mlvs_step_many(hs, warm + 2, use_graph=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = M.mlvs_step_many(hs, steps, use_graph=True)
        torch.cuda.synchronize()
        tb = time.perf_counter() - t0
        upd = st.cell_velocity_updates
        t0 = time.perf_counter()
        for h in hs:
            M.mlvs_step(h, steps)
        torch.cuda.synchronize()
        ts = time.perf_counter() - t0
        out.update({"steps": steps, "updates_per_step": upd / steps,
                    "mean_points_per_cell": upd / steps / out["cells"],
                    "batched": {"ms_per_step": 1e3 * tb / steps, "updates_per_s": upd / tb,
                                "launches_per_step": st.launches / steps},
                    "one_by_one": {"ms_per_step": 1e3 * ts / steps, "updates_per_s": upd / ts},
                    "batching_gain": ts / tb})
    except M.MLVSError as e:
        out["error"] = str(e)
    for s in ss:
        s.close()
    return out


def _unstructured_leg(storage="f32", m=10, n_base=101, umax=6.0, steps=50, warm=5):
    """Two connected cavities (13,600 quads for m = 10; the paper's mesh has 12,012 cells)
    with the paper's density ratio of 1000, gas at rest at T = 1, closed walls at T = 1, one
    velocity space of n_base^2 points: device time per step of the unstructured step and its
    cell-velocity update rate, plus the mass drift over the timed steps."""
    import numpy as np
    from paper_2609_35258_b300 import mlvs as M, workloads
    nodes, cells = workloads.two_cavities(m)
    geo = M.mlvs_umesh_geometry(nodes, cells)
    nc = len(cells)
    W0 = np.zeros((nc, 4))
    W0[:, 0] = np.where(geo["cx"] < 0.0, 1.0, 1e-3)
    W0[:, 3] = 1.0
    c = M.mlvs_uconfig()
    c.storage = {"f32": M.F32, "f64": M.F64}[storage]
    c.R, c.K_internal, c.Pr, c.omega, c.T_ref = 1.0, 0.0, 2.0 / 3.0, 0.81, 1.0
    c.mu_ref, c.Kn = 0.0, 0.05
    c.cfl, c.dt = 0.5, 0.0
    c.compat_cell = c.compat_face = 1
    c.limiter = M.LIMITER_VENKAT
    c.n_base, c.umin, c.umax, c.quadrature = n_base, -umax, umax, M.QUAD_BOOLE
    c.n_wall = 1
    c.wall[0][0], c.wall[0][1], c.wall[0][2] = 0.0, 0.0, 1.0
    c.vpc = 64
    out = {"workload": f"two cavities, {nc} quads, {n_base}^2 velocities on [-{umax:g},{umax:g}]^2, "
                       f"density ratio 1000, {storage}", "cells": nc, "faces": len(geo["L"])}
    h = M.mlvs_ucreate(c, nodes, cells, W0)
    try:
        M.mlvs_ustep(h, warm)
        W1 = M.mlvs_ucells(h, nc)
        ms = M.mlvs_ustep(h, steps)
        M.mlvs_ustep(h, 1)
        W2 = M.mlvs_ucells(h, nc)
        nv = M.mlvs_uinfo(h)[0]
        m1, m2 = np.sum(geo["area"] * W1[0]), np.sum(geo["area"] * W2[0])
        out.update({"ms_per_step": ms / steps, "velocities": nv,
                    "updates_per_s": nc * nv * steps / (ms * 1e-3), "steps": steps,
                    "rel_mass_drift": abs(m2 - m1) / m1,
                    "launches_per_step": 7,
                    # DRAM traffic per update measured with ncu on two_cavities(4) in FP32
                    "hbm_bytes_per_update_measured": 152 if storage == "f32" else None,
                    "algorithmic_bytes_per_update": 16 if storage == "f32" else 32})
    except M.MLVSError as e:
        out["error"] = str(e)
    finally:
        M.mlvs_udestroy(h)
    return out


def _unstructured_isolated(timeout=600):
    """The two-cavity unstructured leg in a child process (its own CUDA context), so that a
    failure there cannot end this benchmark: its JSON result, or the reason it has none."""
    cmd = [sys.executable, "-c", "import json, bench; print('UNSTRUCTURED ' + json.dumps(bench._unstructured_leg()))"]
    try:
        r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=timeout)
    except subprocess.TimeoutExpired:
        return {"error": f"no result within {timeout} s"}
    for line in r.stdout.splitlines():
        if line.startswith("UNSTRUCTURED "):
            return json.loads(line[len("UNSTRUCTURED "):])
    return {"error": f"exit {r.returncode}: " + (r.stderr.strip().splitlines() or ["no output"])[-1][:300]}


def combine_ranks(ms, world, upd_step, steps, device="cuda"):
    """The timed region's length as the maximum over ranks (every rank waits at a barrier
    afterwards) and the whole-job throughput: the updates of all ranks over that time."""
    if world > 1:
        import torch
        import torch.distributed as tdist
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        ms = float(t.item())
        tdist.barrier()
    return ms, world * upd_step * steps / (ms / 1e3)


def _l2(a, b):
    import numpy as np
    return float(np.sqrt(np.sum((a - b) ** 2)) / np.sqrt(np.sum(b ** 2)))


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    torch.cuda.set_device(local_rank)
    from paper_2609_35258_b300 import mlvs as M
    from paper_2609_35258_b300 import workloads
    from paper_2609_35258_b300.solver import Solver

    dist = world > 1
    if dist:
        import torch.distributed as tdist
    stream = torch.cuda.current_stream()
    n = args.cells
    desc = workloads.cavity(n, n_base=101, umax=6.0, Kn=0.075, storage=args.storage)
    ncell = n * n
    nv = 101 * 101
    upd_step = ncell * nv
    s = Solver(desc, stream=stream.cuda_stream)
    M.mlvs_set_graph(s.h, True)                 # two-step CUDA graphs (per-phase runs launch eagerly)
    s.step(args.warmup)
    torch.cuda.synchronize()
    if dist:
        tdist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local_rank)
    clk.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st = s.step(args.steps)          # the headline: no per-launch events in the timed region
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms, value = combine_ranks(e0.elapsed_time(e1), world, upd_step, args.steps)
    torch.cuda.synchronize()
    ms_step = ms / args.steps

    # per-phase times from a second run of the same steps with CUDA events around every
    # launch (on the handle's stream), and the roofline of the dominant kernel from them
    stp = s.step(args.steps, profile=True)
    torch.cuda.synchronize()
    phases = list(stp.ms_phase)
    names = ["finalize_cells", "face_sums", "finalize_faces", "update", "ghost_map", "flux_map"]
    dom = max(range(len(names)), key=lambda i: phases[i])
    fbytes = {"f32": 4, "bf16": 2, "f64": 8}[args.storage]
    algo_per_update = {1: 2 * fbytes, 3: 4 * fbytes}.get(dom, 0)
    kernel_ms = phases[dom] / args.steps
    peak, peak_kind = measured_peaks()
    achieved = algo_per_update * upd_step / (kernel_ms / 1e3) / 1e9 if algo_per_update else None
    wl = f"cavity{n}_uvs101_{args.storage}"
    key = f"{wl}:{names[dom]}"
    tr = TRAFFIC.get(key)
    traffic = tr[0] if tr and tr[1] == kernel_source_hash() else None
    s.close()

    # MLVS on the same cavity: adapt after the warm-up, then K steps with adaptation every
    # ADAPT_INTERVAL steps inside the timed region
    mlvs = None
    if not args.no_mlvs:
        sm_ = Solver(desc, stream=stream.cuda_stream, adaptive=1)
        M.mlvs_set_graph(sm_.h, True)
        sm_.step(max(args.warmup, 200))
        ast = M.mlvs_adapt(sm_.h, M.adapt_params(*MLVS_PARAMS))
        M.mlvs_set_adaptation(sm_.h, M.adapt_params(*MLVS_PARAMS), ADAPT_INTERVAL)
        sm_.step(args.warmup)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        mst = sm_.step(args.steps)
        f1.record(stream)
        torch.cuda.synchronize()
        mms = f0.elapsed_time(f1)
        mupd = mst.cell_velocity_updates
        mstp = sm_.step(args.steps, profile=True)     # per-phase times, a second run
        torch.cuda.synchronize()
        # one more adaptation of the developed state, as the periodic ones inside the run
        rst = M.mlvs_adapt(sm_.h, M.adapt_params(*MLVS_PARAMS))
        mlvs = {"ms_per_step": mms / args.steps, "updates_per_s": mupd / (mms / 1e3),
                "points_per_cell": mupd / args.steps / ncell, "levels": mst.n_levels,
                "speedup_per_step_vs_uvs": ms_step / (mms / args.steps),
                "adapt_ms": ast.ms_total, "criterion_ms": ast.ms_criterion,
                "readapt_ms": {"total": rst.ms_total, "criterion": rst.ms_criterion,
                               "grouping": rst.ms_group, "remap": rst.ms_remap,
                               "cells_moved": rst.n_changed},
                "phases_ms_per_step": {n: p / args.steps for n, p in zip(names, mstp.ms_phase)},
                "includes": f"adaptation every {ADAPT_INTERVAL} steps"}
        sm_.close()

    # time to steady state, UVS and MLVS from rest, and the MLVS error against UVS
    steady = None
    if not args.no_steady and rank == 0:
        su, fu = _steady(desc, stream.cuda_stream, False)
        sv, fv = _steady(desc, stream.cuda_stream, True)
        err = {"rho": _l2(fv[0], fu[0]),
               "u": float(np.sqrt(np.sum((fv[1] - fu[1]) ** 2 + (fv[2] - fu[2]) ** 2)) /
                          np.sqrt(np.sum(fu[1] ** 2 + fu[2] ** 2))),
               "T": _l2(fv[3], fu[3]),
               "q": float(np.sqrt(np.sum((fv[4] - fu[4]) ** 2 + (fv[5] - fu[5]) ** 2)) /
                          np.sqrt(np.sum(fu[4] ** 2 + fu[5] ** 2)))}
        steady = {"uvs": su, "mlvs": sv, "speedup": su["seconds"] / sv["seconds"],
                  "mlvs_vs_uvs_rel_l2": err,
                  "same_error": bool(err["rho"] < 1e-2 and err["u"] < 1e-2 and err["T"] < 1e-2 and err["q"] < 2e-2),
                  "criterion": f"max over rho,u,v,T of |W^n - W^(n-100)|/|W^n| < {STEADY_TOL:g}, "
                               f"at most {STEADY_MAX} steps"}

    # level selector (10-64-64-4, BF16 weights): trained on criterion labels, then used for
    # a fixed-level-set adaptation against the criterion on a held-out 64^2 state
    selector = None
    if not args.no_selector and rank == 0:
        selector = _selector_leg()
    cylinder = None
    if not args.no_cylinder and rank == 0:
        cylinder = {st_: _cylinder_leg(storage=st_, positive_mapping=int(args.positive_mapping))
                    for st_ in ("f32", "bf16")}
    unstructured = _unstructured_isolated() if (not args.no_unstructured and rank == 0) else None
    sod = _sod_leg() if (not args.no_sod and rank == 0) else None
    batch = _batch_leg() if (not args.no_batch and rank == 0) else None

    # end-to-end through the public API: host init upload, steps, host moment reads
    e2e = None
    if not args.no_e2e:
        torch.cuda.synchronize()
        ke = max(1, min(args.steps, 50))
        t0 = time.perf_counter()
        s2 = Solver(desc, stream=stream.cuda_stream)
        for _ in range(ke):
            s2.step(1)
            _ = M.mlvs_moments(s2.h, 0, M.RHO | M.U | M.V | M.T, ncell)
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        s2.close()
        e2e = {"value": upd_step * ke / te, "unit": UNIT,
               "h2d_bytes_per_step": int(desc["init"].nbytes / ke),
               "d2h_bytes_per_step": int(4 * ncell * 8),
               "steps": ke, "includes": "create + init upload + steps + per-step host moment read"}

    cpu = None
    if rank == 0 and not args.no_cpu:
        rate, t, upd = oracle_rate(16, 4)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"16x16-cell cavity on the same 101^2 velocity grid, 4 FP64 oracle steps "
                         f"({upd} updates, {t:.1f} s, numpy single thread)"}
        try:
            rate_a, t_a, upd_a, procs = oracle_rate_all_cores(12, 2)
            cpu["all_cores"] = {"value": rate_a, "unit": UNIT, "cores": procs, "kind": "oracle",
                                "sample": f"{procs} independent 12x12-cell cavities on the same 101^2 "
                                          f"velocity grid, 2 FP64 oracle steps each, one process per core "
                                          f"({upd_a} updates, {t_a:.1f} s)"}
        except Exception as e:                      # the single-thread figure stands alone
            cpu["all_cores"] = {"error": str(e)[:200]}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.storage, "data": "synthetic",
            "config": {"workload": wl, "cells": ncell,
                       "velocities": nv, "levels": "UVS 101^2 (value); MLVS quadtree 101^2/51^2/25^2",
                       "Kn": 0.075,
                       "l2": f"inputs larger than L2 (2 x {2 * ncell * nv * {'f32': 4, 'bf16': 2, 'f64': 8}[args.storage] / 1e6:.0f} MB distributions)",
                       "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "hbm", "kernel": names[dom], "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": (achieved / peak) if achieved else None,
                         "peak_kind": f"{peak_kind} hbm_gbs", "traffic": traffic,
                         "algorithmic_bytes_per_update": algo_per_update},
            "phases_ms_per_step": {n: p / args.steps for n, p in zip(names, phases)},
            "phases_from": "a second run of the same number of steps with CUDA events around every launch",
            "step_roofline": {"achieved": 4 * fbytes * upd_step / (ms_step / 1e3) / 1e9, "peak": peak,
                              "unit": "GB/s", "frac": 4 * fbytes * upd_step / (ms_step / 1e3) / 1e9 / peak,
                              "algorithmic_bytes_per_update": 4 * fbytes,
                              "note": "the whole step (every launch) against reading and writing f once"},
            "mlvs": mlvs, "time_to_steady": steady, "selector": selector, "cylinder": cylinder,
            "unstructured": unstructured, "sod": sod, "batch": batch,
            "clocks": clocks, "e2e": e2e, "gpu_launches": st.launches, "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--storage", default="f32", choices=["f32", "bf16", "f64"])
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mlvs", action="store_true")
    ap.add_argument("--no-steady", action="store_true")
    ap.add_argument("--no-selector", action="store_true")
    ap.add_argument("--cells", type=int, default=64, help="cavity cells per side (default 64)")
    ap.add_argument("--no-cylinder", action="store_true",
                    help="skip the Ma 5 cylinder legs (FP32 and BF16: UVS vs MLVS, clustering-threshold "
                         "sweep and runtime-model fit, about 45 s each)")
    ap.add_argument("--positive-mapping", action="store_true",
                    help="cylinder leg: exponential fallback for level switches that go negative")
    ap.add_argument("--no-sod", action="store_true", help="skip the shock-tube latency leg")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the 64-cavity batch leg (adaptive instances stepped as one group)")
    ap.add_argument("--no-unstructured", action="store_true",
                    help="skip the two-cavity unstructured-mesh leg (13,600 quads, 101^2 velocities, "
                         "run in a child process)")
    ap.add_argument("--only-unstructured", type=int, default=0, metavar="M",
                    help="run only the two-cavity unstructured leg, in this process, on the mesh "
                         "two_cavities(M) (M = 10: 13,600 quads), for --steps steps after --warmup "
                         "steps, and print its JSON (for profiling a smaller case)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.only_unstructured:
        print(json.dumps(_unstructured_leg(m=args.only_unstructured, steps=args.steps, warm=args.warmup)))
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(local_rank)
        tdist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as tdist
        tdist.destroy_process_group()


if __name__ == "__main__":
    main()
