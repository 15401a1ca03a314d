#!/usr/bin/env python
"""Benchmark of the TR-based sound-speed gradient (forward + TR + adjoint simulations).

One step = one fwi_gradient call on the 128 x 128 x 64 breast-phantom workload
(256 emitters, 1024 receivers, 4 Rademacher-encoded super-shots, 1500 time
samples, 10-cell PML, literal Alg. 1 pairing): 4 x (1500 + 1499 + 1498)
simulation steps of 2^20 voxels.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on bounded samples of the same
workload (the reference arm: the paper ships no code).
"""
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

METRIC = "Gvoxel-steps/s and gradients/h vs plain form at rel l2<=1e-4; p50/p99 latency"
UNIT = "Gvoxel-steps/s"
WORKLOAD = ("plain method at scale: 128x128x64 breast phantom, 256 emitters + 1024 receivers, "
            "4 Rademacher super-shots, 1500 steps, TR gradient (literal Alg. 1 pairing)")

# Algorithmic DRAM bytes per voxel for one simulation in one launch (FP32 fields,
# half spectra of hx*ny*nz complex FP32 = 8*hx/nx bytes per voxel each).
def alg_bytes_per_voxel(kernel, nx):
    hf = 8.0 * (nx // 2 + 1) / nx
    return {"zpass_momentum": 3 * hf,             # read P_xy, write Q and R
            "plane_momentum": 5 * hf + 24.0,      # read Q, R; write 3 V_xy; v_xi read + write
            "zpass_mass": 6 * hf,                 # 3 spectra read + written
            "plane_mass": 4 * hf + 28.0}[kernel]  # 3 spectra read, P_xy written; rho r/w; c0^2


# DRAM bytes per simulation in one launch, read + write, from ncu on the 128x128x64 gradient:
# every launch of one gradient (40 time steps, one stream group: 4 simulations per launch in
# the forward phase, 8 in the backward phase), L2 not flushed between launches, so write-backs
# are counted where the hardware performs them (often in the next kernel's launch).  The
# command and the per-kernel table are in profiles/step_kernels_128x128x64_gradient.md.  Valid
# only for these kernels at this size and schedule; anything else reports null.  Each kernel's
# launches depend only on the knobs listed for it (the plane kernels do not see z_tile, the z
# passes do not see split_plane).
TRAFFIC_PER_SIM = {"grid": (128, 128, 64),
                   "knobs": {"zpass_momentum": {"specialized": 2, "z_tile": 32, "stream_groups": 1},
                             "zpass_mass": {"specialized": 2, "z_tile": 32, "stream_groups": 1},
                             "plane_momentum": {"specialized": 2, "split_plane": 0, "stream_groups": 1},
                             "plane_mass": {"specialized": 2, "split_plane": 0, "stream_groups": 1}},
                   "bytes": {"zpass_momentum": 7.88e6, "plane_momentum": 39.80e6,
                             "zpass_mass": 18.78e6, "plane_mass": 40.03e6}}


def traffic_per_launch(kernel, grid, schedule, sims_per_launch):
    t = TRAFFIC_PER_SIM
    if tuple(grid) != t["grid"] or any(schedule.get(k) != v for k, v in t["knobs"][kernel].items()):
        return None
    return t["bytes"][kernel] * sims_per_launch


# Multi-GPU use is replicas only: each rank computes its own encoded gradient estimate
# (Sec. 4.5) with no data-path collective; the job is timed as the slowest rank.
def replica_weights(weights, rank):
    """Encoding weights [K][n_src] of one replica: rank 0 keeps the workload's own, every other
    rank draws its own Rademacher super-shots (an independent gradient estimate)."""
    if rank == 0:
        return weights
    from paper_2102_00755_b300 import synth
    rng = np.random.default_rng(1000 + rank)
    return np.stack([synth.rademacher(weights.shape[1], rng) for _ in range(weights.shape[0])])


def job_time_ms(local_ms, world, device=None):
    """Max over ranks of one rank's timed region (ms); needs an initialised process group
    when world > 1."""
    if world == 1:
        return float(local_ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank_step, world, steps, job_ms):
    """Units per second of the whole job: every rank's units over the slowest rank's time."""
    return units_per_rank_step * world * steps / (job_ms / 1e3)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None

    def __enter__(self):
        self.fh = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        self.fh.flush()
        self.fh.seek(0)
        rows = [r.split(",") for r in self.fh.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.fh.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["clock sampling unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


def cpu_baseline(wl, budget_s=15.0, min_steps=6):
    """Time the FP64 oracle's time step on the same grid (bounded sample)."""
    workers = os.cpu_count() or 1
    os.environ["ORACLE_WORKERS"] = str(workers)
    from oracle import pstd
    G = pstd.grid_for(wl)
    S = pstd.State(G.shape)
    c2 = wl.c_model ** 2
    src = pstd.injection_map(G, wl.c_model, wl.src_idx, wl.weights[0])
    pstd.step(G, S, c2, mass_src=src * wl.wavelet[0])      # warm-up (FFT plans)
    t0 = time.perf_counter()
    n = 0
    while n < min_steps or time.perf_counter() - t0 < budget_s:
        pstd.step(G, S, c2, mass_src=src * wl.wavelet[min(n + 1, wl.nt - 1)])
        n += 1
        if n >= 400:
            break
    dt = time.perf_counter() - t0
    return {"value": wl.n_vox * n / dt / 1e9, "unit": UNIT, "cores": workers, "kind": "oracle",
            "sample": f"{n} FP64 oracle time steps of one simulation on the {wl.nx}x{wl.ny}x{wl.nz} "
                      f"grid ({dt:.1f} s); a gradient is 3 simulations of such steps"}


def run_oracle_full(args):
    """Whole FP64 oracle gradients of the 32^3 (300 steps, one source) and 96x96x48 (1000
    steps, exact pairing) configurations on the host cores, wall clock, median of
    --oracle-runs, beside the same gradients on the GPU (CUDA events, median of 10)."""
    import torch

    from oracle import pstd
    from paper_2102_00755_b300 import fwi, synth

    workers = os.cpu_count() or 1
    os.environ["ORACLE_WORKERS"] = str(workers)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    rows = []
    for name, wl, pairing in [("32^3, 300 steps, 1 source, 64 receivers (literal)", synth.config1(), "literal"),
                              ("96x96x48, 1000 steps, 32 + 128 transducers (exact)", synth.config4(), "exact")]:
        G = pstd.grid_for(wl)
        w = wl.weights[0]
        f_obs = pstd.forward(G, wl.c_true, wl.src_idx, w, wl.wavelet, wl.rec_idx)[0]
        ts = []
        for _ in range(args.oracle_runs):
            t0 = time.perf_counter()
            pstd.fwi_gradient(G, wl.c_model, wl.src_idx, w, wl.wavelet, wl.rec_idx, wl.layer_idx,
                              wl.gamma_idx, f_obs, pairing=pairing, c_rec=wl.c_rec)
            ts.append(time.perf_counter() - t0)
        plan = fwi.Plan.from_workload(wl, pairing=pairing, max_shots=1, device=dev)
        c = torch.tensor(wl.c_model, dtype=torch.float32, device=dev).reshape(-1)
        wt = torch.tensor(wl.weights, dtype=torch.float32, device=dev)
        ot = torch.tensor(synth.f32(f_obs)[None], dtype=torch.float32, device=dev)
        plan.gradient(c, wt, ot)
        torch.cuda.synchronize(dev)
        gt = []
        for _ in range(10):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            plan.gradient(c, wt, ot)
            b.record(stream)
            torch.cuda.synchronize(dev)
            gt.append(a.elapsed_time(b))
        assert plan.status() == fwi.FWI_OK
        vs = plan.voxel_steps(1, True)
        o_s, g_ms = statistics.median(ts), statistics.median(gt)
        rows.append({"config": name, "voxel_steps": vs, "oracle_wall_s": ts, "oracle_median_s": o_s,
                     "oracle_gvoxel_steps_per_s": vs / o_s / 1e9, "gpu_median_ms": g_ms,
                     "gpu_gvoxel_steps_per_s": vs / (g_ms / 1e3) / 1e9, "gpu_over_oracle": o_s / (g_ms / 1e3)})
        plan.close()
    print(json.dumps({"workload": "oracle timing: whole gradients, FP64 oracle vs the GPU path",
                      "cores": workers, "runs": args.oracle_runs, "rows": rows}), flush=True)


def run_reference(args):
    """Reference arm: the FP64 CPU oracle on bounded samples of the same workload."""
    from paper_2102_00755_b300 import synth
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = synth.config2()
    os.environ["ORACLE_WORKERS"] = str(os.cpu_count() or 1)
    from oracle import pstd
    G = pstd.grid_for(wl)
    S = pstd.State(G.shape)
    c2 = wl.c_model ** 2
    src = pstd.injection_map(G, wl.c_model, wl.src_idx, wl.weights[0])
    per_step = 4                      # oracle time steps per benchmark step (bounded sample)
    times = []
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        for n in range(per_step):
            pstd.step(G, S, c2, mass_src=src * wl.wavelet[(it * per_step + n) % wl.nt])
        if it >= args.warmup:
            times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = wl.n_vox * per_step * args.steps / tot / 1e9
    sample = (f"{per_step} FP64 oracle time steps of one simulation per step on the "
              f"{wl.nx}x{wl.ny}x{wl.nz} grid")
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "impl": "reference",
           "config": {"workload": WORKLOAD, "grid": [wl.nx, wl.ny, wl.nz], "nt": wl.nt},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def grouped_batch(dev, nt=0):
    """The uneven-grid configuration grouped by grid: per grid, one per-shot-model plan whose
    super-shots are that grid's instances (each with its own model, data and gradient), the
    schedule of each plan chosen by the autotuner.  Returns the 16 workloads, the groups, the
    tuned schedules, the plans with their inputs (c, weights, encoded observed data), and the
    voxel-steps and algorithmic bytes of one gradient of every instance."""
    import torch

    from paper_2102_00755_b300 import autotune, fwi, synth

    wls = [synth.config3_instance(i) for i in range(16)]
    if nt:
        for wl in wls:
            wl.nt = nt
            wl.wavelet = wl.wavelet[:nt]
    groups = {}
    for wl in wls:
        groups.setdefault((wl.nx, wl.ny, wl.nz), []).append(wl)
    tuned = {}
    for key, g in groups.items():       # one schedule per grid size, chosen by the autotuner
        tuned[key] = autotune.tune(g[0], K=len(g), steps=24, reps=3, save=False)["schedule"]
    f32 = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    # grouped form: per grid, the instances are the super-shots of one per-shot-model plan
    gplans, gcs, gws, gobs = [], [], [], []
    for key, g in groups.items():
        plan = fwi.Plan.from_workload(g[0], max_shots=len(g), per_shot_models=True, device=dev)
        autotune.set_schedule(plan, tuned[key])
        w = f32(np.stack([wl.weights[0] for wl in g]))
        c_true = f32(np.stack([wl.c_true for wl in g])).reshape(-1)
        gobs.append(plan.forward(c_true, w))          # each instance's data from its own true model
        gcs.append(f32(np.stack([wl.c_model for wl in g])).reshape(-1))
        gws.append(w)
        gplans.append(plan)
    vsteps = sum(p.voxel_steps(len(g), True) for p, g in zip(gplans, groups.values()))
    bpv_step = sum(p.voxel_steps(len(g), True) * sum(alg_bytes_per_voxel(k, key[0]) for k in fwi.KERNELS)
                   for p, g, key in zip(gplans, groups.values(), groups.keys()))
    return wls, groups, tuned, (gplans, gcs, gws, gobs), vsteps, bpv_step


def run_batch(args):
    """16 encoded-gradient instances of uneven grids (4 each of 64^3, 96x96x48, 128x128x64,
    160x160x80; 1200..2000 steps).  The batched form groups the instances by grid: one plan
    per grid whose super-shots are the instances (each with its own model, data and
    gradient, sharing every launch), the four plans captured as one CUDA graph.  Compared
    with: one single-instance plan per instance in one graph, the instances one after
    another, and the plain form (one simulation per launch sequence)."""
    import torch

    from paper_2102_00755_b300 import autotune, fwi

    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    wls, groups, tuned, (gplans, gcs, gws, gobs), vsteps, bpv_step = grouped_batch(dev, args.nt)
    f32 = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    batch = fwi.Batch(gplans)
    t0 = time.perf_counter()
    batch.gradient(gcs, gws, gobs)
    torch.cuda.synchronize(dev)
    capture_s = time.perf_counter() - t0

    def timed(fn, reps):
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize(dev)
            ts.append(a.elapsed_time(b))
        return sum(ts) / len(ts)

    # Graph concurrency, chosen by measurement like an FFT schedule: which plans run one after
    # another on which of the chains that run side by side.  The plans in batch order are
    # 64^3, 96x96x48, 128x128x64, 160x160x80.  Side by side, plans that each fill the GPU mostly
    # share L2; the largest grid's one-CTA-per-SM plane launches leave SMs idle in their last
    # wave, which a smaller plan beside it can fill.
    largest = max(range(len(gplans)), key=lambda i: gplans[i].n_vox)
    arrangements = {"one chain": [0] * len(gplans),
                    "largest beside the rest": [1 if i == largest else 0 for i in range(len(gplans))],
                    "two mixed chains": [i % 2 for i in range(len(gplans))],
                    "one chain per grid": list(range(len(gplans)))}
    by_arrangement = {}
    for name, chain in arrangements.items():
        batch.set_chains(chain)
        batch.gradient(gcs, gws, gobs)
        by_arrangement[name] = timed(lambda: batch.gradient(gcs, gws, gobs), 1)
    best = min(by_arrangement, key=by_arrangement.get)
    batch.set_chains(arrangements[best])
    for _ in range(args.warmup - 1):
        batch.gradient(gcs, gws, gobs)
    with ClockSampler(0) as clk:
        ms_graph = timed(lambda: batch.gradient(gcs, gws, gobs), args.steps)
    nodes_grouped = batch.nodes()
    assert all(p.status() == fwi.FWI_OK for p in gplans)

    def grouped_sequential():
        for p, c, w, o in zip(gplans, gcs, gws, gobs):
            p.gradient(c, w, o)
    grouped_sequential()
    ms_gseq = timed(grouped_sequential, 1)
    per_grid = {}
    for (key, g), p, c, w, o in zip(groups.items(), gplans, gcs, gws, gobs):
        ms = timed(lambda: p.gradient(c, w, o), 1)
        per_grid["x".join(map(str, key))] = {"instances": len(g), "ms": ms,
                                             "gvoxel_steps_per_s": p.voxel_steps(len(g), True) / (ms / 1e3) / 1e9}
    del batch
    for p in gplans:
        p.close()
    # one single-instance plan per instance: in one graph, one after another, plain
    plans, cs, ws, obs = [], [], [], []
    for wl in wls:
        plan = fwi.Plan.from_workload(wl, max_shots=1, device=dev)
        autotune.set_schedule(plan, dict(tuned[(wl.nx, wl.ny, wl.nz)], stream_groups=1))
        w = f32(wl.weights)
        obs.append(plan.forward(f32(wl.c_true).reshape(-1), w))
        plans.append(plan)
        cs.append(f32(wl.c_model).reshape(-1))
        ws.append(w)
    batch1 = fwi.Batch(plans)
    batch1.gradient(cs, ws, obs)
    ms_graph1 = timed(lambda: batch1.gradient(cs, ws, obs), 1)
    nodes_single = batch1.nodes()

    def sequential():
        for p, c, w, o in zip(plans, cs, ws, obs):
            p.gradient(c, w, o)
    sequential()
    ms_seq = timed(sequential, 1)
    del batch1
    for p in plans:
        p.close()
    plains = [fwi.Plan.from_workload(wl, max_shots=1, sims_per_launch=1, device=dev) for wl in wls]
    for p, wl in zip(plains, wls):
        autotune.set_schedule(p, dict(tuned[(wl.nx, wl.ny, wl.nz)], stream_groups=1))

    def plain():
        for p, c, w, o in zip(plains, cs, ws, obs):
            p.gradient(c, w, o)
    plain()
    ms_plain = timed(plain, 1)
    G = lambda ms: vsteps / (ms / 1e3) / 1e9
    hbm, kind = peaks()
    step_gbs = bpv_step / (ms_graph / 1e3) / 1e9
    out = {"metric": METRIC, "value": G(ms_graph), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_graph, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "batching: 16 encoded gradients of uneven grids (4 each of 64^3, "
                                  "96x96x48, 128x128x64, 160x160x80), 1200-2000 steps, grouped by grid into "
                                  "four per-shot-model plans captured as one graph (chains chosen by measurement)",
                      "voxel_steps_per_step": vsteps, "graph_nodes": nodes_grouped,
                      "schedules": {"x".join(map(str, k)): v for k, v in tuned.items()},
                      "capture_and_first_run_s": capture_s},
           "gradients_per_h": 3600.0 * 16 / (ms_graph / 1e3),
           "roofline": {"bound": "hbm", "kernel": "whole step (all four step kernels)",
                        "achieved": step_gbs, "peak": hbm, "peak_kind": kind, "unit": "GB/s",
                        "frac": step_gbs / hbm, "traffic": None,
                        "alg_bytes_per_voxel_step": bpv_step / vsteps,
                        "note": "algorithmic bytes of every step kernel of every instance over the graph time"},
           "graph_chains": {"chosen": best, "chain_of_plan": arrangements[best], "ms_by_arrangement": by_arrangement,
                            "plan_order": ["x".join(map(str, k)) for k in groups],
                            "form": "which of the four grouped plans run one after another on which chain"},
           "grouped_sequential": {"value": G(ms_gseq), "ms_per_step": ms_gseq, "per_grid": per_grid,
                                  "form": "the four grouped plans one after another, no graph"},
           "single_instance_graph": {"value": G(ms_graph1), "ms_per_step": ms_graph1, "graph_nodes": nodes_single,
                                     "form": "16 single-instance plans captured as one graph"},
           "sequential": {"value": G(ms_seq), "ms_per_step": ms_seq,
                          "gradients_per_h": 3600.0 * 16 / (ms_seq / 1e3),
                          "form": "16 single-instance plans one after another"},
           "plain": {"value": G(ms_plain), "ms_per_step": ms_plain,
                     "gradients_per_h": 3600.0 * 16 / (ms_plain / 1e3),
                     "form": "one simulation per launch sequence, instances one after another"},
           "clocks": clk.summary()}
    print(json.dumps(out), flush=True)


def run_serve(args):
    """Serving: a seeded Poisson stream of forward and gradient requests over the three
    multigrid levels (135x135x96 / 243x243x135 / 480x480x256 with PML; 1000 / 2000 / 4000
    steps; 1024 receivers; 2..8 encoded emitters out of 8), level mix 128:128:32, half
    gradients, served by the continuous-batching server (admission by free HBM)."""
    import torch

    from paper_2102_00755_b300 import fwi, serve, synth

    dev = torch.device("cuda", 0)
    names, levels, t_data = [], [], {}
    for L in range(3):
        wl = synth.serving_level(L, n_src=8, seed=1000 + L)
        if args.nt:
            nt = max(8, int(args.nt * wl.nt / synth.SERVING_LEVELS[2][2]))
            wl.nt, wl.wavelet = nt, wl.wavelet[:nt]
        t0 = time.perf_counter()
        levels.append(serve.make_level(f"L{L}", wl, device=dev))
        t_data[f"L{L}"] = time.perf_counter() - t0
        names.append(f"L{L}")
    server = serve.Server(levels, device=dev, max_inflight=args.inflight)
    # warm the two smaller levels (module loading, first uncaptured call, graph capture)
    warm = [serve.Request(-1 - i, nm, kind, np.eye(8)[0], 0.0)
            for i, (nm, kind) in enumerate([(n, k) for n in names[:2] for k in ("forward", "gradient")] * 2)]
    server.run(warm, realtime=False)
    hbm, kind = peaks()

    def serve_stream(n, rate, seed):
        reqs = serve.poisson_stream(names, [128, 128, 32], n, rate, 8, seed=seed, stratified=True)
        with ClockSampler(0) as clk:
            out = server.run(reqs, realtime=True)
        st, res = out["stats"], out["results"]
        assert all(p.status() == fwi.FWI_OK for slots in server.pool.values() for p in [s.plan for s in slots])
        per = {}
        for nm in names:
            for kind_ in ("forward", "gradient"):
                lat = [r.latency for r in res if r.level == nm and r.kind == kind_]
                svc = [r.done - r.admitted for r in res if r.level == nm and r.kind == kind_]
                if lat:
                    per[f"{nm}-{kind_}"] = {"n": len(lat), "p50_s": float(np.percentile(lat, 50)),
                                            "p99_s": float(np.percentile(lat, 99)),
                                            "median_in_service_s": float(np.median(svc))}
        gvs = st["gvoxel_steps_per_s"]
        # HBM fraction of the achieved rate under two byte models per voxel-step: the whole-plane
        # two-pass kernels' 125 B and the 52 B state floor (v, rho read + written, c0 read)
        st["hbm_frac"] = {"at_125B_per_voxel_step": gvs * 125.125 / hbm, "at_52B_state_floor": gvs * 52.0 / hbm,
                          "peak_gbs": hbm, "peak_kind": kind}
        return st, per, clk.summary()

    stats, per, clocks = serve_stream(args.requests, args.rate, 1000)
    sweep = []
    for rate in [float(r) for r in args.rates.split(",") if r.strip()]:
        st, pr, ck = serve_stream(args.sweep_requests, rate, 2000)
        sweep.append({"rate_req_per_s": rate, "requests": st["requests"], "p50_s": st["p50_s"], "p99_s": st["p99_s"],
                      "offered_req_per_s": st["offered_req_per_s"], "achieved_req_per_s": st["achieved_req_per_s"],
                      "gvoxel_steps_per_s": st["gvoxel_steps_per_s"], "gradients_per_h": st["gradients_per_h"],
                      "hbm_frac": st["hbm_frac"], "per_level": pr, "clocks": ck})
    # highest swept rate the server kept up with (achieved >= 90 % of offered: no growing queue)
    kept = [p for p in sweep if p["achieved_req_per_s"] and p["offered_req_per_s"]
            and p["achieved_req_per_s"] >= 0.9 * p["offered_req_per_s"]]
    sustainable = max(kept, key=lambda p: p["rate_req_per_s"]) if kept else None
    grid = {nm: [lv.wl.nx, lv.wl.ny, lv.wl.nz, lv.wl.nt] for nm, lv in zip(names, levels)}
    line = {"metric": METRIC, "value": stats["gvoxel_steps_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": stats["requests"], "warmup": len(warm),
            "ms_per_step": 1e3 * stats["wall_s"] / max(stats["requests"], 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "impl": "ours",
            "config": {"workload": "serving: Poisson stream of forward/gradient requests over multigrid "
                                   "levels 135x135x96, 243x243x135, 480x480x256 (PML incl.)",
                       "levels": grid, "requests": args.requests, "rate_req_per_s": args.rate,
                       "level_mix": [128, 128, 32], "level_mix_drawn": "stratified (exact counts, seeded order)",
                       "p_gradient": 0.5, "emitters_per_request": "2..8",
                       "max_inflight": args.inflight, "raw_data_generation_s": t_data},
            "latency_s": {"p50": stats["p50_s"], "p99": stats["p99_s"]},
            "gradients_per_h": stats["gradients_per_h"], "serve_stats": stats, "per_level": per,
            "rate_sweep": sweep,
            "sustainable": ({"rate_req_per_s": sustainable["rate_req_per_s"], "p50_s": sustainable["p50_s"],
                             "p99_s": sustainable["p99_s"], "gvoxel_steps_per_s": sustainable["gvoxel_steps_per_s"],
                             "rule": "highest swept rate with achieved >= 0.9 x offered requests/s"}
                            if sustainable else None),
            "clocks": clocks}
    print(json.dumps(line), flush=True)
    server.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--plain-steps", type=int, default=1)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--tr-box-steps", type=int, default=2,
                    help="gradients timed with the TR re-simulation on a box enclosing Gamma (0: skip)")
    ap.add_argument("--batch-steps", type=int, default=1,
                    help="batched uneven-grid gradients timed beside the headline (single GPU; 0: skip)")
    ap.add_argument("--serve-requests", type=int, default=24,
                    help="requests of the short serving stream timed beside the headline (single GPU; 0: skip)")
    ap.add_argument("--serve-rate", type=float, default=2.0, help="its mean arrival rate (requests/s)")
    ap.add_argument("--nt", type=int, default=0,
                    help="override the number of time samples (small profiling cases only)")
    ap.add_argument("--schedule", default="",
                    help="fixed FFT schedule 'specialized,radix_order,z_tile,split_plane' instead of "
                         "autotuning (reproducible launch sequences for profiling)")
    ap.add_argument("--requests", type=int, default=256, help="serve: length of the request stream")
    ap.add_argument("--rates", default="", help="serve: comma-separated arrival rates of a rate sweep")
    ap.add_argument("--sweep-requests", type=int, default=32, help="serve: requests per sweep point")
    ap.add_argument("--rate", type=float, default=4.0, help="serve: mean arrival rate (requests/s)")
    ap.add_argument("--inflight", type=int, default=8, help="serve: admitted requests at most")
    ap.add_argument("--level", type=int, default=2, help="level: serving grid (0, 1, 2)")
    ap.add_argument("--pz", type=int, default=0, help="level: physical z extent override (profiling)")
    ap.add_argument("--oracle-runs", type=int, default=3, help="oracle: whole oracle gradients per config")
    ap.add_argument("--instance", type=int, default=12, help="instance: which of the 16 uneven-grid instances")
    ap.add_argument("--workload", default="plain", choices=["plain", "batch", "serve", "level", "oracle", "instance"],
                    help="plain: the 128x128x64 gradient (the reported line); batch: the 16-instance "
                         "uneven-grid configuration as one captured graph vs sequential forms; "
                         "serve: the Poisson request stream over the three multigrid levels; "
                         "level: one gradient (one super-shot) on a serving grid; instance: one gradient of "
                         "one uneven-grid batch instance; oracle: whole FP64 "
                         "oracle gradients of the 32^3 and 96x96x48 configurations beside the GPU's")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "batch":
        run_batch(args)
        return
    if args.workload == "serve":
        run_serve(args)
        return
    if args.workload == "oracle":
        run_oracle_full(args)
        return

    import torch
    import torch.distributed as dist

    from paper_2102_00755_b300 import fwi, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    if args.workload == "level":
        wl = synth.serving_level(args.level, n_src=8, seed=1000 + args.level, pz=args.pz or None)
    elif args.workload == "instance":
        wl = synth.config3_instance(args.instance)
    else:
        wl = synth.config2()
    if args.nt:
        wl.nt = args.nt
        wl.wavelet = wl.wavelet[:args.nt]
    workload = WORKLOAD if args.workload == "plain" else (
        f"uneven-grid batch instance {args.instance}: one TR gradient (one super-shot of 128 emitters, 512 "
        f"receivers) on the {wl.nx}x{wl.ny}x{wl.nz} grid, {wl.nt} steps" if args.workload == "instance" else
        f"serving level {args.level}: one TR gradient (one super-shot of 8 emitters, 1024 receivers) "
        f"on the {wl.nx}x{wl.ny}x{wl.nz} grid, {wl.nt} steps")
    K = wl.weights.shape[0]
    wl.weights = replica_weights(wl.weights, rank)   # independent estimates per GPU (Sec. 4.5)
    from paper_2102_00755_b300 import autotune
    if args.schedule:
        schedule = dict(zip(autotune.KNOBS, (int(v) for v in args.schedule.split(","))))
    else:
        schedule = autotune.tune(wl, K=K, steps=24, reps=3, device=dev, save=False)["schedule"]
    plan = fwi.Plan.from_workload(wl, pairing="literal", max_shots=K, device=dev)
    if autotune.set_schedule(plan, schedule) != fwi.FWI_OK:
        raise RuntimeError(f"schedule {schedule} is not available for this grid")
    c_true = torch.tensor(wl.c_true, dtype=torch.float32, device=dev).reshape(-1)
    c_model = torch.tensor(wl.c_model, dtype=torch.float32, device=dev).reshape(-1)
    w = torch.tensor(wl.weights, dtype=torch.float32, device=dev)
    # encoded observed data by linearity: forward of the encoded true model
    observed = plan.forward(c_true, w)
    misfit = torch.empty(K, dtype=torch.float64, device=dev)
    grad = torch.empty(wl.n_vox, dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2
    vsteps = plan.voxel_steps(K, True)
    launches = plan.launches(K, True)

    def step():
        plan.gradient(c_model, w, observed, misfit=misfit, grad=grad)

    # warm-up; the last warm-up step times every kernel (CUDA events) for the time shares
    # (the first calls also load modules and would distort them)
    share_ms = {}
    for i in range(args.warmup):
        last = i == args.warmup - 1
        if last:
            plan.profile(enable=True)
        step()
        if last:
            plan.profile(enable=False)
            share_ms = {k: v[0] for k, v in plan.profile_read().items()}
        flush.zero_()
    torch.cuda.synchronize(dev)
    if plan.status() != fwi.FWI_OK:
        raise RuntimeError("gradient failed: " + fwi.fwi_status_string(plan.status()))
    dominant = max(share_ms, key=share_ms.get)

    # timed region (device events around each step; L2 flushed between steps)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    plan.profile(dominant, enable=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
            flush.zero_()
        torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    plan.profile(dominant, enable=False)
    kern_ms, kern_launches, kern_sims = plan.profile_read()[dominant]
    step_ms = [a.elapsed_time(b) for a, b in ev]
    tot_ms = job_time_ms(sum(step_ms), world, dev)
    value = whole_job_rate(vsteps, world, args.steps, tot_ms) / 1e9
    grads_per_h = 3600.0 * whole_job_rate(1, world, args.steps, tot_ms)
    clocks = clk.summary()
    assert plan.status() == fwi.FWI_OK

    # roofline of the dominant kernel over the timed region
    hbm, kind = peaks()
    bpv = alg_bytes_per_voxel(dominant, wl.nx)
    alg_bytes = bpv * wl.n_vox * kern_sims
    achieved = alg_bytes / (kern_ms / 1e3) / 1e9 if kern_ms > 0 else None
    # the whole step: algorithmic bytes of all four kernels per voxel-step over the step time
    # (with two stream groups, launches of different kernels overlap, so a kernel's own event
    # time includes time shared with the other group's kernels)
    step_bpv = sum(alg_bytes_per_voxel(k, wl.nx) for k in fwi.KERNELS)
    step_gbs = step_bpv * vsteps * args.steps / (tot_ms / 1e3) / 1e9
    # the same kernel in one untimed gradient with one stream group (all simulations of a
    # phase in each launch, nothing overlapping it): the kernel's own efficiency
    iso = None
    if schedule.get("stream_groups", 1) > 1:
        autotune.set_schedule(plan, dict(schedule, stream_groups=1))
        plan.profile(dominant, enable=True)
        step()
        torch.cuda.synchronize(dev)
        plan.profile(dominant, enable=False)
        i_ms, i_launches, i_sims = plan.profile_read()[dominant]
        autotune.set_schedule(plan, schedule)
        i_ach = bpv * wl.n_vox * i_sims / (i_ms / 1e3) / 1e9
        iso = {"achieved": i_ach, "frac": i_ach / hbm, "avg_launch_ms": i_ms / max(i_launches, 1),
               "sims_per_launch": i_sims / max(i_launches, 1), "stream_groups": 1}
    if iso is None:                # one stream group already: the timed launches are the kernel's own
        iso = {"achieved": achieved, "frac": achieved / hbm if achieved else None,
               "avg_launch_ms": kern_ms / max(kern_launches, 1),
               "sims_per_launch": kern_sims / max(kern_launches, 1), "stream_groups": 1}
    iso_sched = dict(schedule, stream_groups=1)
    roofline = {"bound": "hbm", "kernel": dominant, "achieved": iso["achieved"], "peak": hbm,
                "peak_kind": kind, "unit": "GB/s", "frac": iso["frac"],
                "traffic": traffic_per_launch(dominant, (wl.nx, wl.ny, wl.nz), iso_sched, iso["sims_per_launch"]),
                "traffic_note": ("ncu DRAM read + write bytes per simulation of this kernel over consecutive "
                                 "launches of one gradient with one stream group, L2 not flushed between "
                                 "launches (write-backs land where the hardware does them), times the "
                                 "simulations per launch; null unless the kernels, grid and schedule are "
                                 "those of the capture"),
                "alg_bytes_per_launch": bpv * wl.n_vox * iso["sims_per_launch"],
                "alg_bytes_per_voxel": bpv,
                "avg_launch_ms": iso["avg_launch_ms"], "sims_per_launch": iso["sims_per_launch"],
                "measured_as": ("CUDA events on the kernel's stream around each of its launches in one "
                                "gradient with one stream group (every simulation of a phase in each "
                                "launch, no other kernel running beside it)"),
                "overlapped": {"achieved": achieved, "frac": achieved / hbm if achieved else None,
                               "avg_launch_ms": kern_ms / max(kern_launches, 1), "launches_timed": kern_launches,
                               "note": ("the same kernel's CUDA-event time over the timed region, where its "
                                        "launches overlap the other stream groups' kernels")},
                "step": {"alg_bytes_per_voxel_step": step_bpv, "achieved": step_gbs, "frac": step_gbs / hbm,
                         "note": "all four kernels' algorithmic bytes per voxel-step over the whole step time"},
                "kernel_share_of_step": {k: v / sum(share_ms.values()) for k, v in share_ms.items()}}

    # plain form: one simulation per launch sequence, same work
    plain = None
    if args.plain_steps > 0:
        pplan = fwi.Plan.from_workload(wl, pairing="literal", max_shots=K, sims_per_launch=1, device=dev)
        autotune.set_schedule(pplan, dict(schedule, stream_groups=1))   # sequential simulations
        pplan.gradient(c_model, w, observed, misfit=misfit, grad=grad)
        torch.cuda.synchronize(dev)
        pt = []
        for i in range(args.plain_steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            pplan.gradient(c_model, w, observed, misfit=misfit, grad=grad)
            b.record(stream)
            flush.zero_()
            torch.cuda.synchronize(dev)
            pt.append(a.elapsed_time(b))
        pms = sum(pt) / len(pt)
        plain = {"value": vsteps / (pms / 1e3) / 1e9, "unit": UNIT,
                 "gradients_per_h": 3600.0 / (pms / 1e3), "ms_per_step": pms,
                 "form": "one simulation per launch sequence, simulations one after another "
                         "(sims_per_launch = 1, one stream group)"}
        pplan.close()
        del pplan

    # TR re-simulation restricted to a box enclosing Gamma (Sec. 3.1): the same gradient with
    # its TR simulations on a 96 x 96 x 64 box (margin 8, PML 8 inside the box)
    trbox = None
    if args.tr_box_steps > 0 and args.workload == "plain" and not args.nt:
        box = synth.tr_box(wl, 8, 8, sizes=(32, 48, 64, 80, 96, 128))
        bplan = fwi.Plan.from_workload(wl, pairing="literal", max_shots=K, device=dev, tr_box=box)
        autotune.set_schedule(bplan, schedule)
        bplan.gradient(c_model, w, observed, misfit=misfit, grad=grad)
        torch.cuda.synchronize(dev)
        bt = []
        for i in range(args.tr_box_steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            bplan.gradient(c_model, w, observed, misfit=misfit, grad=grad)
            b.record(stream)
            flush.zero_()
            torch.cuda.synchronize(dev)
            bt.append(a.elapsed_time(b))
        assert bplan.status() == fwi.FWI_OK
        bms = sum(bt) / len(bt)
        bvs = bplan.voxel_steps(K, True)
        trbox = {"value": bvs / (bms / 1e3) / 1e9, "unit": UNIT, "ms_per_step": bms,
                 "gradients_per_h": 3600.0 / (bms / 1e3), "voxel_steps_per_step": bvs,
                 "box": {"origin": list(box[0]), "size": list(box[1]), "pml": list(box[2])},
                 "gradient_speedup": (tot_ms / args.steps) / bms,
                 "form": ("TR simulations on a box enclosing Gamma (Sec. 3.1), adjoint and forward on the "
                          "whole grid; oracle parity with the same box in tests/test_gpu_tr_box.py")}
        bplan.close()
        del bplan

    # the batched form: the 16 uneven-grid instances grouped by grid into four plans replayed as
    # one captured graph, the plans in one chain (the arrangement `--workload batch` measures best)
    batched = None
    if args.batch_steps > 0 and args.workload == "plain" and not args.nt and world == 1:
        _, bgroups, btuned, (gplans, gcs, gws, gobs), bvsteps, bbytes = grouped_batch(dev)
        batch = fwi.Batch(gplans)
        batch.set_chains([0] * len(gplans))
        t0 = time.perf_counter()
        batch.gradient(gcs, gws, gobs)                 # capture and first replay
        torch.cuda.synchronize(dev)
        capture_s = time.perf_counter() - t0
        flush.zero_()
        bt = []
        with ClockSampler(local) as bclk:
            for i in range(args.batch_steps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                batch.gradient(gcs, gws, gobs)
                b.record(stream)
                flush.zero_()
                torch.cuda.synchronize(dev)
                bt.append(a.elapsed_time(b))
        assert all(p.status() == fwi.FWI_OK for p in gplans)
        bms = sum(bt) / len(bt)
        bgbs = bbytes / (bms / 1e3) / 1e9
        batched = {"value": bvsteps / (bms / 1e3) / 1e9, "unit": UNIT, "ms_per_step": bms, "steps": args.batch_steps,
                   "gradients_per_h": 3600.0 * 16 / (bms / 1e3), "voxel_steps_per_step": bvsteps,
                   "graph_nodes": batch.nodes(), "capture_and_first_run_s": capture_s,
                   "schedules": {"x".join(map(str, k)): v for k, v in btuned.items()},
                   "step_roofline": {"achieved": bgbs, "frac": bgbs / hbm, "unit": "GB/s",
                                     "alg_bytes_per_voxel_step": bbytes / bvsteps},
                   "clocks": bclk.summary(),
                   "form": ("16 encoded gradients of uneven grids (4 each of 64^3, 96x96x48, 128x128x64, "
                            "160x160x80; 1200-2000 steps), grouped by grid into four per-shot-model plans "
                            "replayed as one captured graph, the plans in one chain")}
        del batch
        for p in gplans:
            p.close()

    # the serving loop on a short Poisson stream over the 135x135x96 level (1000 steps, forward and
    # gradient requests, 2..8 encoded emitters): latency percentiles beside throughput, and how many
    # admitted requests were on the GPU at once
    served = None
    if args.serve_requests > 0 and args.workload == "plain" and not args.nt and world == 1:
        from paper_2102_00755_b300 import serve
        lv = serve.make_level("L0", synth.serving_level(0, n_src=8, seed=1000), device=dev)
        server = serve.Server([lv], device=dev, max_inflight=args.inflight)
        warm = [serve.Request(-1 - i, "L0", kind, np.eye(8)[0], 0.0)
                for i, kind in enumerate(("forward", "gradient") * 2)]
        server.run(warm, realtime=False)           # module loading, first calls, graph capture
        reqs = serve.poisson_stream(["L0"], [1], args.serve_requests, args.serve_rate, 8, seed=3000,
                                    stratified=True)
        with ClockSampler(local) as sclk:
            out = server.run(reqs, realtime=True)
        sst, res = out["stats"], out["results"]
        assert all(s_.plan.status() == fwi.FWI_OK for s_ in server.pool["L0"])
        edges = sorted([(r.admitted, 1) for r in res] + [(r.done, -1) for r in res])
        cur = peak = 0
        for _, d in edges:
            cur += d
            peak = max(peak, cur)
        svc = [r.done - r.admitted for r in res]
        served = {"value": sst["gvoxel_steps_per_s"], "unit": UNIT,
                  "latency_s": {"p50": sst["p50_s"], "p99": sst["p99_s"]},
                  "offered_req_per_s": sst["offered_req_per_s"], "achieved_req_per_s": sst["achieved_req_per_s"],
                  "requests": sst["requests"], "gradients": sst["gradients"], "gradients_per_h": sst["gradients_per_h"],
                  "in_service_s": {"p50": float(np.percentile(svc, 50)), "p99": float(np.percentile(svc, 99))},
                  "max_requests_on_gpu": peak, "mean_requests_on_gpu": float(sum(svc) / sst["wall_s"]),
                  "hbm_frac_at_125B_per_voxel_step": sst["gvoxel_steps_per_s"] * 125.125 / hbm,
                  "clocks": sclk.summary(),
                  "form": (f"{args.serve_requests} requests (half gradients, 2..8 encoded emitters) arriving as "
                           f"a seeded Poisson stream at {args.serve_rate} req/s on the 135x135x96 serving level "
                           f"(1000 steps, PML), admitted by free HBM up to {args.inflight} at a time, each on its "
                           f"own stream, pooled plans replaying captured graphs")}
        server.close()
        del server, lv

    # end to end through the public API with host buffers (pinned), copies inside
    e2e = None
    if args.e2e_steps > 0:
        hc = c_model.cpu().pin_memory()
        hw = w.cpu().pin_memory()
        ho = observed.cpu().pin_memory()
        hm = torch.empty(K, dtype=torch.float64).pin_memory()
        hg = torch.empty(wl.n_vox, dtype=torch.float64).pin_memory()
        et = []
        for i in range(args.e2e_steps + 1):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            dc = hc.to(dev, non_blocking=True)
            dw = hw.to(dev, non_blocking=True)
            do = ho.to(dev, non_blocking=True)
            m, g = plan.gradient(dc, dw, do)
            hm.copy_(m, non_blocking=True)
            hg.copy_(g, non_blocking=True)
            b.record(stream)
            torch.cuda.synchronize(dev)
            if i > 0:
                et.append(a.elapsed_time(b))
            flush.zero_()
        ems = job_time_ms(sum(et) / len(et), world, dev)
        h2d = hc.numel() * 4 + hw.numel() * 4 + ho.numel() * 4
        e2e = {"value": whole_job_rate(vsteps, world, 1, ems) / 1e9, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": hm.numel() * 8 + hg.numel() * 8, "ms_per_step": ems,
               "gradients_per_h": 3600.0 * whole_job_rate(1, world, 1, ems)}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    cpu = None if args.no_cpu_baseline or world > 1 else cpu_baseline(wl)
    sorted_ms = sorted(step_ms)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload, "grid": [wl.nx, wl.ny, wl.nz], "nt": wl.nt,
                   "super_shots": K, "n_src": int(len(wl.src_idx)), "n_rec": int(len(wl.rec_idx)),
                   "n_gamma": int(len(wl.gamma_idx)), "n_layer": int(len(wl.layer_idx)),
                   "pairing": "literal", "voxel_steps_per_step": vsteps, "fft_schedule": schedule,
                   "l2": "256 MB buffer written between timed steps; working set > 126 MB L2",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "gradients_per_h": grads_per_h,
        "latency_ms": {"p50": float(np.percentile(sorted_ms, 50)), "p99": float(np.percentile(sorted_ms, 99))},
        "plain": plain,
        "batched_vs_plain": (value / plain["value"]) if plain else None,
        "e2e": e2e,
        "tr_box": trbox,
        "batched": batched,
        "served": served,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "clocks": clocks,
        "gpu_launches": launches * args.steps,
    }
    print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
