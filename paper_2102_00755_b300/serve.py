"""Serving loop: continuous batching of forward and gradient requests of several
multigrid grid sizes on one GPU.

A request names a grid level, a kind (forward or gradient) and the encoding
weights of its emitters (Sec. 3.2).  Per level the server holds the model, the
transducer geometry and the raw per-emitter observed data on the device; a
request's observed super-shot is encoded on the device from the raw data
(observed_encoded = 0).  Requests are admitted as soon as a slot and enough
free device memory (the plan's workspace plus its buffers) are available, each
on its own CUDA stream, so admitted requests overlap on the GPU; the wavefields
and the checkpoint-free time-reversal state (the boundary-layer history) live in
the plan's workspace for the request's lifetime.  Each pooled plan's launch
sequence is captured once as a CUDA graph per kind and replayed.

Latency = completion time - arrival time (host clock; completion observed by
polling CUDA events).  The server reports p50 / p99 latency, gradients/h and
Gvoxel-steps/s, and the offered and achieved load.
"""
from __future__ import annotations

import dataclasses
import time
from typing import Dict, List, Optional

import numpy as np
import torch

from . import fwi


@dataclasses.dataclass
class Level:
    """One grid level: geometry, model and raw per-emitter observed data (device)."""
    name: str
    wl: object                        # synth.Workload (geometry, wavelet, models)
    c: torch.Tensor                   # current model [N] FP32
    raw_observed: Optional[torch.Tensor] = None   # [n_src, nt, n_rec] FP32


@dataclasses.dataclass
class Request:
    rid: int
    level: str
    kind: str                         # "forward" or "gradient"
    weights: np.ndarray               # [n_src] encoding weights (zeros for unused emitters)
    arrival: float                    # seconds after the stream starts


@dataclasses.dataclass
class Result:
    rid: int
    level: str
    kind: str
    arrival: float
    admitted: float
    done: float
    traces: Optional[torch.Tensor] = None
    misfit: Optional[torch.Tensor] = None
    grad: Optional[torch.Tensor] = None
    voxel_steps: int = 0

    @property
    def latency(self):
        return self.done - self.arrival


class _Slot:
    """A pooled plan with its buffers, stream and captured graphs."""

    def __init__(self, level: Level, device, pairing, use_graphs):
        wl = level.wl
        self.level = level
        self.plan = fwi.Plan.from_workload(wl, pairing=pairing, max_shots=1, device=device)
        n_src, n_rec = len(wl.src_idx), len(wl.rec_idx)
        self.w = torch.zeros((1, n_src), dtype=torch.float32, device=device)
        self.traces = torch.empty((1, wl.nt, n_rec), dtype=torch.float32, device=device)
        self.misfit = torch.empty(1, dtype=torch.float64, device=device)
        self.grad = torch.empty(wl.n_vox, dtype=torch.float64, device=device)
        self.stream = torch.cuda.Stream(device=device)
        self.graphs: Dict[str, torch.cuda.CUDAGraph] = {}
        self.warm = set()
        self.use_graphs = use_graphs
        self.busy = False
        self.done_event = torch.cuda.Event()
        self.bytes = self.plan.workspace_bytes + self.traces.numel() * 4 + self.grad.numel() * 8

    def _issue(self, kind):
        if kind == "forward":
            self.plan.forward(self.level.c, self.w, self.traces, stream=self.stream)
        else:
            self.plan.gradient(self.level.c, self.w, self.level.raw_observed, encoded=False,
                               misfit=self.misfit, grad=self.grad, traces=self.traces, stream=self.stream)

    def launch(self, kind, weights: np.ndarray):
        with torch.cuda.stream(self.stream):
            self.w.copy_(torch.from_numpy(np.asarray(weights, np.float32)[None]), non_blocking=False)
            if not self.use_graphs or kind not in self.warm:
                self._issue(kind)                 # the first call of a kind runs uncaptured
                self.warm.add(kind)
            else:
                g = self.graphs.get(kind)
                if g is None:
                    g = torch.cuda.CUDAGraph()
                    with torch.cuda.graph(g, stream=self.stream, capture_error_mode="thread_local"):
                        self._issue(kind)
                    self.graphs[kind] = g
                g.replay()
            self.done_event.record(self.stream)


class Server:
    """Continuous-batching server over a fixed set of grid levels."""

    def __init__(self, levels: List[Level], device="cuda", max_inflight=8, mem_budget=None,
                 pairing="literal", use_graphs=True):
        self.levels = {lv.name: lv for lv in levels}
        self.device = torch.device(device)
        self.max_inflight = max_inflight
        if mem_budget is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            self.mem_budget = int(0.9 * free)
        else:
            self.mem_budget = int(mem_budget)
        self.pairing = pairing
        self.use_graphs = use_graphs
        self.pool: Dict[str, List[_Slot]] = {name: [] for name in self.levels}
        self.reserved = 0
        self.refused_for_memory = 0      # requests that had to wait for memory (each counted once)
        self._refused = set()
        self._need = {}                  # slot bytes per level (a plan is built once to size it)

    def _slot_bytes(self, level: Level) -> int:
        wl = level.wl
        P, keep = _problem_for(wl, self.pairing)
        st, plan, ws = fwi.fwi_plan_create(P)
        fwi._check(st, "fwi_plan_create")
        fwi.fwi_plan_destroy(plan)
        return ws + wl.nt * len(wl.rec_idx) * 4 + wl.n_vox * 8

    def _acquire(self, level_name, rid=None) -> Optional[_Slot]:
        for s in self.pool[level_name]:
            if not s.busy:
                return s
        lv = self.levels[level_name]
        if level_name not in self._need:
            self._need[level_name] = self._slot_bytes(lv)
        need = self._need[level_name]
        if self.reserved + need > self.mem_budget:
            if rid not in self._refused:
                self._refused.add(rid)
                self.refused_for_memory += 1
            return None
        s = _Slot(lv, self.device, self.pairing, self.use_graphs)
        self.pool[level_name].append(s)
        self.reserved += s.bytes
        return s

    def _release_idle(self, need_level: str):
        """Free idle slots of other levels when a request cannot get memory."""
        for name, slots in self.pool.items():
            if name == need_level:
                continue
            keep = []
            for s in slots:
                if s.busy:
                    keep.append(s)
                else:
                    self.reserved -= s.bytes
                    s.plan.close()
            self.pool[name] = keep
        torch.cuda.empty_cache()

    def run(self, requests: List[Request], realtime=True, keep_outputs=False, poll_s=2e-4) -> dict:
        """Serve a finite stream; arrival times are honoured when realtime=True."""
        pending = sorted(requests, key=lambda r: r.arrival)
        inflight = []          # (slot, request, admitted_time)
        results: List[Result] = []
        torch.cuda.synchronize(self.device)
        t0 = time.perf_counter()
        i = 0
        while i < len(pending) or inflight:
            now = time.perf_counter() - t0
            # completions
            still = []
            for slot, req, t_adm in inflight:
                if slot.done_event.query():
                    t_done = time.perf_counter() - t0
                    wl = slot.level.wl
                    vs = slot.plan.voxel_steps(1, req.kind == "gradient")
                    res = Result(req.rid, req.level, req.kind, req.arrival, t_adm, t_done, voxel_steps=vs)
                    if keep_outputs:
                        res.traces = slot.traces.clone()
                        if req.kind == "gradient":
                            res.misfit = slot.misfit.clone()
                            res.grad = slot.grad.clone()
                    slot.busy = False
                    results.append(res)
                else:
                    still.append((slot, req, t_adm))
            inflight = still
            # admissions (continuous batching: whenever a slot and memory are free)
            while i < len(pending) and len(inflight) < self.max_inflight:
                req = pending[i]
                if realtime and req.arrival > now:
                    break
                slot = self._acquire(req.level, req.rid)
                if slot is None and not inflight:
                    self._release_idle(req.level)
                    slot = self._acquire(req.level, req.rid)
                if slot is None:
                    break
                slot.busy = True
                slot.launch(req.kind, req.weights)
                inflight.append((slot, req, time.perf_counter() - t0))
                i += 1
            if inflight or (i < len(pending)):
                time.sleep(poll_s)
        wall = time.perf_counter() - t0
        lat = np.array([r.latency for r in results])
        grads = [r for r in results if r.kind == "gradient"]
        vsteps = sum(r.voxel_steps for r in results)
        span = max(r.arrival for r in requests) if requests else 0.0
        stats = {
            "requests": len(results), "gradients": len(grads), "wall_s": wall,
            "p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_s": float(np.percentile(lat, 99)) if len(lat) else None,
            "gradients_per_h": 3600.0 * len(grads) / wall if wall > 0 else None,
            "gvoxel_steps_per_s": vsteps / wall / 1e9 if wall > 0 else None,
            "offered_req_per_s": len(requests) / span if span > 0 else None,
            "achieved_req_per_s": len(results) / wall if wall > 0 else None,
            "max_inflight": self.max_inflight, "refused_for_memory": self.refused_for_memory,
            "mem_budget_gb": self.mem_budget / 1e9,
        }
        return {"stats": stats, "results": sorted(results, key=lambda r: r.rid)}

    def close(self):
        for slots in self.pool.values():
            for s in slots:
                s.plan.close()
        self.pool = {name: [] for name in self.levels}
        self.reserved = 0


def _problem_for(wl, pairing):
    """fwi_problem of a workload (used to query a plan's workspace size)."""
    import numpy as _np
    keep = [_np.ascontiguousarray(a, dtype=_np.int32) for a in (wl.src_idx, wl.rec_idx, wl.layer_idx, wl.gamma_idx)]
    wav = _np.ascontiguousarray(wl.wavelet, dtype=_np.float32)
    P = fwi.fwi_problem()
    P.nx, P.ny, P.nz = wl.nx, wl.ny, wl.nz
    P.pml[0], P.pml[1], P.pml[2] = wl.pml
    P.dx, P.dt, P.c_ref, P.rho0, P.pml_alpha, P.c_rec = wl.dx, wl.dt, wl.c_ref, wl.rho0, wl.pml_alpha, 0.0
    P.nt, P.n_src, P.n_rec, P.n_layer, P.n_gamma = wl.nt, *[len(k) for k in keep]
    import ctypes
    ip = ctypes.POINTER(ctypes.c_int32)
    P.src_idx, P.rec_idx, P.layer_idx, P.gamma_idx = [k.ctypes.data_as(ip) for k in keep]
    P.wavelet = wav.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    P.pairing = fwi.PAIRING[pairing]
    P.max_shots = 1
    P.sims_per_launch = 0
    return P, (keep, wav)


def make_level(name, wl, device="cuda") -> Level:
    """Build a level: current model on the device and raw per-emitter observed data
    (one forward per emitter of the true model, through this library)."""
    dev = torch.device(device)
    c_true = torch.tensor(wl.c_true, dtype=torch.float32, device=dev).reshape(-1)
    c = torch.tensor(wl.c_model, dtype=torch.float32, device=dev).reshape(-1)
    n_src = len(wl.src_idx)
    # forward only: no boundary-layer history is recorded, so the plan gets one-voxel
    # Gamma and layer lists instead of reserving K * nt * |layer| floats
    fwd = dataclasses.replace(wl, layer_idx=wl.layer_idx[:1], gamma_idx=wl.gamma_idx[:1])
    plan = fwi.Plan.from_workload(fwd, max_shots=min(n_src, 8), device=dev)
    raw = torch.empty((n_src, wl.nt, len(wl.rec_idx)), dtype=torch.float32, device=dev)
    for s0 in range(0, n_src, 8):
        k = min(8, n_src - s0)
        w = torch.zeros((k, n_src), dtype=torch.float32, device=dev)
        w[torch.arange(k), torch.arange(s0, s0 + k)] = 1.0
        plan.forward(c_true, w, raw[s0:s0 + k])
    torch.cuda.synchronize(dev)
    plan.close()
    del plan
    torch.cuda.empty_cache()
    return Level(name, wl, c, raw)


def stratified_draw(mix: List[float], n: int, rng) -> np.ndarray:
    """Category of each of n draws with counts exactly proportional to mix (largest-remainder
    rounding), in a seeded random order."""
    p = np.asarray(mix, dtype=np.float64) / np.sum(mix)
    counts = np.floor(p * n).astype(int)
    rest = p * n - counts
    for i in np.argsort(-rest, kind="stable")[:n - counts.sum()]:
        counts[i] += 1
    cats = np.repeat(np.arange(len(mix)), counts)
    rng.shuffle(cats)
    return cats


def poisson_stream(levels: List[str], mix: List[float], n: int, rate: float, n_src: int, seed: int,
                   min_src: int = 2, max_src: int = 8, p_gradient: float = 0.5,
                   stratified: bool = False) -> List[Request]:
    """Seeded Poisson arrivals; level by mix weights; kind by p_gradient; 2..8 active
    emitters with Rademacher weights (the remaining emitters get weight 0).  With
    stratified=True the level counts are exactly proportional to the mix and each level's
    requests are split between gradients and forwards by p_gradient (seeded order), so a
    finite stream carries the intended mix instead of a random draw of it."""
    rng = np.random.default_rng(seed)
    t = 0.0
    p = np.asarray(mix, dtype=np.float64) / np.sum(mix)
    out = []
    if stratified:
        lv_of = stratified_draw(mix, n, rng)
        kind_of = np.zeros(n, dtype=bool)
        for li in range(len(levels)):
            idx = np.flatnonzero(lv_of == li)
            kind_of[idx] = stratified_draw([p_gradient, 1.0 - p_gradient], len(idx), rng) == 0
    for rid in range(n):
        t += rng.exponential(1.0 / rate)
        if stratified:
            lv = levels[lv_of[rid]]
            kind = "gradient" if kind_of[rid] else "forward"
        else:
            lv = levels[rng.choice(len(levels), p=p)]
            kind = "gradient" if rng.random() < p_gradient else "forward"
        k = int(rng.integers(min_src, min(max_src, n_src) + 1))
        w = np.zeros(n_src)
        active = rng.choice(n_src, size=k, replace=False)
        w[active] = np.where(rng.integers(0, 2, size=k) == 1, 1.0, -1.0)
        out.append(Request(rid, lv, kind, w, t))
    return out
