"""FFT schedule autotuner.

For a grid shape and batch size, time short forward runs of a probe plan under
every candidate schedule (specialised vs runtime radix schedules, radix order,
z-pass tile width, split planes, stream groups) with CUDA events and keep the
fastest.  A gradient's forward phase advances K simulations and its backward phase
2K (adjoint and TR of each super-shot), so a candidate's score is the time of a
K-shot plus a 2K-shot forward run.  Results are cached in a JSON file keyed by
"nx,ny,nz,K" (default ~/.cache/fwi_b300/schedules.json, or $FWI_SCHEDULE_CACHE).
"""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np
import torch

from . import fwi

CANDIDATES = [dict(specialized=s, radix_order=r, z_tile=t, split_plane=sp, stream_groups=g)
              for sp in (0, 1) for s in (2, 1, 0) for r in (0, 1, 2) for t in (32, 16) for g in (1, 2, 4)
              if not (s >= 1 and r != 0) and not (sp == 1 and s == 1) and not (g > 1 and s != 2)]
KNOBS = ("specialized", "radix_order", "z_tile", "split_plane", "stream_groups")
MAX_SHOTS = 8          # a plan's largest batch of super-shots


def cache_path() -> str:
    return os.environ.get("FWI_SCHEDULE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "fwi_b300", "schedules.json"))


def _load(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def key_of(nx, ny, nz, K) -> str:
    return f"{nx},{ny},{nz},{K}"


def set_schedule(plan, sched: dict) -> int:
    s = fwi.fwi_schedule(sched["specialized"], sched["radix_order"], sched["z_tile"],
                         sched.get("split_plane", 0), sched.get("stream_groups", 1))
    return fwi.lib().fwi_plan_set_schedule(plan.handle, ctypes.byref(s))


def get_schedule(plan) -> dict:
    s = fwi.fwi_schedule()
    fwi._check(fwi.lib().fwi_plan_get_schedule(plan.handle, ctypes.byref(s)), "fwi_plan_get_schedule")
    return dict(specialized=s.specialized, radix_order=s.radix_order, z_tile=s.z_tile,
                split_plane=s.split_plane, stream_groups=s.stream_groups)


def tune(wl, K: int = 1, steps: int = 24, reps: int = 3, device="cuda", save=True, verbose=False) -> dict:
    """Pick the fastest schedule for wl's grid and K super-shots; returns
    {"schedule": ..., "ms": ..., "timings": [...]} and stores it in the cache.
    "ms" is a candidate's score: a K-shot plus a 2K-shot forward run of `steps` steps."""
    dev = torch.device(device)
    wav = np.asarray(wl.wavelet[:steps], dtype=np.float32)
    K2 = min(2 * K, MAX_SHOTS)
    probe = fwi.Plan(nx=wl.nx, ny=wl.ny, nz=wl.nz, pml=wl.pml, dx=wl.dx, dt=wl.dt, c_ref=wl.c_ref,
                     rho0=wl.rho0, pml_alpha=wl.pml_alpha, nt=steps, src_idx=wl.src_idx,
                     rec_idx=wl.rec_idx, layer_idx=wl.layer_idx, gamma_idx=wl.gamma_idx, wavelet=wav,
                     max_shots=K2, device=dev)
    c = torch.tensor(wl.c_model, dtype=torch.float32, device=dev).reshape(-1)
    w = torch.ones((K2, len(wl.src_idx)), dtype=torch.float32, device=dev)
    traces = torch.empty((K2, steps, len(wl.rec_idx)), dtype=torch.float32, device=dev)

    def best_ms(k):
        best = float("inf")
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            probe.forward(c, w[:k], traces[:k])
            b.record()
            torch.cuda.synchronize(dev)
            best = min(best, a.elapsed_time(b))
        return best

    timings = []
    for cand in CANDIDATES:
        if set_schedule(probe, cand) != fwi.FWI_OK:
            continue
        probe.forward(c, w, traces)
        torch.cuda.synchronize(dev)
        ms_k = best_ms(K)
        ms_2k = best_ms(K2) if K2 != K else ms_k
        timings.append(dict(cand, ms=ms_k + ms_2k, ms_k=ms_k, ms_2k=ms_2k))
        if verbose:
            print(cand, f"{ms_k + ms_2k:.3f} ms")
    probe.close()
    win = min(timings, key=lambda t: t["ms"])
    result = {"schedule": {k: win[k] for k in KNOBS},
              "ms": win["ms"], "steps": steps, "timings": timings}
    if save:
        path = cache_path()
        data = _load(path)
        data[key_of(wl.nx, wl.ny, wl.nz, K)] = result
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path + ".tmp", "w") as fh:
            json.dump(data, fh, indent=1)
        os.replace(path + ".tmp", path)
    return result


def apply_cached(plan, nx, ny, nz, K) -> bool:
    """Apply a cached schedule to `plan`; False if the cache has none for this shape."""
    ent = _load(cache_path()).get(key_of(nx, ny, nz, K))
    if not ent:
        return False
    return set_schedule(plan, ent["schedule"]) == fwi.FWI_OK
