"""Stochastic L-BFGS (Alg. 2) driving fwi_gradient, on the device.

`SLBFGS` runs Alg. 2's control flow on the host: per iteration i the gradient
estimator is evaluated twice with the same stochastic approximation n = i,
at u and at the trial point u + nu z; the pair enters the device history; the
step z - H G_z is projected onto [u_min, u_max]; the energy estimate is
min(F_u, F_z), and after its first increase the iterates are averaged with
weights w(i) (i^3 by default).  Every vector operation runs in the library's
kernels (two-loop recursion, projected step, averaging); PyTorch only holds the
device buffers.

`FwiEstimator` is the estimator g(u, theta, n) of Sec. 3.2: the mean misfit of K
super-shots with Rademacher weights drawn from seed n, and its gradient with
respect to the chosen parameter (u = c, 1/c or 1/c^2, the squared slowness
found fastest in Sec. 4.4), from fwi_gradient (or the delayed encoding of
Eq. 13 when tau > 0, delays d_i tau with d_i ~ U[0, 1] from the same seed).

Readings where Alg. 2 leaves a choice: H_0 = (s'y / y'y) I of the newest pair
unless h0 is given; pairs without positive curvature are not stored; no line
search; the trial point is projected onto the bounds too, and the stored pair
is (u_trial - u, G_z - G_u).
"""
from __future__ import annotations

import math
from typing import Callable, List, Optional, Tuple

import torch

from . import fwi, synth

PARAM_KINDS = {"speed": 0, "slowness": 1, "squared_slowness": 2}


def _vp(t: torch.Tensor, dtype):
    return fwi._dptr(t, dtype, "vector")


class LBFGSHistory:
    """Device L-BFGS history of at most m pairs (fwi_lbfgs_*)."""

    def __init__(self, n: int, m: int, device=None):
        self.n, self.m = int(n), int(m)
        st, self.handle, ws = fwi.fwi_lbfgs_create(self.n, self.m)
        fwi._check(st, "fwi_lbfgs_create")
        dev = torch.device(device) if device is not None else torch.device("cuda")
        self.ws = torch.empty(ws + 256, dtype=torch.uint8, device=dev)
        base = self.ws.data_ptr()
        off = (-base) % 256
        fwi._check(fwi.fwi_lbfgs_bind_workspace(self.handle, base + off, ws), "fwi_lbfgs_bind_workspace")

    def push(self, s: torch.Tensor, y: torch.Tensor, stream=None) -> bool:
        st, stored = fwi.fwi_lbfgs_push(self.handle, _vp(s, torch.float64), _vp(y, torch.float64),
                                        fwi._stream_handle(stream))
        fwi._check(st, "fwi_lbfgs_push")
        return stored

    def apply(self, g: torch.Tensor, h0: float = 0.0, out: torch.Tensor = None, stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty_like(g)
        fwi._check(fwi.fwi_lbfgs_apply(self.handle, _vp(g, torch.float64), float(h0), _vp(out, torch.float64),
                                       fwi._stream_handle(stream)), "fwi_lbfgs_apply")
        return out

    def __len__(self):
        return fwi.fwi_lbfgs_size(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            fwi.fwi_lbfgs_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def step_project(u: torch.Tensor, z: torch.Tensor, nu: float, u_min: float, u_max: float, stream=None):
    fwi._check(fwi.fwi_vec_step_project(u.numel(), _vp(u, torch.float64), _vp(z, torch.float64), float(nu),
                                        float(u_min), float(u_max), fwi._stream_handle(stream)),
               "fwi_vec_step_project")


def accumulate(acc: torch.Tensor, u: torch.Tensor, w: float, stream=None):
    fwi._check(fwi.fwi_vec_accumulate(acc.numel(), _vp(acc, torch.float64), _vp(u, torch.float64), float(w),
                                      fwi._stream_handle(stream)), "fwi_vec_accumulate")


class SLBFGS:
    """Alg. 2.  estimator(u, theta, n) -> (F: float, G: FP64 CUDA tensor like u)."""

    def __init__(self, estimator: Callable, nu: float, m: int = 64, h0: Optional[float] = None,
                 weight: Callable[[int], float] = lambda i: float(i) ** 3, u_min: float = -math.inf,
                 u_max: float = math.inf, theta: Callable[[int], float] = lambda i: 0.0):
        self.estimator, self.nu, self.m, self.h0 = estimator, float(nu), int(m), h0
        self.weight, self.u_min, self.u_max, self.theta = weight, float(u_min), float(u_max), theta

    def run(self, u0: torch.Tensor, n_evl: int) -> Tuple[torch.Tensor, List[float]]:
        u = u0.detach().to(torch.float64).clone().contiguous()
        hist = LBFGSHistory(u.numel(), self.m, u.device)
        u_bar = torch.zeros_like(u)
        u_hat = u.clone()
        z, hz, trial, s, y = (torch.empty_like(u) for _ in range(5))
        w_bar, J_prev, averaging, i, evl = 0.0, math.inf, False, 0, 0
        h0 = 0.0 if self.h0 is None else float(self.h0)
        Js: List[float] = []
        while evl < n_evl:
            i += 1
            F_u, G_u = self.estimator(u, self.theta(i), i)
            evl += 1
            hist.apply(G_u, h0, out=hz)                 # z = -H G_u
            z.zero_()
            accumulate(z, hz, -1.0)
            trial.copy_(u)
            step_project(trial, z, self.nu, self.u_min, self.u_max)
            F_z, G_z = self.estimator(trial, self.theta(i), i)
            evl += 1
            s.copy_(trial)                              # s = u_trial - u, y = G_z - G_u
            accumulate(s, u, -1.0)
            y.copy_(G_z)
            accumulate(y, G_u, -1.0)
            hist.push(s, y)
            hist.apply(G_z, h0, out=hz)                 # z = z - H G_z
            accumulate(z, hz, -1.0)
            step_project(u, z, self.nu, self.u_min, self.u_max)
            J = min(F_u, F_z)
            if averaging:
                w = self.weight(i)
                accumulate(u_bar, u, w)
                w_bar += w
                u_hat.zero_()
                accumulate(u_hat, u_bar, 1.0 / w_bar)
            else:
                if J > J_prev:
                    averaging = True
                u_hat.copy_(u)
            J_prev = J
            Js.append(J)
        hist.close()
        return u_hat, Js


class FwiEstimator:
    """g(u, theta, n): mean misfit and gradient of K encoded super-shots (Sec. 3.2).

    plan:      fwi.Plan (max_shots >= K)
    raw:       device [n_src][nt_data][n_rec] per-emitter observed data (encoded on the
               device with the seed-n weights and, with tau > 0, delays)
    param:     "speed", "slowness" or "squared_slowness"
    """

    def __init__(self, plan, raw: torch.Tensor, K: int, param: str = "squared_slowness", tau: int = 0,
                 seed0: int = 0):
        self.plan, self.raw, self.K, self.kind = plan, raw, int(K), PARAM_KINDS[param]
        self.tau, self.seed0 = int(tau), int(seed0)
        self.n_src = raw.shape[0]
        self.c = torch.empty(plan.n_vox, dtype=torch.float32, device=raw.device)
        self.gu = None

    def speed(self, u: torch.Tensor) -> torch.Tensor:
        fwi._check(fwi.fwi_param_to_speed(u.numel(), self.kind, _vp(u, torch.float64), _vp(self.c, torch.float32),
                                          fwi._stream_handle(None)), "fwi_param_to_speed")
        return self.c

    def __call__(self, u: torch.Tensor, theta: float, n: int):
        c = self.speed(u)
        w, d = synth.encoding_draws(self.seed0 + n, self.K, self.n_src, self.tau)
        wt = torch.tensor(w, dtype=torch.float32, device=u.device)
        if self.tau > 0:
            D, gc = self.plan.gradient(c, wt, self.raw, encoded=False,
                                       delays=torch.tensor(d, dtype=torch.int32, device=u.device))
        else:
            D, gc = self.plan.gradient(c, wt, self.raw, encoded=False)
        st = self.plan.status()
        if st != fwi.FWI_OK:
            raise fwi.FwiError(st, "fwi_gradient")
        gu = torch.empty_like(u)
        fwi._check(fwi.fwi_grad_to_param(u.numel(), self.kind, _vp(c, torch.float32), _vp(gc, torch.float64),
                                         _vp(gu, torch.float64), fwi._stream_handle(None)), "fwi_grad_to_param")
        return float(D.mean().item()), gu
