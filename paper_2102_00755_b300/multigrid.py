"""Grid transfers of the coarse-to-fine scheme (Sec. 3.3, App. C) on the device.

`Resampler` wraps fwi_resampler_*: separable periodic Fourier resampling of a
[n2][n1][n0] FP32 array, with an optional Blackman (model) or Kaiser (time
series) window per axis and an output scale.  `upsample_model` moves a sound
speed model from a coarse physical grid to a finer one (Blackman smoothing);
`downsample_data` moves per-emitter traces [n_src][nt][n_rec] to a coarser time
grid (Kaiser low-pass) and scales them by eta^(d-1); `embed_physical` /
`physical` move between a computational grid (PML inside) and its physical part.
"""
from __future__ import annotations

import torch

from . import fwi

WINDOW = {"none": 0, "blackman": 1, "kaiser": 2}


class Resampler:
    def __init__(self, shape_in, shape_out, windows=("none", "none", "none"), beta: float = 4.0,
                 scale: float = 1.0, device=None):
        """shape_in / shape_out: (n2, n1, n0) array shapes; windows per axis (n0, n1, n2)."""
        n_in = (shape_in[2], shape_in[1], shape_in[0])
        n_out = (shape_out[2], shape_out[1], shape_out[0])
        self.shape_out = tuple(shape_out)
        st, self.handle, ws = fwi.fwi_resampler_create(n_in, n_out, [WINDOW[w] for w in windows], beta, scale)
        fwi._check(st, "fwi_resampler_create")
        dev = torch.device(device) if device is not None else torch.device("cuda")
        self.ws = torch.empty(ws + 256, dtype=torch.uint8, device=dev)
        base = self.ws.data_ptr()
        fwi._check(fwi.fwi_resampler_bind_workspace(self.handle, base + (-base) % 256, ws),
                   "fwi_resampler_bind_workspace")

    def __call__(self, x: torch.Tensor, out: torch.Tensor = None, stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty(self.shape_out, dtype=torch.float32, device=x.device)
        fwi._check(fwi.fwi_resample(self.handle, fwi._dptr(x, torch.float32, "in"), fwi._dptr(out, torch.float32, "out"),
                                    fwi._stream_handle(stream)), "fwi_resample")
        return out

    def close(self):
        if getattr(self, "handle", None):
            fwi.fwi_resampler_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def upsample_model(c: torch.Tensor, shape_fine) -> torch.Tensor:
    """Fourier interpolation with Blackman smoothing of a model [nz][ny][nx] (App. C)."""
    r = Resampler(c.shape, shape_fine, ("blackman", "blackman", "blackman"), device=c.device)
    return r(c.contiguous())


def downsample_data(data: torch.Tensor, nt_out: int, eta: float, d: int = 3, beta: float = 4.0) -> torch.Tensor:
    """Per-emitter traces [n_src][nt][n_rec] to nt_out samples: Kaiser-windowed Fourier
    resampling in time, scaled by eta^(d-1) (App. C)."""
    n_src, nt, n_rec = data.shape
    r = Resampler(data.shape, (n_src, nt_out, n_rec), ("none", "kaiser", "none"), beta=beta,
                  scale=float(eta) ** (d - 1), device=data.device)
    return r(data.contiguous())


def physical(c: torch.Tensor, pml) -> torch.Tensor:
    """The physical part [pz:-pz, py:-py, px:-px] of a model on a grid with the PML inside."""
    px, py, pz = pml
    nz, ny, nx = c.shape
    return c[pz:nz - pz, py:ny - py, px:nx - px].contiguous()


def embed_physical(c_phys: torch.Tensor, shape, pml, fill: float) -> torch.Tensor:
    """A model on the computational grid `shape` (nz, ny, nx) whose physical part is c_phys
    and whose PML region is `fill` (water)."""
    px, py, pz = pml
    out = torch.full(shape, fill, dtype=torch.float32, device=c_phys.device)
    out[pz:shape[0] - pz, py:shape[1] - py, px:shape[2] - px] = c_phys
    return out


def coarse_to_fine(stages, n_evl, nu: float = 1.0, m: int = 8, h0_frac: float = 0.01, K: int = 1,
                   param: str = "squared_slowness", c_min: float = 1350.0, c_max: float = 1800.0, seed0: int = 0):
    """Coarse-to-fine inversion (Sec. 3.3): SLBFGS (Alg. 2) on each grid in turn, the
    result transferred to the next grid by `upsample_model` on the physical region.

    stages: list of (plan, raw observed data [n_src][nt][n_rec] on that grid, pml,
            shape (nz, ny, nx)), coarse to fine, each plan with max_shots >= K; n_evl:
            estimator evaluations per stage; K: super-shots per estimate.
    Returns the final model [nz][ny][nx] and the energy estimates of every stage.
    The initial model of the first stage is water.  h0 is chosen per stage so that the
    first step changes the parameter by about h0_frac of its norm.
    """
    from . import slbfgs
    from .synth import C_WATER
    kind = slbfgs.PARAM_KINDS[param]
    to_u = {0: lambda c: c, 1: lambda c: 1.0 / c, 2: lambda c: 1.0 / (c * c)}[kind]
    u_lo, u_hi = sorted((to_u(c_min), to_u(c_max)))
    c = None
    energies = []
    for plan, raw, pml, shape in stages:
        if c is None:
            c = torch.full(shape, C_WATER, dtype=torch.float32, device=raw.device)
        else:
            phys = upsample_model(physical(c, prev_pml), (shape[0] - 2 * pml[2], shape[1] - 2 * pml[1],
                                                          shape[2] - 2 * pml[0]))
            c = embed_physical(phys, shape, pml, C_WATER)
        est = slbfgs.FwiEstimator(plan, raw, K=K, param=param, seed0=seed0)
        u0 = to_u(c.reshape(-1).to(torch.float64))
        _, g0 = est(u0, 0.0, 0)
        h0 = h0_frac * float(u0.norm()) / max(float(g0.norm()), 1e-300)
        u, Js = slbfgs.SLBFGS(est, nu=nu, m=m, h0=h0, u_min=u_lo, u_max=u_hi).run(u0, n_evl)
        c = est.speed(u.contiguous()).clone().reshape(shape)
        energies.append(Js)
        prev_pml = pml
    return c, energies
