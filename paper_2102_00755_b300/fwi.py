"""Thin Python binding of the C ABI in include/fwi.h (argument marshalling only).

Every step of the hot path runs in libfwi.so's CUDA kernels; PyTorch only
provides device memory and streams.  There is no CPU fallback: if the library
is missing or cannot be loaded, every call raises.

The functions fwi_plan_create ... fwi_status_string mirror the C entry points
one to one; `Plan` is a convenience wrapper that owns the workspace tensor.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfwi.so")

FWI_OK = 0
FWI_EINVAL = 1
FWI_ENOMEM = 2
FWI_EUNSTABLE = 3
FWI_ETIMEOUT = 4
FWI_ECUDA = 5
FWI_ECANCELLED = 6
FWI_ENOTSUP = 7

PAIRING = {"literal": 0, "exact": 1}

C_SYMBOLS = ("fwi_plan_create", "fwi_plan_set_tr_box", "fwi_plan_bind_workspace", "fwi_forward", "fwi_gradient",
             "fwi_forward_delayed", "fwi_gradient_delayed",
             "fwi_plan_status", "fwi_plan_voxel_steps", "fwi_plan_launches", "fwi_plan_profile",
             "fwi_plan_profile_read", "fwi_plan_set_schedule", "fwi_plan_get_schedule",
             "fwi_adjoint_source_noalloc", "fwi_batch_create",
             "fwi_batch_gradient", "fwi_batch_nodes", "fwi_batch_set_chains", "fwi_batch_destroy",
             "fwi_plan_destroy",
             "fwi_status_string", "fwi_last_cuda_error", "fwi_lbfgs_create", "fwi_lbfgs_bind_workspace",
             "fwi_lbfgs_push", "fwi_lbfgs_apply", "fwi_lbfgs_size", "fwi_lbfgs_destroy", "fwi_vec_step_project",
             "fwi_vec_accumulate", "fwi_param_to_speed", "fwi_grad_to_param", "fwi_resampler_create",
             "fwi_resampler_bind_workspace", "fwi_resample", "fwi_resampler_destroy")

NOALLOC_MAX_PARTIALS = 8192

KERNELS = {"zpass_momentum": 0, "plane_momentum": 1, "zpass_mass": 2, "plane_mass": 3}


class FwiError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        extra = ""
        if status == FWI_ECUDA:
            extra = " [" + lib().fwi_last_cuda_error().decode() + "]"
        super().__init__(f"{where}: {fwi_status_string(status)} (status {status}){extra}")


class fwi_schedule(ctypes.Structure):
    _fields_ = [("specialized", ctypes.c_int32), ("radix_order", ctypes.c_int32), ("z_tile", ctypes.c_int32),
                ("split_plane", ctypes.c_int32), ("stream_groups", ctypes.c_int32)]


class fwi_problem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("pml", ctypes.c_int32 * 3),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double), ("c_ref", ctypes.c_double),
        ("rho0", ctypes.c_double), ("pml_alpha", ctypes.c_double), ("c_rec", ctypes.c_double),
        ("nt", ctypes.c_int32), ("n_src", ctypes.c_int32), ("n_rec", ctypes.c_int32),
        ("n_layer", ctypes.c_int32), ("n_gamma", ctypes.c_int32),
        ("src_idx", ctypes.POINTER(ctypes.c_int32)), ("rec_idx", ctypes.POINTER(ctypes.c_int32)),
        ("layer_idx", ctypes.POINTER(ctypes.c_int32)), ("gamma_idx", ctypes.POINTER(ctypes.c_int32)),
        ("wavelet", ctypes.POINTER(ctypes.c_float)),
        ("pairing", ctypes.c_int32), ("max_shots", ctypes.c_int32),
        ("sims_per_launch", ctypes.c_int32), ("per_shot_models", ctypes.c_int32),
    ]


_lib = None


def lib():
    """Load libfwi.so (built in-tree); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"CUDA library not built: {LIB_PATH} (run paper_2102_00755_b300/build.py)")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
        L.fwi_plan_create.argtypes = [ctypes.POINTER(fwi_problem), ctypes.POINTER(sz), ctypes.POINTER(vp)]
        L.fwi_plan_create.restype = ctypes.c_int
        L.fwi_plan_bind_workspace.argtypes = [vp, vp, sz]
        L.fwi_plan_set_tr_box.restype = ctypes.c_int
        L.fwi_plan_set_tr_box.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                          ctypes.POINTER(sz)]
        L.fwi_plan_bind_workspace.restype = ctypes.c_int
        L.fwi_forward.argtypes = [vp, vp, vp, i32, vp, vp]
        L.fwi_forward.restype = ctypes.c_int
        L.fwi_gradient.argtypes = [vp, vp, vp, i32, vp, i32, vp, vp, vp, vp]
        L.fwi_gradient.restype = ctypes.c_int
        L.fwi_forward_delayed.argtypes = [vp, vp, vp, vp, i32, vp, vp]
        L.fwi_forward_delayed.restype = ctypes.c_int
        L.fwi_gradient_delayed.argtypes = [vp, vp, vp, vp, i32, vp, i32, i32, vp, vp, vp, vp]
        L.fwi_gradient_delayed.restype = ctypes.c_int
        L.fwi_plan_status.argtypes = [vp]
        L.fwi_plan_status.restype = ctypes.c_int
        L.fwi_plan_voxel_steps.argtypes = [vp, i32, i32]
        L.fwi_plan_voxel_steps.restype = i64
        L.fwi_plan_launches.argtypes = [vp, i32, i32]
        L.fwi_plan_launches.restype = i64
        L.fwi_plan_profile.argtypes = [vp, i32, i32, i32]
        L.fwi_plan_profile.restype = ctypes.c_int
        L.fwi_plan_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64),
                                            ctypes.POINTER(i64)]  # arrays of 4
        L.fwi_plan_profile_read.restype = ctypes.c_int
        L.fwi_adjoint_source_noalloc.argtypes = [vp, vp, i32, i32, i32, vp, vp, vp]
        L.fwi_adjoint_source_noalloc.restype = ctypes.c_int
        L.fwi_plan_set_schedule.argtypes = [vp, ctypes.POINTER(fwi_schedule)]
        L.fwi_plan_set_schedule.restype = ctypes.c_int
        L.fwi_plan_get_schedule.argtypes = [vp, ctypes.POINTER(fwi_schedule)]
        L.fwi_plan_get_schedule.restype = ctypes.c_int
        L.fwi_batch_create.argtypes = [i32, ctypes.POINTER(vp), ctypes.POINTER(vp)]
        L.fwi_batch_create.restype = ctypes.c_int
        L.fwi_batch_gradient.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(i32),
                                         ctypes.POINTER(vp), ctypes.POINTER(i32), ctypes.POINTER(vp),
                                         ctypes.POINTER(vp), vp]
        L.fwi_batch_gradient.restype = ctypes.c_int
        L.fwi_batch_nodes.argtypes = [vp]
        L.fwi_batch_nodes.restype = i64
        L.fwi_batch_set_chains.argtypes = [vp, ctypes.POINTER(i32)]
        L.fwi_batch_set_chains.restype = ctypes.c_int
        L.fwi_batch_destroy.argtypes = [vp]
        L.fwi_batch_destroy.restype = ctypes.c_int
        L.fwi_plan_destroy.argtypes = [vp]
        L.fwi_plan_destroy.restype = ctypes.c_int
        L.fwi_last_cuda_error.argtypes = []
        L.fwi_last_cuda_error.restype = ctypes.c_char_p
        L.fwi_status_string.argtypes = [ctypes.c_int]
        L.fwi_status_string.restype = ctypes.c_char_p
        dbl = ctypes.c_double
        L.fwi_lbfgs_create.argtypes = [i64, i32, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(vp)]
        L.fwi_lbfgs_create.restype = ctypes.c_int
        L.fwi_lbfgs_bind_workspace.argtypes = [vp, vp, ctypes.c_size_t]
        L.fwi_lbfgs_bind_workspace.restype = ctypes.c_int
        L.fwi_lbfgs_push.argtypes = [vp, vp, vp, vp, ctypes.POINTER(i32)]
        L.fwi_lbfgs_push.restype = ctypes.c_int
        L.fwi_lbfgs_apply.argtypes = [vp, vp, dbl, vp, vp]
        L.fwi_lbfgs_apply.restype = ctypes.c_int
        L.fwi_lbfgs_size.argtypes = [vp]
        L.fwi_lbfgs_size.restype = i32
        L.fwi_lbfgs_destroy.argtypes = [vp]
        L.fwi_lbfgs_destroy.restype = ctypes.c_int
        L.fwi_vec_step_project.argtypes = [i64, vp, vp, dbl, dbl, dbl, vp]
        L.fwi_vec_step_project.restype = ctypes.c_int
        L.fwi_vec_accumulate.argtypes = [i64, vp, vp, dbl, vp]
        L.fwi_vec_accumulate.restype = ctypes.c_int
        L.fwi_param_to_speed.argtypes = [i64, i32, vp, vp, vp]
        L.fwi_param_to_speed.restype = ctypes.c_int
        L.fwi_grad_to_param.argtypes = [i64, i32, vp, vp, vp, vp]
        L.fwi_grad_to_param.restype = ctypes.c_int
        i32x3 = ctypes.c_int32 * 3
        L.fwi_resampler_create.argtypes = [i32x3, i32x3, i32x3, dbl, dbl, ctypes.POINTER(ctypes.c_size_t),
                                           ctypes.POINTER(vp)]
        L.fwi_resampler_create.restype = ctypes.c_int
        L.fwi_resampler_bind_workspace.argtypes = [vp, vp, ctypes.c_size_t]
        L.fwi_resampler_bind_workspace.restype = ctypes.c_int
        L.fwi_resample.argtypes = [vp, vp, vp, vp]
        L.fwi_resample.restype = ctypes.c_int
        L.fwi_resampler_destroy.argtypes = [vp]
        L.fwi_resampler_destroy.restype = ctypes.c_int
        _lib = L
    return _lib


# ---- one-to-one wrappers of the C entry points ---------------------------------------
def fwi_status_string(status: int) -> str:
    return lib().fwi_status_string(status).decode()


def fwi_plan_create(prob: fwi_problem):
    ws = ctypes.c_size_t(0)
    plan = ctypes.c_void_p(0)
    st = lib().fwi_plan_create(ctypes.byref(prob), ctypes.byref(ws), ctypes.byref(plan))
    return st, plan, ws.value


def fwi_plan_set_tr_box(plan, origin, size, pml):
    """(status, new workspace bytes): TR re-simulation on the box [origin, origin + size)
    with a PML of pml cells inside it (x, y, z each)."""
    arr = ctypes.c_int32 * 3
    ws = ctypes.c_size_t(0)
    st = lib().fwi_plan_set_tr_box(plan, arr(*map(int, origin)), arr(*map(int, size)), arr(*map(int, pml)),
                                   ctypes.byref(ws))
    return st, ws.value


def fwi_plan_bind_workspace(plan, ptr: int, nbytes: int) -> int:
    return lib().fwi_plan_bind_workspace(plan, ctypes.c_void_p(ptr), nbytes)


def fwi_forward(plan, c_ptr, w_ptr, K, traces_ptr, stream) -> int:
    return lib().fwi_forward(plan, c_ptr, w_ptr, K, traces_ptr, stream)


def fwi_gradient(plan, c_ptr, w_ptr, K, obs_ptr, obs_encoded, misfit_ptr, grad_ptr, traces_ptr,
                 stream) -> int:
    return lib().fwi_gradient(plan, c_ptr, w_ptr, K, obs_ptr, obs_encoded, misfit_ptr, grad_ptr,
                              traces_ptr, stream)


def fwi_forward_delayed(plan, c_ptr, w_ptr, d_ptr, K, traces_ptr, stream) -> int:
    return lib().fwi_forward_delayed(plan, c_ptr, w_ptr, d_ptr, K, traces_ptr, stream)


def fwi_gradient_delayed(plan, c_ptr, w_ptr, d_ptr, K, obs_ptr, obs_encoded, obs_nt, misfit_ptr, grad_ptr,
                         traces_ptr, stream) -> int:
    return lib().fwi_gradient_delayed(plan, c_ptr, w_ptr, d_ptr, K, obs_ptr, obs_encoded, obs_nt, misfit_ptr,
                                      grad_ptr, traces_ptr, stream)


def fwi_lbfgs_create(n, m):
    ws = ctypes.c_size_t(0)
    h = ctypes.c_void_p(0)
    st = lib().fwi_lbfgs_create(n, m, ctypes.byref(ws), ctypes.byref(h))
    return st, h, ws.value


def fwi_lbfgs_bind_workspace(h, ptr: int, nbytes: int) -> int:
    return lib().fwi_lbfgs_bind_workspace(h, ctypes.c_void_p(ptr), nbytes)


def fwi_lbfgs_push(h, s_ptr, y_ptr, stream):
    stored = ctypes.c_int32(0)
    st = lib().fwi_lbfgs_push(h, s_ptr, y_ptr, stream, ctypes.byref(stored))
    return st, bool(stored.value)


def fwi_lbfgs_apply(h, g_ptr, h0, out_ptr, stream) -> int:
    return lib().fwi_lbfgs_apply(h, g_ptr, h0, out_ptr, stream)


def fwi_lbfgs_size(h) -> int:
    return lib().fwi_lbfgs_size(h)


def fwi_lbfgs_destroy(h) -> int:
    return lib().fwi_lbfgs_destroy(h)


def fwi_vec_step_project(n, u_ptr, z_ptr, nu, u_min, u_max, stream) -> int:
    return lib().fwi_vec_step_project(n, u_ptr, z_ptr, nu, u_min, u_max, stream)


def fwi_vec_accumulate(n, acc_ptr, u_ptr, w, stream) -> int:
    return lib().fwi_vec_accumulate(n, acc_ptr, u_ptr, w, stream)


def fwi_param_to_speed(n, kind, u_ptr, c_ptr, stream) -> int:
    return lib().fwi_param_to_speed(n, kind, u_ptr, c_ptr, stream)


def fwi_grad_to_param(n, kind, c_ptr, gc_ptr, gu_ptr, stream) -> int:
    return lib().fwi_grad_to_param(n, kind, c_ptr, gc_ptr, gu_ptr, stream)


def fwi_resampler_create(n_in, n_out, window, beta, scale=1.0):
    ws = ctypes.c_size_t(0)
    h = ctypes.c_void_p(0)
    a = ctypes.c_int32 * 3
    st = lib().fwi_resampler_create(a(*n_in), a(*n_out), a(*window), float(beta), float(scale), ctypes.byref(ws),
                                    ctypes.byref(h))
    return st, h, ws.value


def fwi_resampler_bind_workspace(h, ptr: int, nbytes: int) -> int:
    return lib().fwi_resampler_bind_workspace(h, ctypes.c_void_p(ptr), nbytes)


def fwi_resample(h, in_ptr, out_ptr, stream) -> int:
    return lib().fwi_resample(h, in_ptr, out_ptr, stream)


def fwi_resampler_destroy(h) -> int:
    return lib().fwi_resampler_destroy(h)


def fwi_plan_status(plan) -> int:
    return lib().fwi_plan_status(plan)


def fwi_plan_voxel_steps(plan, K, gradient) -> int:
    return lib().fwi_plan_voxel_steps(plan, K, gradient)


def fwi_plan_launches(plan, K, gradient) -> int:
    return lib().fwi_plan_launches(plan, K, gradient)


def fwi_plan_profile(plan, kernel, enable, capacity) -> int:
    return lib().fwi_plan_profile(plan, kernel, enable, capacity)


def fwi_plan_profile_read(plan):
    ms = (ctypes.c_double * 4)()
    n = (ctypes.c_int64 * 4)()
    s = (ctypes.c_int64 * 4)()
    st = lib().fwi_plan_profile_read(plan, ms, n, s)
    return st, list(ms), list(n), list(s)


def fwi_adjoint_source_noalloc(traces_ptr, observed_ptr, K, nt, n_rec, qcum_ptr, misfit_ptr,
                               stream) -> int:
    """Allocation-free adjoint source (misfit + cumulative residual) for callers that
    cannot allocate device memory; see include/fwi.h for limits and sharing rules."""
    return lib().fwi_adjoint_source_noalloc(traces_ptr, observed_ptr, K, nt, n_rec, qcum_ptr,
                                            misfit_ptr, stream)


def fwi_plan_set_schedule(plan, schedule: fwi_schedule) -> int:
    return lib().fwi_plan_set_schedule(plan, ctypes.byref(schedule))


def fwi_plan_get_schedule(plan, schedule: fwi_schedule) -> int:
    return lib().fwi_plan_get_schedule(plan, ctypes.byref(schedule))


def fwi_batch_create(plans):
    arr = (ctypes.c_void_p * len(plans))(*[p.value if isinstance(p, ctypes.c_void_p) else p for p in plans])
    out = ctypes.c_void_p(0)
    st = lib().fwi_batch_create(len(plans), arr, ctypes.byref(out))
    return st, out


def fwi_batch_gradient(batch, c, w, K, observed, encoded, misfit, grad, stream) -> int:
    n = len(c)
    P = lambda xs: (ctypes.c_void_p * n)(*xs)
    return lib().fwi_batch_gradient(batch, P(c), P(w), (ctypes.c_int32 * n)(*K), P(observed),
                                    (ctypes.c_int32 * n)(*encoded), P(misfit), P(grad), stream)


def fwi_batch_nodes(batch) -> int:
    return lib().fwi_batch_nodes(batch)


def fwi_batch_destroy(batch) -> int:
    return lib().fwi_batch_destroy(batch)


def fwi_plan_destroy(plan) -> int:
    return lib().fwi_plan_destroy(plan)


# ---- convenience wrapper --------------------------------------------------------------
def _i32(a):
    import numpy as np
    return np.ascontiguousarray(a, dtype=np.int32)


def _check(st, where):
    if st != FWI_OK:
        raise FwiError(st, where)


def _stream_handle(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(t: torch.Tensor, dtype, name):
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous CUDA {dtype} tensor")
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """A plan for one grid and transducer setup; owns its device workspace tensor.

    Geometry comes from keyword arguments mirroring fwi_problem (index lists and
    wavelet as host arrays).  `device` selects the CUDA device for the workspace.
    """

    def __init__(self, *, nx, ny, nz, pml, dx, dt, c_ref, rho0, pml_alpha, nt, src_idx, rec_idx,
                 layer_idx, gamma_idx, wavelet, pairing="literal", max_shots=1, c_rec=0.0,
                 sims_per_launch=0, device="cuda", workspace=None, tr_box=None, per_shot_models=False):
        import numpy as np
        self._keep = [_i32(src_idx), _i32(rec_idx), _i32(layer_idx), _i32(gamma_idx),
                      np.ascontiguousarray(wavelet, dtype=np.float32)]
        s, r, l, g, w = self._keep
        P = fwi_problem()
        P.nx, P.ny, P.nz = nx, ny, nz
        P.pml[0], P.pml[1], P.pml[2] = pml
        P.dx, P.dt, P.c_ref, P.rho0, P.pml_alpha, P.c_rec = dx, dt, c_ref, rho0, pml_alpha, c_rec
        P.nt, P.n_src, P.n_rec, P.n_layer, P.n_gamma = nt, len(s), len(r), len(l), len(g)
        ip = ctypes.POINTER(ctypes.c_int32)
        P.src_idx = s.ctypes.data_as(ip)
        P.rec_idx = r.ctypes.data_as(ip)
        P.layer_idx = l.ctypes.data_as(ip)
        P.gamma_idx = g.ctypes.data_as(ip)
        P.wavelet = w.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        P.pairing = PAIRING[pairing] if isinstance(pairing, str) else int(pairing)
        P.max_shots = max_shots
        P.sims_per_launch = sims_per_launch
        P.per_shot_models = 1 if per_shot_models else 0
        self.per_shot_models = bool(per_shot_models)
        self.prob = P
        st, plan, nbytes = fwi_plan_create(P)
        _check(st, "fwi_plan_create")
        self.handle = plan
        self.tr_box = tr_box
        if tr_box is not None:            # (origin, size, pml): TR re-simulation on a box (Sec. 3.1)
            st, nbytes = fwi_plan_set_tr_box(plan, *tr_box)
            _check(st, "fwi_plan_set_tr_box")
        self.workspace_bytes = nbytes
        self.nx, self.ny, self.nz, self.nt = nx, ny, nz, nt
        self.n_src, self.n_rec, self.max_shots = len(s), len(r), max_shots
        self.device = torch.device(device)
        if workspace is None:
            workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        self.workspace = workspace
        base = workspace.data_ptr()
        aligned = (base + 255) & ~255
        if aligned + nbytes > base + workspace.numel():
            raise ValueError("workspace tensor too small")
        with torch.cuda.device(self.device):
            _check(fwi_plan_bind_workspace(plan, aligned, nbytes), "fwi_plan_bind_workspace")

    @classmethod
    def from_workload(cls, wl, *, pairing="literal", max_shots=None, c_rec=None, pml_on=True, **kw):
        return cls(nx=wl.nx, ny=wl.ny, nz=wl.nz, pml=wl.pml if pml_on else (0, 0, 0), dx=wl.dx,
                   dt=wl.dt, c_ref=wl.c_ref, rho0=wl.rho0, pml_alpha=wl.pml_alpha, nt=wl.nt,
                   src_idx=wl.src_idx, rec_idx=wl.rec_idx, layer_idx=wl.layer_idx,
                   gamma_idx=wl.gamma_idx, wavelet=wl.wavelet, pairing=pairing,
                   max_shots=max_shots or len(wl.weights),
                   c_rec=wl.c_rec if c_rec is None else c_rec, **kw)

    @property
    def n_vox(self):
        return self.nx * self.ny * self.nz

    def forward(self, c: torch.Tensor, weights: torch.Tensor, traces: torch.Tensor = None,
                stream=None, delays: torch.Tensor = None) -> torch.Tensor:
        """Forward traces; `delays` (int32 [K][n_src], time steps) selects the delayed
        source encoding (fwi_forward_delayed)."""
        K = weights.shape[0]
        if traces is None:
            traces = torch.empty((K, self.nt, self.n_rec), dtype=torch.float32, device=c.device)
        self._check_sizes(K, c, weights, traces=traces, delays=delays)
        if delays is None:
            st = fwi_forward(self.handle, _dptr(c, torch.float32, "c"), _dptr(weights, torch.float32, "weights"),
                             K, _dptr(traces, torch.float32, "traces"), _stream_handle(stream))
            _check(st, "fwi_forward")
        else:
            st = fwi_forward_delayed(self.handle, _dptr(c, torch.float32, "c"),
                                     _dptr(weights, torch.float32, "weights"), _dptr(delays, torch.int32, "delays"),
                                     K, _dptr(traces, torch.float32, "traces"), _stream_handle(stream))
            _check(st, "fwi_forward_delayed")
        return traces

    def gradient(self, c: torch.Tensor, weights: torch.Tensor, observed: torch.Tensor, encoded=True,
                 misfit=None, grad=None, traces=None, stream=None, delays: torch.Tensor = None):
        """Misfit and gradient; with `delays` (int32 [K][n_src]) the delayed source encoding
        (fwi_gradient_delayed; raw observed data may be shorter than nt)."""
        K = weights.shape[0]
        if misfit is None:
            misfit = torch.empty(K, dtype=torch.float64, device=c.device)
        if grad is None:
            grad = torch.empty((K if self.per_shot_models else 1) * self.n_vox, dtype=torch.float64,
                               device=c.device)
        obs_nt = observed.shape[1] if (delays is not None and observed.dim() == 3) else self.nt
        self._check_sizes(K, c, weights, traces=traces, delays=delays, grad=grad, misfit=misfit,
                          observed=observed, encoded=encoded, obs_nt=obs_nt)
        tp = _dptr(traces, torch.float32, "traces") if traces is not None else ctypes.c_void_p(0)
        if delays is None:
            st = fwi_gradient(self.handle, _dptr(c, torch.float32, "c"),
                              _dptr(weights, torch.float32, "weights"), K,
                              _dptr(observed, torch.float32, "observed"), 1 if encoded else 0,
                              _dptr(misfit, torch.float64, "misfit"), _dptr(grad, torch.float64, "grad"),
                              tp, _stream_handle(stream))
            _check(st, "fwi_gradient")
        else:
            st = fwi_gradient_delayed(self.handle, _dptr(c, torch.float32, "c"),
                                      _dptr(weights, torch.float32, "weights"),
                                      _dptr(delays, torch.int32, "delays"), K,
                                      _dptr(observed, torch.float32, "observed"), 1 if encoded else 0, obs_nt,
                                      _dptr(misfit, torch.float64, "misfit"), _dptr(grad, torch.float64, "grad"),
                                      tp, _stream_handle(stream))
            _check(st, "fwi_gradient_delayed")
        return misfit, grad

    def _check_sizes(self, K, c, weights, traces=None, delays=None, grad=None, misfit=None, observed=None,
                     encoded=True, obs_nt=None):
        """The C ABI takes bare pointers: refuse tensors smaller than the call will touch."""
        need = {"c": (c, (K if self.per_shot_models else 1) * self.n_vox),
                "weights": (weights, K * self.n_src),
                "traces": (traces, K * self.nt * self.n_rec),
                "delays": (delays, K * self.n_src),
                "grad": (grad, (K if self.per_shot_models else 1) * self.n_vox),
                "misfit": (misfit, K),
                "observed": (observed, (K if encoded else self.n_src) * (obs_nt or self.nt) * self.n_rec)}
        for name, (t, n) in need.items():
            if t is not None and t.numel() < n:
                raise ValueError(f"{name}: {t.numel()} elements, the call needs {n}")

    def status(self) -> int:
        return fwi_plan_status(self.handle)

    def profile(self, kernels=("zpass_momentum", "plane_momentum", "zpass_mass", "plane_mass"),
                enable=True, capacity=65536):
        """Time every launch of the named kernels with CUDA events (see fwi_plan_profile)."""
        if isinstance(kernels, str):
            kernels = (kernels,)
        mask = 0
        for k in kernels:
            mask |= 1 << KERNELS[k]
        _check(fwi_plan_profile(self.handle, mask, 1 if enable else 0, capacity), "fwi_plan_profile")

    def profile_read(self):
        """{kernel: (total ms, launches, simulations processed)} since profiling was enabled."""
        st, ms, n, sims = fwi_plan_profile_read(self.handle)
        _check(st, "fwi_plan_profile_read")
        return {k: (ms[i], n[i], sims[i]) for k, i in KERNELS.items()}

    def voxel_steps(self, K, gradient=True) -> int:
        return fwi_plan_voxel_steps(self.handle, K, 1 if gradient else 0)

    def launches(self, K, gradient=True) -> int:
        return fwi_plan_launches(self.handle, K, 1 if gradient else 0)

    def close(self):
        if getattr(self, "handle", None):
            fwi_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several plans (possibly of different grid sizes) run as one captured CUDA graph."""

    def __init__(self, plans):
        self.plans = list(plans)
        st, self.handle = fwi_batch_create([p.handle for p in self.plans])
        _check(st, "fwi_batch_create")
        self._out = None     # output buffers kept across calls (they are part of the graph key)

    def gradient(self, cs, weights, observed, encoded=None, misfits=None, grads=None, stream=None):
        """Gradients of every member plan in one graph launch.  Without misfits/grads the
        batch returns its own output buffers, the same tensors on every call with the same
        shot counts, so that repeated calls replay the captured graph instead of capturing
        a new one (new output pointers would change the graph key); copy them before the
        next call if they must be kept."""
        n = len(self.plans)
        encoded = encoded or [True] * n
        if misfits is None or grads is None:
            shape = tuple((w.shape[0], str(c.device)) for c, w in zip(cs, weights))
            if self._out is None or self._out[0] != shape:
                self._out = (shape,
                             [torch.empty(w.shape[0], dtype=torch.float64, device=c.device)
                              for c, w in zip(cs, weights)],
                             [torch.empty((w.shape[0] if p.per_shot_models else 1) * p.n_vox,
                                          dtype=torch.float64, device=c.device)
                              for p, c, w in zip(self.plans, cs, weights)])
            misfits = self._out[1] if misfits is None else misfits
            grads = self._out[2] if grads is None else grads
        if not (len(cs) == len(weights) == len(observed) == len(encoded) == len(misfits) == len(grads) == n):
            raise ValueError("one entry per plan expected in every argument list")
        for p, c, w, o, e, m, g in zip(self.plans, cs, weights, observed, encoded, misfits, grads):
            p._check_sizes(w.shape[0], c, w, grad=g, misfit=m, observed=o, encoded=e)
        st = fwi_batch_gradient(self.handle,
                                [_dptr(c, torch.float32, "c").value for c in cs],
                                [_dptr(w, torch.float32, "weights").value for w in weights],
                                [w.shape[0] for w in weights],
                                [_dptr(o, torch.float32, "observed").value for o in observed],
                                [1 if e else 0 for e in encoded],
                                [_dptr(m, torch.float64, "misfit").value for m in misfits],
                                [_dptr(g, torch.float64, "grad").value for g in grads],
                                _stream_handle(stream))
        _check(st, "fwi_batch_gradient")
        return misfits, grads

    def nodes(self) -> int:
        return fwi_batch_nodes(self.handle)

    def set_chains(self, chain=None):
        """Plan i on chain chain[i]; chains run side by side, each chain's plans in sequence
        (None: one chain per plan; see fwi_batch_set_chains)."""
        arr = None if chain is None else (ctypes.c_int32 * len(self.plans))(*map(int, chain))
        _check(lib().fwi_batch_set_chains(self.handle, arr), "fwi_batch_set_chains")

    def close(self):
        if getattr(self, "handle", None):
            fwi_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
