"""The allocation-free adjoint-source entry point, checked against fwi_gradient.

fwi_adjoint_source_noalloc serves callers that cannot allocate device memory
(they run from a fixed, pre-carved memory pool or must keep their device
footprint constant): its scratch is a file-scope device array instead of a
workspace.  On two calls in a row (the second, smaller one reuses the array the
first, larger one left behind) its misfit must equal both the misfit that
fwi_gradient reports for the same simulated traces and observed data and
0.5 ||q||^2 summed in FP64 on the host, and its cumulative residual must equal
the FP64 cumulative sum of the time-reversed residual.

This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2102_00755_b300 import build as fbuild
from paper_2102_00755_b300 import fwi, synth

pytestmark = pytest.mark.gpu

TOL_MISFIT = 1e-12     # same FP64 arithmetic; only the summation order may differ
TOL_Q = 1e-6           # FP32 storage of an FP64 running sum


def _dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _case(K, n_rec, seed):
    """Simulated and observed traces of one workload, and fwi_gradient's misfit for them."""
    wl = synth.small_workload(24, 20, 18, 80, pml=4, n_src=3, n_rec=n_rec, K=K, layer=2, seed=seed)
    plan = fwi.Plan.from_workload(wl, max_shots=K)
    w = _dev(wl.weights)
    observed = plan.forward(_dev(wl.c_true).reshape(-1), w)
    traces = torch.empty((K, wl.nt, n_rec), dtype=torch.float32, device="cuda")
    D_ref, _ = plan.gradient(_dev(wl.c_model).reshape(-1), w, observed, traces=traces)
    assert plan.status() == fwi.FWI_OK
    return traces, observed, D_ref.cpu().numpy()


def test_noalloc_adjoint_source_matches_gradient_entry_point():
    # The first call is the larger one (3 shots x 2 blocks of receivers = 6 partial sums in
    # the shared array), the second the smaller (2 x 1): a second call that read partial
    # sums left behind by the first would give a wrong misfit.
    fbuild.build()
    cases = [_case(3, 300, 7), _case(2, 24, 8)]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, (traces, observed, D_ref) in enumerate(cases):
        K, nt, n_rec = traces.shape
        f = traces.cpu().numpy().astype(np.float64)
        o = observed.cpu().numpy().astype(np.float64)
        q = f[:, ::-1] - o[:, ::-1]                       # time-reversed residual, FP64
        D_fp64 = 0.5 * np.sum(q * q, axis=(1, 2))
        Q_ref = np.cumsum(q, axis=1)
        qcum = torch.full((K, nt, n_rec), float("nan"), dtype=torch.float32, device="cuda")
        misfit = torch.full((K,), float("nan"), dtype=torch.float64, device="cuda")
        st = fwi.fwi_adjoint_source_noalloc(_ptr(traces), _ptr(observed), K, nt, n_rec, _ptr(qcum),
                                            _ptr(misfit), stream)
        assert st == fwi.FWI_OK, call
        torch.cuda.synchronize()
        D = misfit.cpu().numpy()
        assert np.all(D_fp64 > 0), call
        # against the existing entry point's misfit (same traces and observed data) ...
        assert np.all(np.abs(D - D_ref) <= TOL_MISFIT * np.abs(D_ref)), (call, D, D_ref)
        # ... and against 0.5 ||q||^2 summed in FP64 on the host from the copied traces
        assert np.all(np.abs(D - D_fp64) <= TOL_MISFIT * D_fp64), (call, D, D_fp64)
        Q = qcum.cpu().numpy()
        assert np.linalg.norm(Q - Q_ref) <= TOL_Q * np.linalg.norm(Q_ref), call


def test_noalloc_rejects_sizes_beyond_its_scratch():
    fbuild.build()
    t = torch.zeros(8, dtype=torch.float32, device="cuda")
    d = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    too_many_receivers = 256 * (fwi.NOALLOC_MAX_PARTIALS // 4 + 1)
    st = fwi.fwi_adjoint_source_noalloc(_ptr(t), _ptr(t), 4, 1, too_many_receivers, _ptr(t), _ptr(d),
                                        stream)
    assert st == fwi.FWI_EINVAL
    st = fwi.fwi_adjoint_source_noalloc(_ptr(t), _ptr(t), 33, 1, 1, _ptr(t), _ptr(d), stream)
    assert st == fwi.FWI_EINVAL
