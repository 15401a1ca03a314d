"""Host-side argument checks of the optimiser and grid-transfer entry points (Alg. 2,
App. C): every rejection happens before any device work (no GPU needed)."""
import ctypes

import pytest

from paper_2102_00755_b300 import build as fbuild
from paper_2102_00755_b300 import fwi


@pytest.fixture(scope="module")
def L():
    fbuild.build()
    return fwi.lib()


def test_lbfgs_create_and_bind_checks(L):
    for n, m in ((0, 4), (-3, 4), (100, 0), (100, 1025)):
        st, h, _ = fwi.fwi_lbfgs_create(n, m)
        assert st == fwi.FWI_EINVAL
    st, h, ws = fwi.fwi_lbfgs_create(1000, 8)
    assert st == fwi.FWI_OK and ws >= 2 * 8 * 1000 * 4       # FP32 s and y histories
    assert L.fwi_lbfgs_size(h) == 0
    # workspace: null, misaligned (not 256-byte) or too small
    assert fwi.fwi_lbfgs_bind_workspace(h, 0, ws) == fwi.FWI_EINVAL
    assert fwi.fwi_lbfgs_bind_workspace(h, 256 + 8, ws) == fwi.FWI_EINVAL
    assert fwi.fwi_lbfgs_bind_workspace(h, 256, ws - 1) == fwi.FWI_EINVAL
    # no workspace bound: push and apply refuse before any launch
    stored = ctypes.c_int32(-1)
    assert L.fwi_lbfgs_push(h, ctypes.c_void_p(256), ctypes.c_void_p(512), None, ctypes.byref(stored)) == fwi.FWI_EINVAL
    assert L.fwi_lbfgs_apply(h, ctypes.c_void_p(256), 0.0, ctypes.c_void_p(512), None) == fwi.FWI_EINVAL
    assert fwi.fwi_lbfgs_destroy(h) == fwi.FWI_OK


def test_vector_entry_point_checks(L):
    p = ctypes.c_void_p(256)
    assert fwi.fwi_vec_step_project(0, p, p, 1.0, 0.0, 1.0, None) == fwi.FWI_EINVAL
    assert fwi.fwi_vec_step_project(10, p, p, 1.0, 2.0, 1.0, None) == fwi.FWI_EINVAL     # u_min > u_max
    assert fwi.fwi_vec_step_project(10, None, p, 1.0, 0.0, 1.0, None) == fwi.FWI_EINVAL
    assert fwi.fwi_vec_accumulate(-1, p, p, 1.0, None) == fwi.FWI_EINVAL
    for kind in (-1, 3):
        assert fwi.fwi_param_to_speed(10, kind, p, p, None) == fwi.FWI_EINVAL
        assert fwi.fwi_grad_to_param(10, kind, p, p, p, None) == fwi.FWI_EINVAL


def test_resampler_checks(L):
    bad = [((0, 8, 8), (8, 8, 8), (0, 0, 0), 4.0, 1.0),          # empty axis
           ((8, 8, 8), (8, 8, 9000), (0, 0, 0), 4.0, 1.0),       # too long
           ((8, 8, 8), (16, 8, 8), (3, 0, 0), 4.0, 1.0),         # unknown window
           ((8, 8, 8), (16, 8, 8), (2, 0, 0), -1.0, 1.0),        # negative Kaiser beta
           ((8, 8, 8), (16, 8, 8), (0, 0, 0), 4.0, float("nan")),
           ((8, 8, 8), (8, 8, 8), (0, 0, 0), 4.0, 2.0)]          # identity cannot carry a scale
    for n_in, n_out, win, beta, scale in bad:
        st, h, _ = fwi.fwi_resampler_create(n_in, n_out, win, beta, scale)
        assert st == fwi.FWI_EINVAL, (n_in, n_out, win, beta, scale)
    st, h, ws = fwi.fwi_resampler_create((9, 12, 11), (17, 24, 21), (1, 1, 1), 4.0, 1.0)
    assert st == fwi.FWI_OK
    # three FP32 matrices plus two intermediates of the larger partial shape
    mats = 4 * (9 * 17 + 12 * 24 + 11 * 21)
    assert ws >= mats + 2 * 4 * 11 * 24 * 17
    assert fwi.fwi_resampler_bind_workspace(h, 256 + 16, ws) == fwi.FWI_EINVAL
    assert fwi.fwi_resampler_bind_workspace(h, 256, ws - 1) == fwi.FWI_EINVAL
    assert fwi.fwi_resampler_destroy(h) == fwi.FWI_OK
    st, h, _ = fwi.fwi_resampler_create((8, 8, 8), (8, 8, 8), (0, 0, 0), 4.0, 1.0)   # plain copy
    assert st == fwi.FWI_OK
    assert fwi.fwi_resampler_destroy(h) == fwi.FWI_OK
