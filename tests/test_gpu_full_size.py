"""Parity at the full grid sizes the benchmark and the serving levels run.

The time-stepping oracle is too slow at these sizes, so the forward path is
checked against the closed-form traces of a homogeneous periodic medium (App. B:
the k-space scheme is exact per Fourier mode there), which the oracle is pinned
to on small grids.  Every schedule the plan accepts at that size is run (the
480 x 480 planes only fit the split-plane path).  The gradient path is checked
at the largest serving grid through properties that hold at any size: the
misfit equals 0.5 ||f - f_obs||^2 of the returned traces, the gradient is zero
outside Gamma and exactly zero for zero residual, and it is linear in the
residual (the adjoint equation is linear in its source).
"""
import numpy as np
import pytest
import torch

from oracle import closed_form
from paper_2102_00755_b300 import build as fbuild
from paper_2102_00755_b300 import autotune, fwi, synth

from . import oracle_cases as oc

pytestmark = pytest.mark.gpu

TOL_TRACES = 1e-4
TOL_GRAD = 1e-3          # gradient rel l2 of FP32 fields against exact arithmetic
NT = 100


@pytest.fixture(scope="module", autouse=True)
def _built():
    fbuild.build()
    fwi.lib()


def _dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _homogeneous_workload(shape, c):
    """One emitter near a corner, receivers at offsets of 2..15 cells on every axis,
    several of them across the periodic wrap; uniform c; PML thickness 0."""
    nx, ny, nz = shape
    dx = 0.5e-3
    dt = synth.time_step(dx)
    sx, sy, sz = 3, 4, 2
    src = sx + nx * (sy + ny * sz)
    offs = [(5, 0, 0), (0, 7, 0), (0, 0, 9), (-6, 0, 0), (0, -8, 0), (0, 0, -5),
            (4, -4, 3), (-9, 6, -7), (12, 2, 1), (2, 15, -3), (-3, -2, 13), (8, 8, 8)]
    rec = np.array([(sx + a) % nx + nx * (((sy + b) % ny) + ny * ((sz + d) % nz)) for a, b, d in offs],
                   dtype=np.int32)
    cc = np.full((nz, ny, nx), c, dtype=np.float32)
    one = np.array([src], dtype=np.int32)
    wl = synth.Workload(f"homog-{nx}x{ny}x{nz}", nx, ny, nz, (0, 0, 0), dx, dt, NT, cc, cc,
                        one, rec, one, one, synth.ricker(NT, dt, 1.0e6), np.ones((1, 1)))
    return wl, src, rec


SHAPES = [(128, 128, 64), (135, 135, 96), (243, 243, 135), (480, 480, 256)]


@pytest.mark.parametrize("shape,c", [(s, 1500.0) for s in SHAPES] + [((480, 480, 256), 1800.0)])
def test_full_size_forward_matches_closed_form(shape, c):
    wl, src, rec = _homogeneous_workload(shape, c)
    ref = closed_form.homogeneous_traces(shape, wl.dx, wl.dt, wl.c_ref, c, src, rec, wl.wavelet, NT)
    assert np.abs(ref).max() > 0
    plan = fwi.Plan.from_workload(wl, max_shots=1, pml_on=False)
    cdev, w = _dev(wl.c_model).reshape(-1), _dev(wl.weights)
    default = autotune.get_schedule(plan)
    seen = 0
    for cand in [default] + list(autotune.CANDIDATES):
        if autotune.set_schedule(plan, cand) != fwi.FWI_OK:
            continue
        tr = plan.forward(cdev, w).cpu().numpy()[0].astype(np.float64)
        assert plan.status() == fwi.FWI_OK
        assert oc.rel(tr, ref) < TOL_TRACES, (cand, oc.rel(tr, ref))
        seen += 1
    assert seen >= 2
    plan.close()


def test_full_size_gradient_properties_largest_level():
    wl = synth.serving_level(2, n_src=8, seed=1000)
    nt = 100
    wl.nt, wl.wavelet = nt, wl.wavelet[:nt]
    # transducers on Gamma's boundary layer: the forward and adjoint fields enter Gamma
    # within these few steps (from the bowl they would need about 400)
    lay = wl.layer_idx
    wl.src_idx = lay[:: len(lay) // 8][:8].copy()
    wl.rec_idx = lay[len(lay) // 512 // 2:: len(lay) // 512][:512].copy()
    plan = fwi.Plan.from_workload(wl, max_shots=1)
    c = _dev(wl.c_model).reshape(-1)
    w = _dev(wl.weights[:1])
    f = plan.forward(c, w).clone()
    rng = np.random.default_rng(3)
    scale = float(f.abs().max())
    r_a = _dev(scale * 0.1 * rng.standard_normal(f.shape))
    r_b = _dev(scale * 0.1 * rng.standard_normal(f.shape))

    def grad(obs):
        tr = torch.empty_like(f)
        D, g = plan.gradient(c, w, obs, traces=tr)
        torch.cuda.synchronize()
        assert plan.status() == fwi.FWI_OK
        return tr, D.cpu().numpy(), g.cpu().numpy()

    tr0, D0, g0 = grad(f)
    assert torch.equal(tr0, f)
    assert D0[0] == 0.0 and not np.any(g0)
    tr_a, D_a, g_a = grad(f - r_a)
    _, _, g_b = grad(f - r_b)
    _, _, g_ab = grad(f - r_a - r_b)
    res = (tr_a.double() - (f - r_a).double()).cpu().numpy()
    assert abs(D_a[0] - 0.5 * np.sum(res ** 2)) <= 1e-9 * D_a[0]
    gam = np.zeros(wl.n_vox, bool)
    gam[wl.gamma_idx] = True
    assert not np.any(g_a[~gam])
    assert np.any(g_a[gam])
    assert oc.rel(g_ab, g_a + g_b) < 1e-4
    plan.close()


def test_bench_configuration_full_length_gradient_properties():
    """The timed workload itself: the 128x128x64 phantom with all 1500 steps, four super-shots,
    in the default launch configuration (two-step kernels, stream groups).  Properties that hold
    at any size: zero residual gives a zero misfit and gradient; the misfit is 0.5 ||q||^2 of the
    returned traces; the gradient lives on Gamma and is linear in the residual; and it is the
    mean over the super-shots of the per-shot gradients of the same problem run as instances."""
    wl = synth.config2()
    K = len(wl.weights)
    plan = fwi.Plan.from_workload(wl, max_shots=K)
    c = _dev(wl.c_model).reshape(-1)
    w = _dev(wl.weights)
    f = plan.forward(c, w).clone()
    rng = np.random.default_rng(5)
    scale = float(f.abs().max())
    r_a = _dev(scale * 0.05 * rng.standard_normal(f.shape))
    r_b = _dev(scale * 0.05 * rng.standard_normal(f.shape))

    def grad(obs):
        tr = torch.empty_like(f)
        D, g = plan.gradient(c, w, obs, traces=tr)
        torch.cuda.synchronize()
        assert plan.status() == fwi.FWI_OK
        return tr, D.cpu().numpy(), g.cpu().numpy()

    tr0, D0, g0 = grad(f)
    assert torch.equal(tr0, f)
    assert not np.any(D0) and not np.any(g0)
    tr_a, D_a, g_a = grad(f - r_a)
    _, _, g_b = grad(f - r_b)
    _, _, g_ab = grad(f - r_a - r_b)
    res = (tr_a.double() - (f - r_a).double()).cpu().numpy()
    assert np.all(np.abs(D_a - 0.5 * np.sum(res ** 2, axis=(1, 2))) <= 1e-9 * D_a)
    gam = np.zeros(wl.n_vox, bool)
    gam[wl.gamma_idx] = True
    assert not np.any(g_a[~gam]) and np.any(g_a[gam])
    # linear up to FP32 rounding of three 1500-step gradients: the gradient tolerance
    assert oc.rel(g_ab, g_a + g_b) < TOL_GRAD
    plan.close()
    inst = fwi.Plan.from_workload(wl, max_shots=K, per_shot_models=True)
    cs = _dev(np.stack([wl.c_model] * K)).reshape(-1)
    D_i, g_i = inst.gradient(cs, w, f - r_a)
    assert inst.status() == fwi.FWI_OK
    assert np.array_equal(D_i.cpu().numpy(), D_a)
    g_mean = g_i.cpu().numpy().reshape(K, -1).mean(axis=0)
    assert np.abs(g_mean - g_a).max() <= 1e-12 * np.abs(g_a).max()
    inst.close()
