"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: traces rel l2 <= 1e-4, gradient rel l2 <= 1e-3 (FP32 fields over
hundreds of steps against FP64), misfit rel <= 1e-3 (it is a difference of
nearly equal traces squared).
"""
import numpy as np
import pytest
import torch

from paper_2102_00755_b300 import build as fbuild
from paper_2102_00755_b300 import fwi, synth

from . import oracle_cases as oc

pytestmark = pytest.mark.gpu

TOL_TRACES = 1e-4
TOL_GRAD = 1e-3
TOL_MISFIT = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    fbuild.build()
    fwi.lib()
    assert torch.cuda.is_available()


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def run_forward(wl, c, weights, pml_on=True):
    plan = fwi.Plan.from_workload(wl, max_shots=len(weights), pml_on=pml_on)
    tr = plan.forward(dev(c), dev(weights))
    assert plan.status() == fwi.FWI_OK
    return tr.cpu().numpy()


def run_gradient(wl, f_obs, pairing, weights=None, pml_on=True, encoded=True, observed=None):
    W = wl.weights if weights is None else weights
    plan = fwi.Plan.from_workload(wl, pairing=pairing, max_shots=len(W), pml_on=pml_on)
    traces = torch.empty((len(W), wl.nt, len(wl.rec_idx)), dtype=torch.float32, device="cuda")
    obs = dev(f_obs if observed is None else observed)
    D, g = plan.gradient(dev(wl.c_model), dev(W), obs, encoded=encoded, traces=traces)
    assert plan.status() == fwi.FWI_OK
    return traces.cpu().numpy(), D.cpu().numpy(), g.cpu().numpy().reshape(wl.shape)


def test_forward_parity_small_ragged():
    wl, f_obs = oc.small_case()
    f_gpu = run_forward(wl, wl.c_true, wl.weights)
    for k in range(len(wl.weights)):
        assert oc.rel(f_gpu[k], f_obs[k]) < TOL_TRACES


@pytest.mark.parametrize("shape", [(15, 9, 10), (27, 25, 12), (16, 15, 9), (30, 18, 25)])
def test_forward_parity_odd_and_mixed_radix_shapes(shape):
    wl = synth.small_workload(*shape, 40, pml=3, n_src=2, n_rec=12, K=1, seed=3)
    ref = oc.forward(wl, wl.c_model, wl.weights)
    f_gpu = run_forward(wl, wl.c_model, wl.weights)
    assert oc.rel(f_gpu[0], ref[0]) < TOL_TRACES


@pytest.mark.parametrize("pairing", ["literal", "exact"])
def test_gradient_parity_small(pairing):
    wl, f_obs = oc.small_case()
    f_ref, D_ref, g_ref = oc.small_gradient(pairing)
    f_gpu, D_gpu, g_gpu = run_gradient(wl, f_obs, pairing)
    for k in range(len(wl.weights)):
        assert oc.rel(f_gpu[k], f_ref[k]) < TOL_TRACES
    assert np.all(np.abs(D_gpu - D_ref) <= TOL_MISFIT * np.abs(D_ref))
    assert oc.rel(g_gpu, g_ref) < TOL_GRAD
    gam = np.zeros(wl.n_vox, bool)
    gam[wl.gamma_idx] = True
    assert np.all(g_gpu.reshape(-1)[~gam] == 0.0)


def test_gradient_raw_observed_is_encoded_on_device():
    """observed_encoded = 0: per-source data encoded with the weights on the GPU."""
    wl, _ = oc.small_case()
    n_src = len(wl.src_idx)
    raw = oc.observed(wl, weights=np.eye(n_src))            # [n_src, nt, n_rec]
    enc = synth.f32(np.tensordot(wl.weights, raw, axes=1))
    _, D1, g1 = run_gradient(wl, enc, "literal")
    _, D2, g2 = run_gradient(wl, None, "literal", encoded=False, observed=raw)
    assert oc.rel(g2, g1) < 1e-5
    assert np.allclose(D2, D1, rtol=1e-5)


@pytest.mark.parametrize("pairing", ["literal", "exact"])
def test_config1_gradient_parity(pairing):
    """The 32^3 one-source configuration, 300 steps, PML inside, both pairings."""
    wl, f_obs = oc.config1_case()
    f_ref, D_ref, g_ref = oc.config1_gradient(pairing)
    f_gpu, D_gpu, g_gpu = run_gradient(wl, f_obs, pairing)
    assert oc.rel(f_gpu[0], f_ref[0]) < TOL_TRACES
    assert abs(D_gpu[0] - D_ref[0]) <= TOL_MISFIT * D_ref[0]
    assert oc.rel(g_gpu, g_ref) < TOL_GRAD


def test_config1_forward_parity_true_model():
    wl, f_obs = oc.config1_case()
    f_gpu = run_forward(wl, wl.c_true, wl.weights)
    assert oc.rel(f_gpu[0], f_obs[0]) < TOL_TRACES


def test_batched_shots_equal_single_shots():
    """Each super-shot's result is the same alone and batched with others."""
    wl, f_obs = oc.small_case()
    _, D_b, _ = run_gradient(wl, f_obs, "literal")
    f_b = run_forward(wl, wl.c_model, wl.weights)
    for k in range(len(wl.weights)):
        f_1 = run_forward(wl, wl.c_model, wl.weights[k:k + 1])
        assert np.array_equal(f_1[0], f_b[k])
        _, D_1, _ = run_gradient(wl, f_obs[k:k + 1], "literal", weights=wl.weights[k:k + 1])
        assert D_1[0] == D_b[k]


def test_unstable_sound_speed_is_reported():
    wl, _ = oc.small_case()
    plan = fwi.Plan.from_workload(wl)
    c = wl.c_model.copy()
    c.reshape(-1)[5] = 1900.0          # above c_ref = 1800
    plan.forward(dev(c), dev(wl.weights[:1]))
    assert plan.status() == fwi.FWI_EUNSTABLE
    plan.forward(dev(wl.c_model), dev(wl.weights[:1]))
    assert plan.status() == fwi.FWI_OK


def test_call_argument_errors():
    wl, _ = oc.small_case()
    plan = fwi.Plan.from_workload(wl, max_shots=1)
    with pytest.raises(fwi.FwiError) as e:
        plan.forward(dev(wl.c_model), dev(wl.weights))     # K = 2 > max_shots
    assert e.value.status == fwi.FWI_EINVAL


@pytest.mark.parametrize("shape", [(24, 20, 18), (32, 32, 32)])
def test_every_fft_schedule_meets_parity(shape):
    """Every schedule the autotuner may pick (specialised or runtime radix schedules in
    each order, both z tiles) gives oracle-parity traces."""
    from paper_2102_00755_b300 import autotune
    wl = synth.small_workload(*shape, 40, pml=4, n_src=2, n_rec=16, K=1, seed=4)
    ref = oc.forward(wl, wl.c_model, wl.weights)
    plan = fwi.Plan.from_workload(wl, max_shots=1)
    seen = 0
    for cand in autotune.CANDIDATES:
        if autotune.set_schedule(plan, cand) != fwi.FWI_OK:
            continue
        assert autotune.get_schedule(plan) == cand
        tr = plan.forward(dev(wl.c_model), dev(wl.weights)).cpu().numpy()
        assert oc.rel(tr[0], ref[0]) < TOL_TRACES, cand
        seen += 1
    assert seen >= 12


def test_autotuner_picks_and_caches(tmp_path, monkeypatch):
    from paper_2102_00755_b300 import autotune
    monkeypatch.setenv("FWI_SCHEDULE_CACHE", str(tmp_path / "s.json"))
    wl = synth.small_workload(32, 32, 32, 40, pml=4, n_src=2, n_rec=16, K=1, seed=4)
    res = autotune.tune(wl, K=1, steps=8, reps=1)
    assert res["schedule"] in [{k: c[k] for k in autotune.KNOBS} for c in autotune.CANDIDATES]
    plan = fwi.Plan.from_workload(wl, max_shots=1)
    assert autotune.apply_cached(plan, 32, 32, 32, 1)
    assert autotune.get_schedule(plan) == res["schedule"]


def test_plans_of_different_sizes_coexist():
    """A plan bound after a larger one must not restrict the larger plan's launches
    (kernel attributes are shared by every plan using the same kernel)."""
    big = synth.small_workload(48, 40, 30, 30, pml=5, n_src=2, n_rec=12, K=1, seed=22)
    small = synth.small_workload(32, 32, 24, 30, pml=4, n_src=2, n_rec=12, K=1, seed=21)
    p_big = fwi.Plan.from_workload(big, max_shots=1)
    ref = p_big.forward(dev(big.c_model), dev(big.weights)).clone()
    p_small = fwi.Plan.from_workload(small, max_shots=1)
    p_small.forward(dev(small.c_model), dev(small.weights))
    again = p_big.forward(dev(big.c_model), dev(big.weights))
    assert torch.equal(ref, again)


@pytest.mark.parametrize("pairing", ["literal", "exact"])
def test_split_plane_path_gradient_parity(pairing):
    """The split XY path (column and row-pair passes through global memory, used for
    planes that do not fit shared memory) forced on a small grid: gradient parity."""
    from paper_2102_00755_b300 import autotune
    wl, f_obs = oc.small_case()
    f_ref, D_ref, g_ref = oc.small_gradient(pairing)
    plan = fwi.Plan.from_workload(wl, pairing=pairing, max_shots=len(wl.weights))
    assert autotune.set_schedule(plan, dict(specialized=0, radix_order=0, z_tile=16, split_plane=1)) == 0
    traces = torch.empty((len(wl.weights), wl.nt, len(wl.rec_idx)), dtype=torch.float32, device="cuda")
    D, g = plan.gradient(dev(wl.c_model), dev(wl.weights), dev(f_obs), traces=traces)
    assert plan.status() == fwi.FWI_OK
    for k in range(len(wl.weights)):
        assert oc.rel(traces[k].cpu().numpy(), f_ref[k]) < TOL_TRACES
    assert np.all(np.abs(D.cpu().numpy() - D_ref) <= TOL_MISFIT * np.abs(D_ref))
    assert oc.rel(g.cpu().numpy().reshape(wl.shape), g_ref) < TOL_GRAD


@pytest.mark.parametrize("shape,pairing", [((32, 32, 20), "literal"), ((64, 64, 12), "exact"),
                                           ((96, 96, 10), "literal"), ((128, 128, 8), "exact"),
                                           ((135, 135, 8), "exact"),
                                           ((160, 160, 8), "literal")])
def test_two_step_plane_kernels_gradient_parity(shape, pairing):
    """The two-step register-transform plane kernels (schedule specialized = 2) on every
    plane size they are built for: forward traces, misfit and gradient (adjoint and
    time-reversal roles of the mass kernel) against the oracle."""
    from paper_2102_00755_b300 import autotune
    # 0.5 MHz over 90 steps: the pulse crosses Gamma, so the residual is a few percent of
    # the traces (a misfit of rounding-level residuals would only measure FP32 noise)
    wl = synth.small_workload(*shape, 90, pml=3, n_src=3, n_rec=20, K=2, layer=2, seed=11,
                              f0=0.5e6, gamma_frac=0.3)
    f_obs = oc.observed(wl)
    f_ref, D_ref, g_ref = oc.gradient(wl, f_obs, pairing, c_rec=wl.c_rec)
    plan = fwi.Plan.from_workload(wl, pairing=pairing, max_shots=len(wl.weights))
    sched = dict(specialized=2, radix_order=0, z_tile=32, split_plane=0)
    assert autotune.set_schedule(plan, sched) == fwi.FWI_OK
    traces = torch.empty((len(wl.weights), wl.nt, len(wl.rec_idx)), dtype=torch.float32, device="cuda")
    D, g = plan.gradient(dev(wl.c_model), dev(wl.weights), dev(f_obs), traces=traces)
    assert plan.status() == fwi.FWI_OK
    for k in range(len(wl.weights)):
        assert oc.rel(traces[k].cpu().numpy(), f_ref[k]) < TOL_TRACES
    assert np.all(np.abs(D.cpu().numpy() - D_ref) <= TOL_MISFIT * np.abs(D_ref))
    assert oc.rel(g.cpu().numpy().reshape(wl.shape), g_ref) < TOL_GRAD


@pytest.mark.parametrize("shape,pairing", [((243, 243, 8), "literal"), ((256, 256, 6), "exact"),
                                            ((480, 480, 6), "exact")])
def test_two_step_split_plane_gradient_parity(shape, pairing):
    """The two-step split-plane kernels (column passes and row-pair passes through global
    memory, schedule specialized = 2 with split planes) against the oracle gradient."""
    from paper_2102_00755_b300 import autotune
    wl = synth.small_workload(*shape, 90, pml=3, n_src=3, n_rec=20, K=2, layer=2, seed=12,
                              f0=0.5e6, gamma_frac=0.3)
    f_obs = oc.observed(wl)
    f_ref, D_ref, g_ref = oc.gradient(wl, f_obs, pairing, c_rec=wl.c_rec)
    plan = fwi.Plan.from_workload(wl, pairing=pairing, max_shots=len(wl.weights))
    assert autotune.set_schedule(plan, dict(specialized=2, radix_order=0, z_tile=16, split_plane=1)) == fwi.FWI_OK
    traces = torch.empty((len(wl.weights), wl.nt, len(wl.rec_idx)), dtype=torch.float32, device="cuda")
    D, g = plan.gradient(dev(wl.c_model), dev(wl.weights), dev(f_obs), traces=traces)
    assert plan.status() == fwi.FWI_OK
    for k in range(len(wl.weights)):
        assert oc.rel(traces[k].cpu().numpy(), f_ref[k]) < TOL_TRACES
    assert np.all(np.abs(D.cpu().numpy() - D_ref) <= TOL_MISFIT * np.abs(D_ref))
    assert oc.rel(g.cpu().numpy().reshape(wl.shape), g_ref) < TOL_GRAD


def test_two_stream_groups_are_bit_identical():
    """stream_groups = 2 or 4 (super-shots split over streams) changes only the launch
    grouping: traces, misfits and gradients equal those of one group bit for bit."""
    from paper_2102_00755_b300 import autotune
    wl, f_obs = oc.small_case()
    plan = fwi.Plan.from_workload(wl, pairing="literal", max_shots=len(wl.weights))
    c, w, o = dev(wl.c_model), dev(wl.weights), dev(f_obs)
    outs = []
    for g in (1, 2, 4):
        sched = dict(specialized=1, radix_order=0, z_tile=32, split_plane=0, stream_groups=g)
        assert autotune.set_schedule(plan, sched) == fwi.FWI_OK
        tr = plan.forward(c, w).clone()
        D, grad = plan.gradient(c, w, o)
        outs.append((tr, D.clone(), grad.clone()))
    assert plan.status() == fwi.FWI_OK
    for other in outs[1:]:
        for a, b in zip(outs[0], other):
            assert torch.equal(a, b)
