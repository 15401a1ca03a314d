"""Plans whose super-shots are independent instances (per_shot_models = 1): each shot has
its own sound-speed model, observed data and gradient, and all of them share every launch
of the grid they have in common.  Each instance's result must equal the same problem run
alone (bit for bit: the same kernels on the same values) and the FP64 oracle's.
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


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _instances(shape=(24, 20, 18), nt=80, seed=7):
    """Two instances on one grid: the workload's model and a perturbed one, each with its
    own encoding weights and observed data from its own true model."""
    wl = synth.small_workload(*shape, nt, pml=4, K=2, layer=2, seed=seed)
    rng = np.random.default_rng(seed + 1)
    gam = np.zeros(wl.n_vox)
    gam[wl.gamma_idx] = 1.0
    c1 = synth.f32(wl.c_model + rng.uniform(-15.0, 15.0, size=wl.shape) * gam.reshape(wl.shape))
    t1 = synth.f32(wl.c_true + 10.0 * gam.reshape(wl.shape))
    models = [wl.c_model, c1]
    trues = [wl.c_true, t1]
    obs = [oc.observed(wl, weights=wl.weights[k:k + 1])[0] if k == 0 else None for k in range(2)]
    wl1 = synth.Workload(**{**wl.__dict__, "c_true": t1, "c_model": c1})
    obs[1] = oc.observed(wl1, weights=wl.weights[1:2])[0]
    return wl, models, trues, np.stack(obs)


def _alone(wl, c, w, f_obs, pairing, tr_box=None):
    plan = fwi.Plan.from_workload(wl, pairing=pairing, max_shots=1, tr_box=tr_box)
    tr = torch.empty((1, wl.nt, len(wl.rec_idx)), dtype=torch.float32, device="cuda")
    D, g = plan.gradient(_dev(c).reshape(-1), _dev(w[None]), _dev(f_obs[None]), traces=tr)
    assert plan.status() == fwi.FWI_OK
    return tr.cpu().numpy()[0], D.cpu().numpy()[0], g.cpu().numpy()


@pytest.mark.parametrize("pairing,box", [("literal", False), ("exact", False), ("literal", True)])
def test_instances_equal_their_runs_alone(pairing, box):
    wl, models, _, f_obs = _instances()
    tr_box = synth.tr_box(wl, 1, 2) if box else None
    plan = fwi.Plan.from_workload(wl, pairing=pairing, max_shots=2, per_shot_models=True, tr_box=tr_box)
    tr = torch.empty((2, wl.nt, len(wl.rec_idx)), dtype=torch.float32, device="cuda")
    c = _dev(np.stack(models)).reshape(-1)
    D, g = plan.gradient(c, _dev(wl.weights), _dev(f_obs), traces=tr)
    assert plan.status() == fwi.FWI_OK
    assert g.numel() == 2 * wl.n_vox
    g = g.cpu().numpy().reshape(2, -1)
    for k in range(2):
        tr1, D1, g1 = _alone(wl, models[k], wl.weights[k], f_obs[k], pairing, tr_box)
        assert np.array_equal(tr.cpu().numpy()[k], tr1)
        assert D.cpu().numpy()[k] == D1
        assert np.array_equal(g[k], g1)
    # forward with per-shot models too
    f = plan.forward(c, _dev(wl.weights)).cpu().numpy()
    assert np.array_equal(f, tr.cpu().numpy())


def test_instance_with_its_own_model_matches_the_oracle():
    wl, models, _, f_obs = _instances()
    plan = fwi.Plan.from_workload(wl, pairing="literal", max_shots=2, per_shot_models=True)
    tr = torch.empty((2, wl.nt, len(wl.rec_idx)), dtype=torch.float32, device="cuda")
    D, g = plan.gradient(_dev(np.stack(models)).reshape(-1), _dev(wl.weights), _dev(f_obs), traces=tr)
    assert plan.status() == fwi.FWI_OK
    g = g.cpu().numpy().reshape(2, *wl.shape)
    for k in range(2):
        wlk = synth.Workload(**{**wl.__dict__, "c_model": models[k]})
        f_ref, D_ref, g_ref = oc.gradient(wlk, f_obs[k:k + 1], "literal", c_rec=wl.c_rec,
                                          weights=wl.weights[k:k + 1])
        assert oc.rel(tr.cpu().numpy()[k], f_ref[0]) < TOL_TRACES
        assert abs(D.cpu().numpy()[k] - D_ref[0]) <= TOL_MISFIT * D_ref[0]
        assert oc.rel(g[k], g_ref) < TOL_GRAD


def test_batch_of_instance_plans_equals_separate_calls():
    """Two grids, two instances each, in one captured graph: every instance's misfit and
    gradient equal the per-plan calls bit for bit, on a replay and with the plans side by side
    or in one chain."""
    cases = [_instances((24, 20, 18), 60, 7), _instances((20, 20, 16), 60, 9)]
    plans, cs, ws, obs = [], [], [], []
    for wl, models, _, f_obs in cases:
        plans.append(fwi.Plan.from_workload(wl, max_shots=2, per_shot_models=True))
        cs.append(_dev(np.stack(models)).reshape(-1))
        ws.append(_dev(wl.weights))
        obs.append(_dev(f_obs))
    ref = [p.gradient(c, w, o) for p, c, w, o in zip(plans, cs, ws, obs)]
    ref = [(D.clone(), g.clone()) for D, g in ref]
    batch = fwi.Batch(plans)
    for chain in (None, None, [0, 0], [1, 0]):   # capture, replay, one chain, chains in reverse
        batch.set_chains(chain)
        Ds, gs = batch.gradient(cs, ws, obs)
        torch.cuda.synchronize()
        for (D0, g0), D1, g1 in zip(ref, Ds, gs):
            assert torch.equal(D0, D1) and torch.equal(g0, g1)
    assert all(p.status() == fwi.FWI_OK for p in plans)
