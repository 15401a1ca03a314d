"""Batched form: uneven-grid instances captured into one CUDA graph give exactly the
results of separate calls (and of the oracle, within the parity tolerances)."""
import numpy as np
import pytest
import torch

from paper_2102_00755_b300 import build as fbuild
from paper_2102_00755_b300 import fwi, synth

from . import oracle_cases as oc

pytestmark = pytest.mark.gpu


def _dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _instances(nt):
    """The uneven-grid batch configuration (64^3, 96x96x48, 128x128x64, 160x160x80),
    one instance per size, with a shortened time axis."""
    out = []
    for i in (0, 4, 8, 12):
        wl = synth.config3_instance(i)
        wl.nt = nt
        wl.wavelet = wl.wavelet[:nt]
        out.append(wl)
    return out


def _prepare(wls):
    plans, cs, ws, obs = [], [], [], []
    for wl in wls:
        plan = fwi.Plan.from_workload(wl, max_shots=1)
        w = _dev(wl.weights)
        obs.append(plan.forward(_dev(wl.c_true).reshape(-1), w))
        plans.append(plan)
        cs.append(_dev(wl.c_model).reshape(-1))
        ws.append(w)
    return plans, cs, ws, obs


def test_batch_graph_equals_separate_calls():
    fbuild.build()
    wls = _instances(48)
    plans, cs, ws, obs = _prepare(wls)
    alone = [p.gradient(c, w, o) for p, c, w, o in zip(plans, cs, ws, obs)]
    alone = [(D.cpu().numpy(), g.cpu().numpy()) for D, g in alone]
    batch = fwi.Batch(plans)
    Ds = [torch.empty(1, dtype=torch.float64, device="cuda") for _ in plans]
    gs = [torch.empty(p.n_vox, dtype=torch.float64, device="cuda") for p in plans]
    for rep in range(2):                       # capture, then replay the same graph
        for g in gs:
            g.fill_(np.nan)
        batch.gradient(cs, ws, obs, misfits=Ds, grads=gs)
        torch.cuda.synchronize()
        assert batch.nodes() > 0
        for k, p in enumerate(plans):
            assert p.status() == fwi.FWI_OK
            assert np.array_equal(Ds[k].cpu().numpy(), alone[k][0]), (rep, k)
            assert np.array_equal(gs[k].cpu().numpy(), alone[k][1]), (rep, k)


def test_batch_instance_matches_oracle():
    """One small ragged instance inside a batch with a larger one still meets parity."""
    fbuild.build()
    wl_small, f_obs = oc.small_case()
    f_ref, D_ref, g_ref = oc.small_gradient("literal")
    big = _instances(32)[1]
    plans, cs, ws, obs = _prepare([big])
    p_small = fwi.Plan.from_workload(wl_small, max_shots=len(wl_small.weights))
    plans.append(p_small)
    cs.append(_dev(wl_small.c_model).reshape(-1))
    ws.append(_dev(wl_small.weights))
    obs.append(_dev(f_obs))
    Ds, gs = fwi.Batch(plans).gradient(cs, ws, obs)
    torch.cuda.synchronize()
    assert np.all(np.abs(Ds[1].cpu().numpy() - D_ref) <= 1e-3 * np.abs(D_ref))
    g = gs[1].cpu().numpy().reshape(wl_small.shape)
    assert oc.rel(g, g_ref) < 1e-3


def test_batch_recaptures_after_rebinding_and_schedule_change():
    """A member plan bound to a new workspace, or given a new schedule, between two batch
    calls: the batch must not replay a graph holding the old workspace or launch shapes.
    The old workspace (still allocated) is zeroed after the rebinding: a stale replay would
    read empty tables and give other results (zeros keep every table index in bounds)."""
    from paper_2102_00755_b300 import autotune
    fbuild.build()
    wls = _instances(32)[:2]
    plans, cs, ws, obs = _prepare(wls)
    alone = [p.gradient(c, w, o) for p, c, w, o in zip(plans, cs, ws, obs)]
    alone = [(D.clone(), g.clone()) for D, g in alone]
    batch = fwi.Batch(plans)
    Ds, gs = batch.gradient(cs, ws, obs)
    torch.cuda.synchronize()
    # rebind plan 0 to a fresh workspace; clear the old one (still allocated)
    p0 = plans[0]
    old = p0.workspace
    new = torch.empty_like(old)
    base = new.data_ptr()
    aligned = (base + 255) & ~255
    assert fwi.fwi_plan_bind_workspace(p0.handle, aligned, p0.workspace_bytes) == fwi.FWI_OK
    p0.workspace = new
    old.zero_()
    Ds, gs = batch.gradient(cs, ws, obs)
    torch.cuda.synchronize()
    for (D0, g0), D1, g1 in zip(alone, Ds, gs):
        assert torch.equal(D0, D1) and torch.equal(g0, g1)
    # a schedule change of plan 1 (z tile 16): the batch follows it like a separate call
    sched = dict(autotune.get_schedule(plans[1]), z_tile=16)
    assert autotune.set_schedule(plans[1], sched) == fwi.FWI_OK
    D1a, g1a = plans[1].gradient(cs[1], ws[1], obs[1])
    D1a, g1a = D1a.clone(), g1a.clone()
    Ds, gs = batch.gradient(cs, ws, obs)
    torch.cuda.synchronize()
    assert torch.equal(Ds[1], D1a) and torch.equal(gs[1], g1a)
    assert all(p.status() == fwi.FWI_OK for p in plans)
    del old


def test_batch_refuses_a_plan_listed_twice():
    """Two chains of one batch would run a plan listed twice over one workspace at once."""
    fbuild.build()
    plan = fwi.Plan.from_workload(_instances(8)[0], max_shots=1)
    st, handle = fwi.fwi_batch_create([plan.handle, plan.handle])
    assert st == fwi.FWI_EINVAL and not handle
    with pytest.raises(RuntimeError):
        fwi.Batch([plan, plan])
