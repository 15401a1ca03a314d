"""Delayed source encoding (Sec. 3.2, Eq. 13) through the C ABI against the oracle."""
import numpy as np
import pytest
import torch

from oracle import pstd
from paper_2102_00755_b300 import build as fbuild
from paper_2102_00755_b300 import fwi, synth

from . import oracle_cases as oc

pytestmark = pytest.mark.gpu

TOL_TRACES = 1e-4
TOL_GRAD = 1e-3
TOL_MISFIT = 1e-3
NT_DATA, TAU = 80, 24          # recorded samples T, largest delay tau (time steps)


@pytest.fixture(scope="module", autouse=True)
def _built():
    fbuild.build()
    fwi.lib()


def _dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _case():
    """24x20x18 ragged grid; plan window T + tau, the wavelet zero-padded to it; per-super-shot
    delays d_i tau with d_i ~ U[0, 1] drawn from a seeded generator, rounded to whole steps."""
    wl = synth.small_workload(24, 20, 18, NT_DATA, pml=4, K=2, layer=2, seed=7)
    nt = NT_DATA + TAU
    wav = np.zeros(nt, dtype=np.float32)
    wav[:NT_DATA] = wl.wavelet
    rng = np.random.default_rng(31)
    delays = np.rint(rng.uniform(0.0, 1.0, size=wl.weights.shape) * TAU).astype(np.int32)
    return wl, nt, wav, delays


def _plan(wl, nt, wav, pairing="literal"):
    return fwi.Plan(nx=wl.nx, ny=wl.ny, nz=wl.nz, pml=wl.pml, dx=wl.dx, dt=wl.dt, c_ref=wl.c_ref, rho0=wl.rho0,
                    pml_alpha=wl.pml_alpha, nt=nt, src_idx=wl.src_idx, rec_idx=wl.rec_idx,
                    layer_idx=wl.layer_idx, gamma_idx=wl.gamma_idx, wavelet=wav, pairing=pairing,
                    max_shots=len(wl.weights), c_rec=wl.c_rec)


def test_zero_delays_equal_plain_calls():
    wl, nt, wav, _ = _case()
    plan = _plan(wl, nt, wav)
    c, w = _dev(wl.c_model).reshape(-1), _dev(wl.weights)
    zero = torch.zeros(wl.weights.shape, dtype=torch.int32, device="cuda")
    a = plan.forward(c, w).clone()
    b = plan.forward(c, w, delays=zero)
    assert torch.equal(a, b)
    obs = plan.forward(_dev(wl.c_true).reshape(-1), w).clone()
    D1, g1 = plan.gradient(c, w, obs)
    D1, g1 = D1.clone(), g1.clone()
    D2, g2 = plan.gradient(c, w, obs, delays=zero)
    assert torch.equal(D1, D2) and torch.equal(g1, g2)


def test_delayed_forward_matches_oracle():
    wl, nt, wav, delays = _case()
    plan = _plan(wl, nt, wav)
    tr = plan.forward(_dev(wl.c_model).reshape(-1), _dev(wl.weights), delays=_dev(delays, torch.int32))
    assert plan.status() == fwi.FWI_OK
    tr = tr.cpu().numpy()
    G = pstd.grid_for(wl)
    for k in range(len(wl.weights)):
        ref, _ = pstd.forward(G, wl.c_model, wl.src_idx, wl.weights[k], wav.astype(np.float64), wl.rec_idx,
                              delays=delays[k])
        assert oc.rel(tr[k], ref) < TOL_TRACES


@pytest.mark.parametrize("pairing", ["literal", "exact"])
def test_delayed_gradient_with_device_encoding_matches_oracle(pairing):
    """Raw per-source data (T samples) are delay-encoded on the device into the T + tau window."""
    wl, nt, wav, delays = _case()
    G = pstd.grid_for(wl)
    n_src = len(wl.src_idx)
    raw = np.stack([pstd.forward(G, wl.c_true, wl.src_idx, np.eye(n_src)[i], wl.wavelet, wl.rec_idx)[0]
                    for i in range(n_src)])
    raw = synth.f32(raw)                                   # [n_src][T][n_rec], both sides see these
    plan = _plan(wl, nt, wav, pairing)
    traces = torch.empty((len(wl.weights), nt, len(wl.rec_idx)), dtype=torch.float32, device="cuda")
    D, g = plan.gradient(_dev(wl.c_model).reshape(-1), _dev(wl.weights), _dev(raw), encoded=False,
                         traces=traces, delays=_dev(delays, torch.int32))
    assert plan.status() == fwi.FWI_OK
    D, g = D.cpu().numpy(), g.cpu().numpy().reshape(wl.shape)
    Ds, gs = [], []
    for k in range(len(wl.weights)):
        f_obs = pstd.encode_data(wl.weights[k], raw, delays=delays[k], nt=nt)
        f, Dk, gk = pstd.fwi_gradient(G, wl.c_model, wl.src_idx, wl.weights[k], wav.astype(np.float64),
                                      wl.rec_idx, wl.layer_idx, wl.gamma_idx, f_obs, pairing=pairing,
                                      c_rec=wl.c_rec, delays=delays[k])
        assert oc.rel(traces[k].cpu().numpy(), f) < TOL_TRACES
        Ds.append(Dk)
        gs.append(gk)
    assert np.all(np.abs(D - np.array(Ds)) <= TOL_MISFIT * np.abs(np.array(Ds)))
    assert oc.rel(g, np.mean(gs, axis=0)) < TOL_GRAD
