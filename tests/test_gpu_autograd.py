"""The time-reversal adjoint as torch.autograd.Function, checked against the FP64
oracle's gradient and against central finite differences of the misfit."""
import os

import numpy as np
import pytest
import torch

from oracle import pstd
from paper_2102_00755_b300 import build as fbuild
from paper_2102_00755_b300 import fwi, synth
from paper_2102_00755_b300.autograd import FwiLoss, fwi_misfit

from . import oracle_cases as oc

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "config4_fd.npz")


def _dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def test_autograd_small_without_pml_matches_finite_differences():
    """No PML, layer = Gamma, exact pairing: the autograd gradient is the derivative of
    the discrete misfit; compare with the oracle's gradient and FP64 central differences."""
    fbuild.build()
    wl = synth.small_workload(16, 15, 12, 70, pml=0, layer=6, n_src=2, n_rec=20, K=1, f0=0.3e6, seed=9)
    assert len(wl.layer_idx) == len(wl.gamma_idx)
    G = pstd.grid_for(wl, pml_on=False)
    f_obs = synth.f32(pstd.forward(G, wl.c_true, wl.src_idx, wl.weights[0], wl.wavelet, wl.rec_idx)[0])
    _, D_ref, g_ref = pstd.fwi_gradient(G, wl.c_model, wl.src_idx, wl.weights[0], wl.wavelet, wl.rec_idx,
                                        wl.layer_idx, wl.gamma_idx, f_obs, pairing="exact", c_rec=wl.c_rec)
    plan = fwi.Plan.from_workload(wl, pairing="exact", max_shots=1, pml_on=False)
    c = _dev(wl.c_model).requires_grad_(True)
    loss = fwi_misfit(c, plan, _dev(wl.weights), _dev(f_obs[None]))
    loss.backward()
    g = c.grad.cpu().numpy().astype(np.float64)
    assert abs(loss.item() - D_ref) <= 1e-3 * D_ref
    assert oc.rel(g, g_ref) < 1e-3

    def D(cm):
        f, _ = pstd.forward(G, cm, wl.src_idx, wl.weights[0], wl.wavelet, wl.rec_idx)
        return pstd.adjoint_source(f, f_obs)[0]

    h = 1e-2
    for seed in (1, 2, 3):
        d = synth.smooth_direction(wl, seed)
        fd = (D(wl.c_model + h * d) - D(wl.c_model - h * d)) / (2 * h)
        assert abs(float(np.sum(g * d)) - fd) <= 2e-3 * abs(fd), seed


def test_autograd_module_and_grad_accumulation():
    fbuild.build()
    wl, f_obs = oc.small_case()
    plan = fwi.Plan.from_workload(wl, pairing="exact", max_shots=len(wl.weights))
    loss_fn = FwiLoss(plan, _dev(wl.weights), _dev(f_obs))
    c = _dev(wl.c_model).requires_grad_(True)
    (2.0 * loss_fn(c)).backward()
    g2 = c.grad.clone()
    c.grad = None
    loss_fn(c).backward()
    assert torch.allclose(g2, 2.0 * c.grad)
    assert c.grad.dtype == torch.float32 and c.grad.shape == c.shape


@pytest.mark.skipif(not os.path.exists(GOLDEN), reason="oracle reference not generated")
def test_autograd_config4_against_oracle_and_finite_differences():
    """96x96x48 phantom, 32 emitters, 128 receivers, 1000 steps, exact pairing, PML on:
    gradient vs the oracle's (rel l2 <= 1e-3) and directional derivatives vs FP64
    central differences along 8 seeded smooth directions (h = 1e-3 m/s)."""
    fbuild.build()
    ref = np.load(GOLDEN)
    wl = synth.config4()
    plan = fwi.Plan.from_workload(wl, pairing="exact", max_shots=1)
    c = _dev(wl.c_model).requires_grad_(True)
    loss = fwi_misfit(c, plan, _dev(wl.weights), _dev(ref["observed"]))
    loss.backward()
    g = c.grad.cpu().numpy().astype(np.float64).reshape(-1)
    assert abs(loss.item() - float(ref["D0"])) <= 1e-3 * float(ref["D0"])
    g_gam = g[wl.gamma_idx]
    assert oc.rel(g_gam, ref["grad_gamma"]) < 1e-3
    gam = np.zeros(wl.n_vox, bool)
    gam[wl.gamma_idx] = True
    assert np.all(g[~gam] == 0.0)
    for k, seed in enumerate(ref["seeds"]):
        d = synth.smooth_direction(wl, int(seed)).reshape(-1)
        ad = float(np.dot(g, d))
        fd = float(ref["fd"][k])
        # the oracle's own adjoint agrees with FD to the PML's effect; allow that plus FP32
        tol = abs(float(ref["oracle_dir"][k]) - fd) + 2e-3 * abs(fd)
        assert abs(ad - fd) <= tol, (seed, ad, fd)
