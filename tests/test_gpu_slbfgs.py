"""Stochastic L-BFGS (Alg. 2) on the device against the FP64 oracle of Alg. 2."""
import numpy as np
import pytest
import torch

from oracle import pstd
from oracle import slbfgs as oslbfgs
from paper_2102_00755_b300 import build as fbuild
from paper_2102_00755_b300 import fwi, synth
from paper_2102_00755_b300 import slbfgs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    fbuild.build()
    fwi.lib()


def _d(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def test_device_two_loop_matches_oracle():
    """History of 6 pairs (one pair without curvature skipped, older pairs dropped):
    H g equals the oracle's two-loop recursion (FP32 storage of the pairs)."""
    n, m = 5000, 6
    rng = np.random.default_rng(1)
    diag = rng.uniform(1.0, 30.0, n)
    hist = slbfgs.LBFGSHistory(n, m)
    S, Y = [], []
    for k in range(9):
        s = rng.standard_normal(n)
        y = -s if k == 4 else diag * s + 0.01 * rng.standard_normal(n)
        s32, y32 = s.astype(np.float32).astype(np.float64), y.astype(np.float32).astype(np.float64)
        stored = hist.push(_d(s), _d(y))
        assert stored == oslbfgs.push_pair(S, Y, s, y, m)
        S[-1:], Y[-1:] = ([s32], [y32]) if stored else (S[-1:], Y[-1:])
    assert len(hist) == len(S) == m
    g = rng.standard_normal(n)
    out = hist.apply(_d(g), 0.0).cpu().numpy()
    ref = oslbfgs.two_loop(g, S, Y, oslbfgs.scaling(S, Y, None))
    assert np.linalg.norm(out - ref) <= 1e-5 * np.linalg.norm(ref)
    out2 = hist.apply(_d(g), 0.25).cpu().numpy()
    ref2 = oslbfgs.two_loop(g, S, Y, 0.25)
    assert np.linalg.norm(out2 - ref2) <= 1e-5 * np.linalg.norm(ref2)


def test_elementwise_steps_and_parameterisations():
    rng = np.random.default_rng(2)
    n = 1000
    u, z = rng.uniform(-1, 1, n), rng.standard_normal(n)
    ut = _d(u)
    slbfgs.step_project(ut, _d(z), 0.3, -0.5, 0.6)
    # the device forms u + nu z with one fused multiply-add: equal up to that rounding
    assert np.allclose(ut.cpu().numpy(), np.clip(u + 0.3 * z, -0.5, 0.6), rtol=1e-15, atol=1e-16)
    acc = _d(u)
    slbfgs.accumulate(acc, _d(z), 2.5)
    assert np.allclose(acc.cpu().numpy(), u + 2.5 * z, rtol=1e-15, atol=1e-15)   # one fused multiply-add
    c = rng.uniform(1400.0, 1700.0, n)
    gc = rng.standard_normal(n)
    for kind, (uc, dcdu) in enumerate([(c, np.ones(n)), (1.0 / c, -c ** 2), (1.0 / c ** 2, -0.5 * c ** 3)]):
        cs = torch.empty(n, dtype=torch.float32, device="cuda")
        assert fwi.fwi_param_to_speed(n, kind, slbfgs._vp(_d(uc), torch.float64), slbfgs._vp(cs, torch.float32),
                                      fwi._stream_handle(None)) == fwi.FWI_OK
        c32 = cs.cpu().numpy()
        assert np.allclose(c32, c, rtol=2e-7)
        gu = torch.empty(n, dtype=torch.float64, device="cuda")
        assert fwi.fwi_grad_to_param(n, kind, slbfgs._vp(cs, torch.float32), slbfgs._vp(_d(gc), torch.float64),
                                     slbfgs._vp(gu, torch.float64), fwi._stream_handle(None)) == fwi.FWI_OK
        ref = gc * (np.ones(n) if kind == 0 else (-(c32.astype(np.float64)) ** 2 if kind == 1
                                                   else -0.5 * c32.astype(np.float64) ** 3))
        assert np.allclose(gu.cpu().numpy(), ref, rtol=1e-12)
        assert np.allclose(ref, gc * dcdu, rtol=1e-5)


def test_slbfgs_stochastic_quadratic_matches_oracle():
    """Same estimator (noise fixed by n) on both sides; bounds active for a few entries."""
    n = 40
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = Q @ np.diag(np.linspace(1.0, 10.0, n)) @ Q.T
    b = rng.standard_normal(n)

    def noise(k):
        return 0.05 * np.random.default_rng(100 + k).standard_normal(n)

    def est_np(u, th, k):
        e = noise(k)
        return 0.5 * u @ A @ u - b @ u + e @ u, A @ u - b + e

    At, bt = _d(A), _d(b)

    def est_gpu(u, th, k):
        e = _d(noise(k))
        G = At @ u - bt + e
        return float((0.5 * u @ (At @ u) - bt @ u + e @ u).item()), G.contiguous()

    u0 = rng.standard_normal(n)
    ref, Js_ref, _ = oslbfgs.slbfgs(u0, est_np, nu=0.8, n_evl=30, m=5, u_min=-1.5, u_max=1.5)
    opt = slbfgs.SLBFGS(est_gpu, nu=0.8, m=5, u_min=-1.5, u_max=1.5)
    got, Js = opt.run(_d(u0), 30)
    assert np.allclose(Js, Js_ref, rtol=1e-5)
    assert np.linalg.norm(got.cpu().numpy() - ref) <= 1e-5 * np.linalg.norm(ref)


def test_slbfgs_fwi_squared_slowness_matches_oracle():
    """Two iterations of Alg. 2 on a small FWI problem in the squared slowness u = 1/c^2
    (Sec. 3.3): device estimator (fwi_gradient) vs the oracle's gradient, same seeded
    encodings; energies and the model update agree."""
    wl = synth.small_workload(16, 15, 12, 60, pml=3, n_src=3, n_rec=16, K=1, layer=2, seed=5)
    G = pstd.grid_for(wl)
    n_src = len(wl.src_idx)
    raw = synth.f32(np.stack([pstd.forward(G, wl.c_true, wl.src_idx, np.eye(n_src)[i], wl.wavelet,
                                           wl.rec_idx)[0] for i in range(n_src)]))
    plan = fwi.Plan.from_workload(wl, pairing="exact", max_shots=1)
    est_gpu = slbfgs.FwiEstimator(plan, torch.as_tensor(raw, dtype=torch.float32, device="cuda"), K=1,
                                  param="squared_slowness",
                                  seed0=40)

    def est_np(u, th, k):
        c = 1.0 / np.sqrt(u.reshape(wl.shape))
        w, _ = synth.encoding_draws(40 + k, 1, n_src)
        f_obs = pstd.encode_data(w[0], raw)
        _, D, gc = pstd.fwi_gradient(G, c, wl.src_idx, w[0], wl.wavelet, wl.rec_idx, wl.layer_idx, wl.gamma_idx,
                                     f_obs, pairing="exact", c_rec=wl.c_rec)
        return D, (gc * (-0.5 * c ** 3)).reshape(-1)

    u0 = 1.0 / wl.c_model.astype(np.float64).reshape(-1) ** 2
    F0, G0 = est_np(u0, 0.0, 1)
    h0 = 0.01 * np.linalg.norm(u0) / np.linalg.norm(G0)     # first step changes c by about 1 %
    bounds = dict(u_min=1.0 / 1800.0 ** 2, u_max=1.0 / 1350.0 ** 2)
    ref, Js_ref, _ = oslbfgs.slbfgs(u0, est_np, nu=1.0, n_evl=4, m=8, h0=h0, **bounds)
    got, Js = slbfgs.SLBFGS(est_gpu, nu=1.0, m=8, h0=h0, **bounds).run(_d(u0), 4)
    assert np.allclose(Js, Js_ref, rtol=2e-3)
    du_ref = ref - u0
    du = got.cpu().numpy() - u0
    assert np.linalg.norm(du_ref) > 0
    assert np.linalg.norm(du - du_ref) <= 5e-3 * np.linalg.norm(du_ref)
