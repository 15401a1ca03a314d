"""Grid transfers of the coarse-to-fine scheme (App. C) through the C ABI against the oracle."""
import numpy as np
import pytest
import torch

from oracle import multigrid as omg
from paper_2102_00755_b300 import build as fbuild
from paper_2102_00755_b300 import fwi, multigrid, synth

from . import oracle_cases as oc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    fbuild.build()
    fwi.lib()


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


@pytest.mark.parametrize("shape_in,shape_out", [((9, 12, 11), (17, 24, 21)), ((20, 16, 12), (39, 32, 23)),
                                                ((16, 15, 14), (8, 15, 7))])
def test_blackman_resampling_matches_oracle(shape_in, shape_out):
    u = np.random.default_rng(sum(shape_in)).standard_normal(shape_in)
    u32 = synth.f32(u)
    got = multigrid.Resampler(shape_in, shape_out, ("blackman",) * 3)(_dev(u32)).cpu().numpy()
    ref = omg.resample(u32, shape_out, "blackman")
    assert oc.rel(got, ref) < 1e-6


def test_plain_fourier_interpolation_is_exact():
    shape_c, shape_f = (9, 12, 11), (17, 24, 21)

    def f(shape, scale):
        z, y, x = np.meshgrid(*[np.arange(n) * scale[a] for a, n in enumerate(shape)], indexing="ij")
        return (1500.0 + 20.0 * np.cos(2 * np.pi * 2 * x / shape[2] / scale[2]) * np.sin(2 * np.pi * y / shape[1] / scale[1])
                + 10.0 * np.cos(2 * np.pi * 3 * z / shape[0] / scale[0] + 0.3))
    uc = f(shape_c, (1.0, 1.0, 1.0))
    uf = f(shape_f, tuple(c / n for c, n in zip(shape_c, shape_f)))
    got = multigrid.Resampler(shape_c, shape_f)(_dev(uc)).cpu().numpy()
    assert np.abs(got - uf).max() < 2e-3          # FP32 storage of values near 1500


def test_data_downsampling_matches_oracle():
    """Traces [n_src][nt][n_rec] to half the samples with the Kaiser low-pass and eta^2."""
    rng = np.random.default_rng(4)
    data = synth.f32(rng.standard_normal((3, 100, 7)))
    got = multigrid.downsample_data(_dev(data), 50, eta=2.0).cpu().numpy()
    ref = omg.downsample_series(data, 50, 1, eta=2.0)
    assert oc.rel(got, ref) < 1e-6


def test_serving_level_model_transfer_matches_oracle():
    """The coarse-to-fine transfer between the first two serving levels: physical part of
    the 135x135x96 model -> Blackman up-sampling to the 221x221x111 physical grid -> embedded
    in the 243x243x135 grid with water in the PML."""
    lo = synth.serving_level(0, n_src=8, seed=3)
    hi = synth.serving_level(1, n_src=8, seed=4)
    c_lo = _dev(lo.c_true)
    phys = multigrid.physical(c_lo, lo.pml)
    shape_hi_phys = (hi.nz - 2 * hi.pml[2], hi.ny - 2 * hi.pml[1], hi.nx - 2 * hi.pml[0])
    up = multigrid.upsample_model(phys, shape_hi_phys)
    ref = omg.upsample_model(phys.cpu().numpy(), shape_hi_phys)
    assert oc.rel(up.cpu().numpy(), ref) < 1e-6
    full = multigrid.embed_physical(up, hi.shape, hi.pml, synth.C_WATER)
    assert full.shape == hi.shape
    assert float(full[0, 0, 0]) == synth.C_WATER
    assert 1400.0 < float(full.min()) and float(full.max()) < 1700.0


def _two_grids(nt_f=240, P=4):
    """One physical experiment on dx = 0.5 mm (fine) and 1 mm (coarse): a 16 x 16 x 12 mm box
    (PML of P cells outside it on each grid), Gamma = ball of 4.5 mm around (8, 8, 6) mm with
    a 3 mm, 1600 m/s inclusion in water, transducers on a bowl of radius 6 mm rounded to the
    1 mm lattice (exact on both grids), a 0.15 MHz pulse on the fine time grid and its
    Kaiser down-sampling (App. C: sources are down-sampled like the data, without eta^2)."""
    phys_mm = (12, 16, 16)
    pts = np.unique(np.rint(synth.bowl_points(36, (8.0, 8.0, 9.0), 6.0)), axis=0)
    dt_f = synth.time_step(0.5e-3)
    wav_f = synth.ricker(nt_f, dt_f, 0.15e6)
    wav_c = multigrid.Resampler((1, nt_f, 1), (1, nt_f // 2, 1), ("none", "kaiser", "none"))(
        _dev(wav_f.reshape(1, -1, 1))).cpu().numpy().reshape(-1)
    out = []
    for dx_mm, nt, wav in ((0.5, nt_f, wav_f), (1.0, nt_f // 2, wav_c)):
        n = tuple(int(round(e / dx_mm)) + 2 * P for e in phys_mm)
        z, y, x = np.meshgrid(*[(np.arange(m) - P) * dx_mm for m in n], indexing="ij")
        r = np.sqrt((x - 8.0) ** 2 + (y - 8.0) ** 2 + (z - 6.0) ** 2)
        gamma = r <= 4.5
        c_true = np.where(r <= 3.0, 1600.0, 1500.0).astype(np.float32)
        water = np.full(n, synth.C_WATER, dtype=np.float32)
        vox = np.ravel_multi_index(tuple(np.rint(pts[:, a] / dx_mm).astype(int) + P for a in (2, 1, 0)), n)
        vox = vox.astype(np.int32)
        out.append(synth.Workload(f"two-grid-{dx_mm}mm", n[2], n[1], n[0], (P, P, P), dx_mm * 1e-3,
                                  synth.time_step(dx_mm * 1e-3), nt, c_true, water, vox[:4], vox[4:],
                                  synth.linear_indices(gamma), synth.linear_indices(synth.boundary_layer(gamma, 2)),
                                  np.asarray(wav, np.float32), np.ones((1, 4))))
    return out


def test_coarse_to_fine_lowers_the_fine_misfit():
    """Data recorded on the fine grid from the true model and down-sampled in time (Kaiser,
    eta^2) drive SLBFGS on the coarse grid (twice the spacing, squared slowness, 4 encoded
    super-shots per estimate); the result, transferred by Blackman up-sampling, lowers the
    fine-grid misfit summed over the emitters (the expectation of the encoded estimator's
    energy, App. E) well below that of the water start."""
    fine, coarse = _two_grids()
    n_src = len(fine.src_idx)
    eye = torch.eye(n_src, device="cuda")
    plan_f = fwi.Plan.from_workload(fine, pairing="exact", max_shots=n_src)
    raw_f = plan_f.forward(_dev(fine.c_true).reshape(-1), eye).clone()
    raw_c = multigrid.downsample_data(raw_f, coarse.nt, eta=2.0)
    plan_c = fwi.Plan.from_workload(coarse, pairing="exact", max_shots=n_src)

    def total(plan, c, raw):        # sum over emitters of D_i: every emitter alone
        return float(plan.gradient(c.reshape(-1).contiguous(), eye, raw, encoded=False)[0].sum())

    water_c = torch.full(coarse.shape, synth.C_WATER, device="cuda")
    c_c, _ = multigrid.coarse_to_fine([(plan_c, raw_c, coarse.pml, coarse.shape)], n_evl=10, K=4, h0_frac=0.003)
    assert total(plan_c, c_c, raw_c) < 0.5 * total(plan_c, water_c, raw_c)
    phys_shape = tuple(n - 2 * p for n, p in zip(fine.shape, fine.pml[::-1]))
    c_f = multigrid.embed_physical(multigrid.upsample_model(multigrid.physical(c_c, coarse.pml), phys_shape),
                                   fine.shape, fine.pml, synth.C_WATER)
    water_f = torch.full(fine.shape, synth.C_WATER, device="cuda")
    assert total(plan_f, c_f, raw_f) < 0.5 * total(plan_f, water_f, raw_f)
