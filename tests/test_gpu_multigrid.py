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
