"""TR re-simulation on a box enclosing Gamma (Sec. 3.1) on the GPU, against the oracle's
box gradient (same box, same PML rule, c0 cropped from the model).

Tolerances as for the whole-grid gradient: traces rel l2 <= 1e-4, misfit <= 1e-3,
gradient <= 1e-3.
"""
import numpy as np
import pytest
import torch

from paper_2102_00755_b300 import build as fbuild
from paper_2102_00755_b300 import fwi, synth

from . import oracle_cases as oc
from oracle import pstd

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


def _gpu(wl, f_obs, pairing, box):
    plan = fwi.Plan.from_workload(wl, pairing=pairing, max_shots=len(wl.weights), tr_box=box)
    traces = torch.empty((len(wl.weights), wl.nt, len(wl.rec_idx)), dtype=torch.float32, device="cuda")
    D, g = plan.gradient(_dev(wl.c_model).reshape(-1), _dev(wl.weights), _dev(f_obs), traces=traces)
    assert plan.status() == fwi.FWI_OK
    return plan, traces.cpu().numpy(), D.cpu().numpy(), g.cpu().numpy().reshape(wl.shape)


def _oracle(wl, f_obs, pairing, box):
    G = pstd.grid_for(wl)
    fs, Ds, gs = [], [], []
    for k, w in enumerate(wl.weights):
        f, D, g = pstd.fwi_gradient(G, wl.c_model, wl.src_idx, w, wl.wavelet, wl.rec_idx, wl.layer_idx,
                                    wl.gamma_idx, f_obs[k], pairing=pairing, c_rec=wl.c_rec, tr_box=box)
        fs.append(f)
        Ds.append(D)
        gs.append(g)
    return np.stack(fs), np.array(Ds), np.mean(gs, axis=0)


def _compare(wl, f_obs, pairing, box):
    f_ref, D_ref, g_ref = _oracle(wl, f_obs, pairing, box)
    plan, tr, D, g = _gpu(wl, f_obs, pairing, box)
    for k in range(len(wl.weights)):
        assert oc.rel(tr[k], f_ref[k]) < TOL_TRACES
    assert np.all(np.abs(D - D_ref) <= TOL_MISFIT * np.abs(D_ref)), (D, D_ref)
    assert oc.rel(g, g_ref) < TOL_GRAD, oc.rel(g, g_ref)
    gam = np.zeros(wl.n_vox, bool)
    gam[wl.gamma_idx] = True
    assert np.all(g.reshape(-1)[~gam] == 0.0)
    return plan


def _small():
    wl = synth.small_workload(36, 36, 30, 90, pml=4, n_src=3, n_rec=30, K=2, layer=3, seed=5, f0=0.4e6,
                              gamma_frac=0.25)
    return wl, oc.observed(wl)


@pytest.mark.parametrize("pairing,margin", [("literal", 2), ("exact", 4)])
def test_tr_box_gradient_parity(pairing, margin):
    wl, f_obs = _small()
    box = synth.tr_box(wl, margin, 3)
    plan = _compare(wl, f_obs, pairing, box)
    # the box's voxel-steps replace the whole grid's in the TR phase
    Nt = wl.nt - 1
    nadj = Nt - 1 if pairing == "literal" else Nt + 1
    nbox = box[1][0] * box[1][1] * box[1][2]
    assert plan.voxel_steps(2, True) == 2 * ((wl.nt + nadj) * wl.n_vox + Nt * nbox)


def test_tr_box_covering_the_grid_is_bit_identical_to_whole_grid_tr():
    """The box plan on the whole grid runs the same kernels on the same values: its
    gradient equals the whole-grid TR gradient bit for bit."""
    wl, f_obs = _small()
    box = ((0, 0, 0), (wl.nx, wl.ny, wl.nz), wl.pml)
    _, tr1, D1, g1 = _gpu(wl, f_obs, "literal", box)
    _, tr2, D2, g2 = _gpu(wl, f_obs, "literal", None)
    assert np.array_equal(tr1, tr2) and np.array_equal(D1, D2) and np.array_equal(g1, g2)


def test_tr_box_on_the_bench_grid():
    """128x128x64 phantom (256 + 1024 transducers, PML 10) with the 96x96x64 box that the
    benchmark's TR-box line times (margin 8, PML 8 inside the box), 160 steps, the first
    two of the benchmark's super-shots (as in the whole-grid parity test of this grid)."""
    wl = synth.phantom_workload("plain-128x128x64", 128, 128, 64, 160, 256, 1024, 2, 1, (2, 3))
    box = synth.tr_box(wl, 8, 8, sizes=(32, 48, 64, 80, 96, 128))
    assert box[1] == (96, 96, 64)
    _compare(wl, oc.observed(wl), "literal", box)
