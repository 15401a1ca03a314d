"""Synthetic serving-level inputs: grid sizes, transducer placement and region lists,
including the thinned z extent used for profiling (no GPU)."""
import numpy as np
import pytest

from paper_2102_00755_b300 import synth


def _zyx(idx, wl):
    x = idx % wl.nx
    y = (idx // wl.nx) % wl.ny
    z = idx // (wl.nx * wl.ny)
    return z, y, x


@pytest.mark.parametrize("level,pz,shape", [(0, None, (96, 135, 135)), (1, None, (135, 243, 243)),
                                            (1, 20, (48, 243, 243)), (2, 20, (48, 480, 480))])
def test_serving_level_geometry(level, pz, shape):
    wl = synth.serving_level(level, n_src=8, seed=3, pz=pz)
    assert wl.shape == shape
    px, py, pzl = wl.pml
    assert (wl.nx - 2 * px, wl.ny - 2 * py) == synth.SERVING_LEVELS[level][0][:2]
    n_vox = wl.nx * wl.ny * wl.nz
    assert len(wl.src_idx) == 8 and len(wl.rec_idx) == 1024
    for idx in (wl.src_idx, wl.rec_idx, wl.gamma_idx, wl.layer_idx):
        assert idx.dtype == np.int32
        assert np.all((idx >= 0) & (idx < n_vox))
    for idx in (wl.gamma_idx, wl.layer_idx):
        assert np.all(np.diff(idx) > 0)                      # sorted, unique
    # every transducer sits in the physical region, outside the PML
    for idx in (wl.src_idx, wl.rec_idx):
        z, y, x = _zyx(idx.astype(np.int64), wl)
        assert np.all((x >= px) & (x < wl.nx - px))
        assert np.all((y >= py) & (y < wl.ny - py))
        assert np.all((z >= pzl) & (z < wl.nz - pzl))
    # models: water outside the breast, sound speeds of soft tissue inside
    assert wl.c_true.shape == shape and wl.c_model.shape == shape
    assert 1300.0 < float(wl.c_true.min()) and float(wl.c_true.max()) < 1800.0
    assert float(wl.c_model[0, 0, 0]) == synth.C_WATER
    assert len(wl.wavelet) == wl.nt
