"""Oracle results for the parity tests, computed once per process and cached.

Only this test helper (and the benchmark's CPU leg) drives the FP64 oracle; the
CUDA path never sees it.  Observed data are the oracle's forward traces of the
true model, rounded to FP32 so that both sides receive identical inputs.
"""
import functools

import numpy as np

from oracle import pstd
from paper_2102_00755_b300 import synth


def observed(wl, weights=None, pml_on=True):
    """Encoded observed traces [K, nt, n_rec] (FP32-rounded) from the true model."""
    G = pstd.grid_for(wl, pml_on)
    W = wl.weights if weights is None else weights
    out = [pstd.forward(G, wl.c_true, wl.src_idx, w, wl.wavelet, wl.rec_idx)[0] for w in W]
    return synth.f32(np.stack(out))


def forward(wl, c, weights, pml_on=True):
    G = pstd.grid_for(wl, pml_on)
    return np.stack([pstd.forward(G, c, wl.src_idx, w, wl.wavelet, wl.rec_idx)[0] for w in weights])


def gradient(wl, f_obs, pairing, c_rec=None, pml_on=True, weights=None):
    """(traces [K, nt, n_rec], misfit [K], mean gradient over K) from the oracle."""
    G = pstd.grid_for(wl, pml_on)
    W = wl.weights if weights is None else weights
    fs, Ds, gs = [], [], []
    for k, w in enumerate(W):
        f, D, g = pstd.fwi_gradient(G, wl.c_model, wl.src_idx, w, wl.wavelet, wl.rec_idx, wl.layer_idx,
                                    wl.gamma_idx, f_obs[k], pairing=pairing, c_rec=c_rec)
        fs.append(f)
        Ds.append(D)
        gs.append(g)
    return np.stack(fs), np.array(Ds), np.mean(gs, axis=0)


@functools.lru_cache(maxsize=None)
def small_case(shape=(24, 20, 18), nt=80, pml=4, K=2, layer=2, seed=7):
    wl = synth.small_workload(*shape, nt, pml=pml, K=K, layer=layer, seed=seed)
    return wl, observed(wl)


@functools.lru_cache(maxsize=None)
def small_gradient(pairing, shape=(24, 20, 18), nt=80):
    wl, f_obs = small_case(shape, nt)
    return gradient(wl, f_obs, pairing, c_rec=wl.c_rec)


@functools.lru_cache(maxsize=None)
def config1_case():
    wl = synth.config1()
    return wl, observed(wl)


@functools.lru_cache(maxsize=None)
def config1_gradient(pairing):
    wl, f_obs = config1_case()
    return gradient(wl, f_obs, pairing, c_rec=wl.c_rec)


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
