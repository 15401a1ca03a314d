"""Write tests/golden/config4_fd.npz: FP64 oracle reference for the differentiation
configuration (96x96x48 phantom, 32 emitters + 128 receivers, 1000 steps, one
Rademacher super-shot, exact pairing, 10-cell PML).

Stored: the observed traces of the true model (FP32-rounded, the input both sides
use), the misfit at the current model, the oracle gradient on Gamma, and central
finite differences of the misfit along 8 seeded smooth directions (h = 1e-3 m/s).
Calls only the oracle (and the seeded input generators).  Run from the repo root:

    python tests/golden/make_config4_fd.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import pstd  # noqa: E402
from paper_2102_00755_b300 import synth  # noqa: E402

H = 1e-3
SEEDS = list(range(100, 108))


def main():
    t0 = time.time()
    wl = synth.config4()
    G = pstd.grid_for(wl)
    w = wl.weights[0]
    f_obs = synth.f32(pstd.forward(G, wl.c_true, wl.src_idx, w, wl.wavelet, wl.rec_idx)[0])
    print("observed", time.time() - t0, flush=True)
    _, D0, grad = pstd.fwi_gradient(G, wl.c_model, wl.src_idx, w, wl.wavelet, wl.rec_idx, wl.layer_idx,
                                    wl.gamma_idx, f_obs, pairing="exact", c_rec=wl.c_rec)
    print("gradient", time.time() - t0, flush=True)

    def misfit(c):
        f, _ = pstd.forward(G, c, wl.src_idx, w, wl.wavelet, wl.rec_idx)
        return pstd.adjoint_source(f, f_obs)[0]

    fd, gd = [], []
    for s in SEEDS:
        d = synth.smooth_direction(wl, s)
        fd.append((misfit(wl.c_model + H * d) - misfit(wl.c_model - H * d)) / (2 * H))
        gd.append(float(np.sum(grad * d)))
        print("direction", s, fd[-1], gd[-1], time.time() - t0, flush=True)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "config4_fd.npz")
    np.savez_compressed(out, observed=f_obs.astype(np.float32)[None], D0=D0,
                        grad_gamma=grad.reshape(-1)[wl.gamma_idx], fd=np.array(fd),
                        oracle_dir=np.array(gd), seeds=np.array(SEEDS), h=H)
    print("wrote", out, time.time() - t0)


if __name__ == "__main__":
    main()
