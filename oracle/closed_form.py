"""Closed-form receiver traces of the k-space scheme in a homogeneous periodic medium.

TEST INFRASTRUCTURE ONLY.  Only the test-suite may import this module; the
product path never does.

App. B states that the kappa-corrected k-space scheme is exact for a
homogeneous medium at c = c_ref.  Written per Fourier mode (PML off, uniform c,
constant rho0), the split-density update of Alg. 1 reduces to

    p_n - 2 x p_(n-1) + p_(n-2) = c^2 beta (s_n - s_(n-1)) e_hat,
    x = 1 - 2 (c/c_ref)^2 sin^2(c_ref dt |k| / 2),   beta = 2 dt / (dx c),

for a unit-weight point source at voxel s (e_hat = exp(-i k.s)); the three
injected density components add 3 * 2 dt / (3 dx c) per unit of s.  Hence
p_n = c^2 beta e_hat y_n with the scalar recurrence
y_n = 2 x y_(n-1) - y_(n-2) + (s_n - s_(n-1)), y_(-1) = y_(-2) = 0, s_(-1) = 0,
and the trace at receiver r is the inverse DFT of that mode sum evaluated at r:

    f_n(r) = (c^2 beta / N) sum_k cos(k.(r - s)) y_n(k).

Because y depends on k only through |k|, the sum runs over the half spectrum
kx >= 0 with weight 2 on the interior kx columns.  The work per time step is a
few passes over (nx/2+1) ny nz doubles, which makes the closed form usable at
grid sizes where the time-stepping oracle is too slow.  It is pinned against
the oracle's forward simulation on small grids.
"""
from __future__ import annotations

import math

import numpy as np


def _k1(n: int, dx: float, half: bool) -> np.ndarray:
    j = np.arange(n // 2 + 1) if half else np.arange(n)
    m = np.where(j < (n + 1) // 2, j, j - n)
    return 2.0 * math.pi * m / (n * dx)


def homogeneous_traces(shape_xyz, dx: float, dt: float, c_ref: float, c: float, src: int,
                       rec_idx, wavelet, nt: int) -> np.ndarray:
    """Traces [nt, n_rec] of a unit-weight point source at linear voxel `src`
    recorded at linear voxels `rec_idx`, uniform sound speed c, no PML."""
    nx, ny, nz = shape_xyz
    kx, ky, kz = _k1(nx, dx, True), _k1(ny, dx, False), _k1(nz, dx, False)
    k2 = kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2
    x2 = 2.0 * (1.0 - 2.0 * (c / c_ref) ** 2 * np.sin(0.5 * c_ref * dt * np.sqrt(k2)) ** 2)
    del k2
    hx = nx // 2 + 1
    wx = np.full(hx, 2.0)
    wx[0] = 1.0
    if nx % 2 == 0:
        wx[-1] = 1.0
    # displacements r - s per axis (integer voxels)
    rec_idx = np.asarray(rec_idx, dtype=np.int64)
    s = int(src)
    sx, sy, sz = s % nx, (s // nx) % ny, s // (nx * ny)
    dxv, dyv, dzv = rec_idx % nx - sx, (rec_idx // nx) % ny - sy, rec_idx // (nx * ny) - sz
    # separable phases: exp(i 2 pi j d / n) per axis
    ex = np.exp(2j * math.pi * np.outer(np.arange(hx), dxv) / nx) * wx[:, None]      # [hx, R]
    ey = np.exp(2j * math.pi * np.outer(np.arange(ny), dyv) / ny)                     # [ny, R]
    ez = np.exp(2j * math.pi * np.outer(np.arange(nz), dzv) / nz)                     # [nz, R]
    exr = np.ascontiguousarray(np.concatenate([ex.real, ex.imag], axis=1))             # [hx, 2R]
    R = len(rec_idx)
    ds = np.diff(np.concatenate([[0.0], np.asarray(wavelet, np.float64)[:nt]]))
    scale = c * c * (2.0 * dt / (dx * c)) / (nx * ny * nz)
    y1 = np.zeros_like(x2)      # y_(n-1)
    y2 = np.zeros_like(x2)      # y_(n-2)
    out = np.zeros((nt, R))
    for n in range(nt):
        # y_n = 2 x y_(n-1) - y_(n-2) + ds_n, written over y_(n-2)
        np.subtract(x2 * y1, y2, out=y2)
        y2 += ds[n]
        y1, y2 = y2, y1
        a = y1.reshape(nz * ny, hx) @ exr                       # [nz*ny, 2R]
        a = (a[:, :R] + 1j * a[:, R:]).reshape(nz, ny, R)
        b = np.einsum("zyr,yr->zr", a, ey)
        out[n] = scale * np.einsum("zr,zr->r", b, ez).real
    return out
