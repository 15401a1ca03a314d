"""Seeded synthetic inputs for the TD-FWI hot path.

This module only *generates inputs*: sound-speed models, transducer voxel
indices, the reconstruction region Gamma and its boundary layer, the emitted
wavelet and the Rademacher encoding weights.  It holds none of the method's
arithmetic (no wave propagation, no spectral operators, no gradients), so the
FP64 CPU oracle and the CUDA path can both consume exactly the same arrays.

Every floating-point array that the CUDA path receives in FP32 (sound speed,
wavelet) is rounded to FP32 here, so both sides see bit-identical inputs.

Geometry follows the paper's setup (Sec. 4.1): point transducers distributed
over a half sphere by the golden-section method, half of them emitting and half
receiving; tissue sound speeds in the 1470..1650 m/s range in 1500 m/s water;
optimisation bounds c_min = 1350, c_max = 1800 m/s; dt = cfl * dx / c_max with
cfl = 0.3.  The OA-Breast phantom used by the paper is not available, so a
seeded ellipsoidal phantom with inclusions and smoothed noise stands in for it.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np
from scipy import ndimage

C_WATER = 1500.0
C_MIN = 1350.0
C_MAX = 1800.0
CFL = 0.3
RHO0 = 1000.0


def f32(a):
    """Round to the nearest FP32 value and return FP64 (bit-identical inputs)."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def time_step(dx: float, c_max: float = C_MAX, cfl: float = CFL) -> float:
    """dt = cfl * dx / c_max (Sec. 4.1)."""
    return cfl * dx / c_max


def ricker(nt: int, dt: float, f0: float, t0: Optional[float] = None) -> np.ndarray:
    """Ricker wavelet s(t_n), t_n = n dt, unit peak amplitude, delayed by t0 = 1.5/f0."""
    if t0 is None:
        t0 = 1.5 / f0
    t = np.arange(nt) * dt - t0
    a = (math.pi * f0 * t) ** 2
    return f32((1.0 - 2.0 * a) * np.exp(-a))


def bowl_points(n_tot: int, centre, radius: float) -> np.ndarray:
    """Golden-section points on the lower half sphere (opening towards +z).

    Point i sits at depth fraction (i + 1/2)/n_tot below the rim, measured from
    the bottom pole upwards (equal-area in z on a sphere), at azimuth
    i * pi * (3 - sqrt 5).  Returns float grid coordinates (x, y, z), shape (n, 3).
    Point 0 is the one closest to the bottom pole.
    """
    i = np.arange(n_tot, dtype=np.float64)
    h = (i + 0.5) / n_tot                  # 0 at the pole .. 1 at the rim
    depth = 1.0 - h                        # cos(polar angle from the -z axis)
    rxy = np.sqrt(np.maximum(0.0, 1.0 - depth ** 2))
    phi = i * math.pi * (3.0 - math.sqrt(5.0))
    cx, cy, cz = centre
    return np.stack([cx + radius * rxy * np.cos(phi),
                     cy + radius * rxy * np.sin(phi),
                     cz - radius * depth], axis=1)


def nearest_voxel(points: np.ndarray, shape_xyz) -> np.ndarray:
    """Linear index i + nx*(j + ny*k) of the nearest grid point (round half away from zero)."""
    nx, ny, nz = shape_xyz
    r = np.sign(points) * np.floor(np.abs(points) + 0.5)
    r = r.astype(np.int64)
    if (r < 0).any() or (r[:, 0] >= nx).any() or (r[:, 1] >= ny).any() or (r[:, 2] >= nz).any():
        raise ValueError("transducer outside the grid")
    return (r[:, 0] + nx * (r[:, 1] + ny * r[:, 2])).astype(np.int32)


def split_emitters(n_tot: int, n_src: int):
    """Every (n_tot // n_src)-th golden-section point emits, the others receive."""
    step = n_tot // n_src
    ids = np.arange(n_tot)
    is_src = (ids % step == 0) & (ids // step < n_src)
    return np.nonzero(is_src)[0], np.nonzero(~is_src)[0]


def coords(shape_xyz):
    """Index grids (X, Y, Z), each shaped (nz, ny, nx) (x fastest in memory)."""
    nx, ny, nz = shape_xyz
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return X.astype(np.float64), Y.astype(np.float64), Z.astype(np.float64)


def ball_mask(shape_xyz, centre, radius) -> np.ndarray:
    X, Y, Z = coords(shape_xyz)
    return (X - centre[0]) ** 2 + (Y - centre[1]) ** 2 + (Z - centre[2]) ** 2 <= radius ** 2


def half_ellipsoid_mask(shape_xyz, centre, semi) -> np.ndarray:
    X, Y, Z = coords(shape_xyz)
    q = ((X - centre[0]) / semi[0]) ** 2 + ((Y - centre[1]) / semi[1]) ** 2 + ((Z - centre[2]) / semi[2]) ** 2
    return (q <= 1.0) & (Z <= centre[2])


def boundary_layer(gamma: np.ndarray, thickness: int) -> np.ndarray:
    """Voxels of Gamma within Chebyshev distance `thickness` of a voxel outside Gamma.

    This is the 'layer of grid points lying on the inner surface of Gamma'
    (Sec. 4.3) on which the forward pressure is recorded and re-imposed.
    Voxels beyond the grid edge count as outside Gamma.
    """
    outside = ~gamma
    near = ndimage.maximum_filter(outside.astype(np.uint8), size=2 * thickness + 1,
                                  mode="constant", cval=1).astype(bool)
    return gamma & near


def linear_indices(mask: np.ndarray) -> np.ndarray:
    """Sorted linear indices (x fastest) of a (nz, ny, nx) mask."""
    return np.flatnonzero(mask.ravel()).astype(np.int32)


def rademacher(n: int, rng: np.random.Generator) -> np.ndarray:
    """w_i = +-1 with equal probability (Sec. 3.2)."""
    return np.where(rng.integers(0, 2, size=n) == 1, 1.0, -1.0)


def breast_phantom(shape_xyz, pml: int, rng: np.random.Generator, with_detail: bool = True):
    """Seeded stand-in for the breast phantom (tissue speeds of Sec. 4.1).

    Half-ellipsoid breast (1480 m/s) hanging into the bowl, six axis-aligned
    ellipsoidal inclusions (1520..1580 m/s) and Gaussian-smoothed noise of
    +-20 m/s inside the breast; water elsewhere.  Returns (c, gamma, bowl).
    """
    nx, ny, nz = shape_xyz
    z_e = nz - pml - 2
    R = min(nx / 2 - pml - 2, ny / 2 - pml - 2, nz - 2 * pml - 3)
    centre = (nx / 2.0, ny / 2.0, float(z_e))
    semi = (0.7 * R, 0.7 * R, 0.8 * R)
    gamma = half_ellipsoid_mask(shape_xyz, centre, semi)
    c = np.full((nz, ny, nx), C_WATER)
    c[gamma] = 1480.0
    # the random draws are made in a fixed order whether or not they are used
    X, Y, Z = coords(shape_xyz)
    incl = []
    for _ in range(6):
        while True:
            p = rng.uniform(-1.0, 1.0, size=3)
            p[2] = -abs(p[2])
            if (p ** 2).sum() <= 1.0:
                break
        ctr = (centre[0] + 0.6 * semi[0] * p[0], centre[1] + 0.6 * semi[1] * p[1],
               centre[2] + 0.6 * semi[2] * p[2])
        ax = rng.uniform(0.08 * R, 0.2 * R, size=3)
        val = rng.uniform(1520.0, 1580.0)
        incl.append((ctr, ax, val))
    noise = rng.standard_normal((nz, ny, nx))
    if with_detail:
        for ctr, ax, val in incl:
            m = (((X - ctr[0]) / ax[0]) ** 2 + ((Y - ctr[1]) / ax[1]) ** 2
                 + ((Z - ctr[2]) / ax[2]) ** 2 <= 1.0) & gamma
            c[m] = val
        sm = ndimage.gaussian_filter(noise, sigma=2.0, mode="reflect", truncate=4.0)
        sm *= 20.0 / np.abs(sm).max()
        c[gamma] += sm[gamma]
    bowl = dict(centre=centre, radius=float(R))
    return f32(c), gamma, bowl


def optimal_pml(n_phys: int, lo: int = 10, hi: int = 20) -> int:
    """PML size in [lo, hi] minimising the largest prime factor of n_phys + 2*pml (App. B)."""
    def lpf(n):
        best, d = 1, 2
        while d * d <= n:
            while n % d == 0:
                best, n = max(best, d), n // d
            d += 1
        return max(best, n) if n > 1 else best
    return min(range(lo, hi + 1), key=lambda p: (lpf(n_phys + 2 * p), p))


@dataclasses.dataclass
class Workload:
    """One synthetic problem: grid, model(s), transducers, regions, wavelet, weights."""
    name: str
    nx: int
    ny: int
    nz: int
    pml: tuple
    dx: float
    dt: float
    nt: int                     # number of time samples = forward iterations
    c_true: np.ndarray          # (nz, ny, nx) FP32-representable
    c_model: np.ndarray         # current model at which the gradient is taken
    src_idx: np.ndarray         # int32 [n_src] emitter voxels
    rec_idx: np.ndarray         # int32 [n_rec] receiver voxels
    gamma_idx: np.ndarray       # int32 sorted voxels of Gamma
    layer_idx: np.ndarray       # int32 sorted voxels of the boundary layer
    wavelet: np.ndarray         # [nt] FP32-representable
    weights: np.ndarray         # [K, n_src] Rademacher
    c_ref: float = C_MAX
    rho0: float = RHO0
    pml_alpha: float = 2.0
    c_rec: float = C_WATER

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def n_vox(self):
        return self.nx * self.ny * self.nz


def config1(nt: int = 300, layer: int = 2, seed: int = 0) -> Workload:
    """32^3 grid with a 10-cell PML inside; 1550 m/s ball of radius 5 in water;
    one pole emitter and 64 receivers on a bowl of radius 14; Gamma = ball r = 8."""
    n, pml, dx = 32, 10, 0.5e-3
    dt = time_step(dx)
    shp = (n, n, n)
    ctr = (16.0, 16.0, 16.0)
    c_model = np.full((n, n, n), C_WATER)
    c_model[ball_mask(shp, ctr, 5.0)] = 1550.0
    c_true = np.full((n, n, n), C_WATER)
    c_true[ball_mask(shp, ctr, 5.0)] = 1560.0
    gamma = ball_mask(shp, ctr, 8.0)
    pts = bowl_points(65, ctr, 14.0)
    src, rec = split_emitters(65, 1)
    vox = nearest_voxel(pts, shp)
    return Workload("plain-32^3", n, n, n, (pml, pml, pml), dx, dt, nt, f32(c_true), f32(c_model),
                    vox[src], vox[rec], linear_indices(gamma),
                    linear_indices(boundary_layer(gamma, layer)),
                    ricker(nt, dt, 1.0e6), np.ones((1, 1)))


def phantom_workload(name: str, nx: int, ny: int, nz: int, nt: int, n_src: int, n_rec: int,
                     K: int, phantom_seed: int, weight_seeds, pml: int = 10, dx: float = 0.5e-3,
                     layer: int = 8, f0: float = 1.0e6) -> Workload:
    """Breast-phantom workload: true model = full phantom, current model = the
    same phantom without inclusions and noise; K Rademacher super-shots."""
    shp = (nx, ny, nz)
    dt = time_step(dx)
    c_true, gamma, bowl = breast_phantom(shp, pml, np.random.default_rng(phantom_seed), True)
    c_model, _, _ = breast_phantom(shp, pml, np.random.default_rng(phantom_seed), False)
    pts = bowl_points(n_src + n_rec, bowl["centre"], bowl["radius"])
    src, rec = split_emitters(n_src + n_rec, n_src)
    vox = nearest_voxel(pts, shp)
    w = np.stack([rademacher(n_src, np.random.default_rng(s)) for s in weight_seeds])[:K]
    return Workload(name, nx, ny, nz, (pml, pml, pml), dx, dt, nt, c_true, c_model,
                    vox[src], vox[rec], linear_indices(gamma),
                    linear_indices(boundary_layer(gamma, layer)), ricker(nt, dt, f0), w)


def config2() -> Workload:
    """128x128x64 phantom, 256 emitters + 1024 receivers, K = 4 super-shots, 1500 steps."""
    return phantom_workload("plain-128x128x64", 128, 128, 64, 1500, 256, 1024, 4, 1, (2, 3, 4, 5))


def config3_instance(i: int) -> Workload:
    """Instance i (0..15) of the uneven-grid batch: 4 each of 64^3, 96x96x48,
    128x128x64, 160x160x80; 512 receivers + 128 emitters; steps linear in nx."""
    sizes = [(64, 64, 64), (96, 96, 48), (128, 128, 64), (160, 160, 80)]
    nx, ny, nz = sizes[i // 4]
    nt = int(round(1200 + (2000 - 1200) * (nx - 64) / (160 - 64)))
    return phantom_workload(f"batch-{nx}x{ny}x{nz}-{i}", nx, ny, nz, nt, 128, 512, 1,
                            10 + i, (100 + i,))


def config4() -> Workload:
    """96x96x48 phantom, 32 emitters + 128 receivers, K = 1, 1000 steps."""
    return phantom_workload("diff-96x96x48", 96, 96, 48, 1000, 32, 128, 1, 100, (101,))


def smooth_235(n: int) -> bool:
    for f in (2, 3, 5):
        while n % f == 0:
            n //= f
    return n == 1


def tr_box(wl: "Workload", margin: int, pml: int, sizes=None):
    """Box for the TR re-simulation restricted to a region enclosing Gamma (Sec. 3.1):
    Gamma's bounding box grown by `margin` cells and a PML of `pml` cells on every side,
    each extent rounded up to the first size in `sizes` (default: 2-3-5-smooth sizes),
    centred on Gamma and kept inside the grid.  Returns (origin, size, pml) as (x, y, z)
    triples, the argument of Plan(tr_box=...) and of the oracle's tr_box."""
    gi = np.asarray(wl.gamma_idx, dtype=np.int64)
    x, y, z = gi % wl.nx, (gi // wl.nx) % wl.ny, gi // (wl.nx * wl.ny)
    lo = [int(x.min()), int(y.min()), int(z.min())]
    hi = [int(x.max()), int(y.max()), int(z.max())]
    n = [wl.nx, wl.ny, wl.nz]
    origin, size = [], []
    for a in range(3):
        need = hi[a] - lo[a] + 1 + 2 * (margin + pml)
        cand = [s for s in (sizes if sizes is not None else range(need, n[a] + 1)) if s >= need and s <= n[a]]
        cand = [s for s in cand if smooth_235(s)]
        m = min(cand) if cand else n[a]
        o = lo[a] - (m - (hi[a] - lo[a] + 1)) // 2
        o = min(max(o, 0), n[a] - m)
        if lo[a] - o < pml or o + m - 1 - hi[a] < pml:
            raise ValueError("Gamma does not fit inside the TR box's PML-free interior")
        origin.append(o)
        size.append(m)
    return tuple(origin), tuple(size), (pml, pml, pml)


def encoding_draws(seed: int, K: int, n_src: int, tau: int = 0):
    """Rademacher weights [K][n_src] and delays [K][n_src] (whole time steps, d ~ U[0, 1]
    times tau, rounded; zero when tau = 0) of the stochastic approximation number `seed`
    of the encoded gradient estimator (Sec. 3.2, Eq. 13)."""
    rng = np.random.default_rng(seed)
    w = np.where(rng.integers(0, 2, size=(K, n_src)) == 1, 1.0, -1.0)
    d = np.rint(rng.uniform(0.0, 1.0, size=(K, n_src)) * tau).astype(np.int32)
    return w, d


def smooth_direction(wl: Workload, seed: int, n_terms: int = 4) -> np.ndarray:
    """Seeded smooth perturbation direction supported in Gamma: a sum of n_terms
    low-order 3D cosines (wavenumbers 0..3 per axis, random phases) restricted to
    Gamma and scaled to max |.| = 1.  Shape (nz, ny, nx)."""
    rng = np.random.default_rng(seed)
    X, Y, Z = coords((wl.nx, wl.ny, wl.nz))
    d = np.zeros(wl.shape)
    for _ in range(n_terms):
        k = rng.integers(0, 4, size=3)
        ph = rng.uniform(0.0, 2.0 * math.pi)
        d += np.cos(2.0 * math.pi * (k[0] * X / wl.nx + k[1] * Y / wl.ny + k[2] * Z / wl.nz) + ph)
    m = np.zeros(wl.n_vox)
    m[wl.gamma_idx] = 1.0
    d *= m.reshape(wl.shape)
    return d / np.abs(d).max()


SERVING_LEVELS = {
    # physical voxels, dx, steps; the PML is added outside by the App. B size rule
    0: ((111, 111, 56), 2.0e-3, 1000),
    1: ((221, 221, 111), 1.0e-3, 2000),
    2: ((442, 442, 222), 0.5e-3, 4000),
}


def serving_level(level: int, n_src: int, seed: int, n_rec: int = 1024, pz: int = None,
                  nt: int = None) -> Workload:
    """A multigrid level of the serving stream: physical grid padded by the PML
    size rule, Ricker frequency scaled with dx (1 MHz at 0.5 mm).  `pz` replaces the
    physical z extent (a thinner grid with the same planes, for profiling); `nt`
    replaces the level's number of time steps (a shorter window of the same pulse)."""
    (px, py, pz0), dx, nt0 = SERVING_LEVELS[level]
    pz = pz0 if pz is None else pz
    nt = nt0 if nt is None else nt
    P = [optimal_pml(n) for n in (px, py, pz)]
    nx, ny, nz = px + 2 * P[0], py + 2 * P[1], pz + 2 * P[2]
    shp = (nx, ny, nz)
    dt = time_step(dx)
    rng = np.random.default_rng(seed)
    # breast in the physical region, bowl radius 0.473 of the physical width
    z_e = P[2] + pz - 2
    # the bowl must stay in the physical region when z is overridden (its lowest point on
    # the first physical plane); for the levels' own extents 0.473 px is the smaller
    R = min(0.473 * px, float(z_e - P[2]))
    centre = (nx / 2.0, ny / 2.0, float(z_e))
    semi = (0.7 * 0.7 * R, 0.7 * 0.7 * R, 0.8 * 0.7 * R)
    gamma = half_ellipsoid_mask(shp, centre, semi)
    c_model = np.full((nz, ny, nx), C_WATER)
    c_model[gamma] = 1480.0
    c_true = c_model.copy()
    c_true[gamma] += rng.uniform(-20.0, 20.0)
    pts = bowl_points(n_src + n_rec, centre, R)
    src, rec = split_emitters(n_src + n_rec, n_src)
    vox = nearest_voxel(pts, shp)
    w = rademacher(n_src, rng)[None, :]
    f0 = 1.0e6 * 0.5e-3 / dx
    return Workload(f"serve-L{level}-{nx}x{ny}x{nz}", nx, ny, nz, tuple(P), dx, dt, nt,
                    f32(c_true), f32(c_model), vox[src], vox[rec], linear_indices(gamma),
                    linear_indices(boundary_layer(gamma, 8)), ricker(nt, dt, f0), w)


def small_workload(nx: int, ny: int, nz: int, nt: int, pml: int = 4, n_src: int = 3,
                   n_rec: int = 24, K: int = 2, layer: int = 2, seed: int = 7,
                   f0: float = 0.25e6, dx: float = 1.0e-3, hetero: bool = True,
                   gamma_frac: float = 0.22) -> Workload:
    """Small ragged-size workload for parity tests (sizes need not be powers of 2)."""
    rng = np.random.default_rng(seed)
    shp = (nx, ny, nz)
    dt = time_step(dx)
    ctr = ((nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0)
    rad = gamma_frac * min(nx, ny, nz)
    gamma = ball_mask(shp, ctr, rad)
    c_model = np.full((nz, ny, nx), C_WATER)
    if hetero:
        c_model += rng.uniform(-30.0, 30.0, size=c_model.shape) * gamma
    c_true = c_model + 25.0 * gamma
    R = min(0.45 * min(nx, ny) - 0.5, (ctr[2] - 0.5) / 0.75)
    pts = bowl_points(n_src + n_rec, (ctr[0], ctr[1], ctr[2] + 0.25 * R), R)
    src, rec = split_emitters(n_src + n_rec, n_src)
    vox = nearest_voxel(pts, shp)
    w = np.stack([rademacher(n_src, rng) for _ in range(K)])
    return Workload(f"small-{nx}x{ny}x{nz}", nx, ny, nz, (pml, pml, pml), dx, dt, nt,
                    f32(c_true), f32(c_model), vox[src], vox[rec], linear_indices(gamma),
                    linear_indices(boundary_layer(gamma, layer)), ricker(nt, dt, f0), w)
