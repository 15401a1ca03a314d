"""FP64 CPU oracle of the time-reversal based sound-speed gradient.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
baseline leg of the benchmark may import this module; the product path never
does and there is no CPU fallback built on it.

It is a plain, slow, literal restatement of the paper's discrete method in
FP64 (numpy/scipy; scipy's FFT is used as the discrete Fourier transform step,
nothing else is borrowed):

* k-space derivative with kappa correction and staggering: App. B, Eqs. 18-19.
* the split-density first-order scheme with PML multipliers and a mass source
  converted from a pressure source by 2 dt / (3 dx c0): Alg. 1, forward part.
* residual reversal, misfit, cumulative sum, time-reversal re-simulation with a
  Dirichlet boundary layer, and the interleaved adjoint/TR loop assembling the
  gradient 2/(dt c0^3) (p+ - 2 p0 + p-) p_adj on Gamma: Alg. 1, second part
  (continuous counterpart Eq. 10 and TR wave equation Eq. 11, Sec. 3.1).
* source encoding: s_hat = sum_i w_i s_i, f_hat = sum_i w_i f_i (Sec. 3.2), and the
  delayed encoding of Eq. 13: s_hat(t) = sum_i w_i s_i(t - d_i tau), f_hat(t) =
  sum_i w_i f_i(t - d_i tau), with each delay d_i tau a whole number of time steps.

Readings where the paper is silent (all listed in the design notes):
* sinc is the unnormalised sin(x)/x, sinc(0) = 1; c_ref = c_max fixes both
  kappa and dt; the Nyquist wavenumber of an even axis is -pi/dx.
* PML: sigma(d) = alpha (c_ref/dx) (d/P)^4 for distance d (cells) into a layer
  of P cells inside the grid, Lambda = exp(-sigma dt / 2), applied twice per
  update as Alg. 1 nests it.  The nesting is pinned by the closed form of a uniformly
  absorbing medium; the profile values are parity unpinned (the paper only says
  "multiplication operators"; the tests pin their qualitative properties only).
* pairing="literal" runs Alg. 1 exactly as printed.  pairing="exact" is the
  exact discrete adjoint of the (PML-free) scheme: the adjoint injects the
  cumulative residual Q^j at its step j = 0..Nt and its state after step j is
  paired with the TR second difference p_(Nt-j) - 2 p_(Nt-j-1) + p_(Nt-j-2)
  (forward states before step 0 are zero).
* history=True replaces the TR re-simulation by the stored forward field on
  Gamma (the paper's "full" gradient, Table 2).
* tr_box restricts the TR re-simulation to a box enclosing Gamma (Sec. 3.1: the TR
  simulation domain only needs to enclose Gamma).  The box is a grid of its own
  with the same dx, dt and c_ref, its own PML inside it (same profile rule), and c0
  cropped from the full model; the boundary layer and Gamma keep their order.

Arrays are shaped (nz, ny, nx), x fastest, linear index i + nx*(j + ny*k).
Component order xi = (x, y, z) maps to array axes (2, 1, 0).
"""
from __future__ import annotations

import math
import os

import numpy as np
from scipy import fft as sfft

AXES = (2, 1, 0)   # array axis of the x, y and z components


def _workers():
    return int(os.environ.get("ORACLE_WORKERS", os.cpu_count() or 1))


def wavenumbers(n: int, dx: float) -> np.ndarray:
    """Discrete wavenumbers k[j] = 2 pi / (n dx) * (j if j < ceil(n/2) else j - n)."""
    j = np.arange(n)
    m = np.where(j < (n + 1) // 2, j, j - n)
    return 2.0 * math.pi * m / (n * dx)


def sinc(a):
    """Unnormalised sinc, sin(a)/a with sinc(0) = 1."""
    a = np.asarray(a, dtype=np.float64)
    out = np.ones_like(a)
    nz = a != 0.0
    out[nz] = np.sin(a[nz]) / a[nz]
    return out


def pml_profile(n: int, P: int, alpha: float, c_ref: float, dx: float, dt: float, staggered: bool):
    """1D PML multiplier Lambda along one axis (reading of App. B's Lambda, Lambda^s).

    Grid point i sits at x = i (normal grid) or x = i + 1/2 (staggered grid);
    the distance into the layer is d = P - x on the low side (x < P) and
    d = x - (n - 1 - P) on the high side (x > n - 1 - P).
    """
    lam = np.ones(n)
    if P <= 0 or alpha == 0.0:
        return lam
    x = np.arange(n) + (0.5 if staggered else 0.0)
    d = np.zeros(n)
    lo = x < P
    hi = x > (n - 1 - P)
    d[lo] = P - x[lo]
    d[hi] = x[hi] - (n - 1 - P)
    sigma = alpha * (c_ref / dx) * (d / P) ** 4
    lam = np.exp(-sigma * dt / 2.0)
    return lam


class Grid:
    """Spectral operators and PML tables of one grid (App. B)."""

    def __init__(self, nx, ny, nz, dx, dt, c_ref, rho0=1000.0, pml=(0, 0, 0), pml_alpha=2.0):
        self.nx, self.ny, self.nz = nx, ny, nz
        self.shape = (nz, ny, nx)
        self.dx, self.dt, self.c_ref, self.rho0 = dx, dt, c_ref, rho0
        k1 = [wavenumbers(n, dx) for n in (nx, ny, nz)]
        kx = k1[0][None, None, :]
        ky = k1[1][None, :, None]
        kz = k1[2][:, None, None]
        kmag = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
        # Eq. 18: kappa = sinc(c_ref dt |k| / 2)
        self.kappa = sinc(c_ref * dt / 2.0 * kmag)
        kk = (kx, ky, kz)
        # Eq. 19: staggered k-space derivative multipliers i k_xi kappa exp(+-i k_xi dx / 2)
        self.d_plus = [1j * k * self.kappa * np.exp(1j * k * dx / 2.0) for k in kk]
        self.d_minus = [1j * k * self.kappa * np.exp(-1j * k * dx / 2.0) for k in kk]
        ns = (nx, ny, nz)
        self.lam = []
        self.lam_s = []
        for a in range(3):
            shp = [1, 1, 1]
            shp[AXES[a]] = ns[a]
            self.lam.append(pml_profile(ns[a], pml[a], pml_alpha, c_ref, dx, dt, False).reshape(shp))
            self.lam_s.append(pml_profile(ns[a], pml[a], pml_alpha, c_ref, dx, dt, True).reshape(shp))

    # -- k-space derivative (Eq. 19) -------------------------------------------------
    def fft(self, g):
        return sfft.fftn(g, workers=_workers())

    def deriv(self, g_hat, mult):
        """F^-1{ mult * g_hat }, real part (the multipliers are Hermitian)."""
        return np.real(sfft.ifftn(mult * g_hat, workers=_workers()))


class State:
    """Fields of one simulation: v_xi, split density rho_xi, pressure p."""

    def __init__(self, shape):
        self.v = [np.zeros(shape) for _ in range(3)]
        self.rho = [np.zeros(shape) for _ in range(3)]
        self.p = np.zeros(shape)


def step(G: Grid, S: State, c2: np.ndarray, mass_src=None, dirichlet=None):
    """One iteration of the scheme (Alg. 1, forward loop body).

    mass_src: array added to every rho_xi after its update (already scaled by
    2 dt / (3 dx c0)).  dirichlet: (idx, values) overwriting rho_xi at those
    voxels after the update (TR boundary condition).
    """
    dt, rho0 = G.dt, G.rho0
    P = G.fft(S.p)
    for a in range(3):                               # momentum conservation
        S.v[a] = G.lam_s[a] * (G.lam_s[a] * S.v[a] - dt / rho0 * G.deriv(P, G.d_plus[a]))
    for a in range(3):                               # mass conservation
        Va = G.fft(S.v[a])
        S.rho[a] = G.lam[a] * (G.lam[a] * S.rho[a] - dt * rho0 * G.deriv(Va, G.d_minus[a]))
        if mass_src is not None:
            S.rho[a] = S.rho[a] + mass_src
    if dirichlet is not None:
        idx, val = dirichlet
        for a in range(3):
            S.rho[a].reshape(-1)[idx] = val
    S.p = c2 * (S.rho[0] + S.rho[1] + S.rho[2])     # pressure-density relation


def injection_map(G: Grid, c: np.ndarray, idx: np.ndarray, amp: np.ndarray) -> np.ndarray:
    """(2 dt / (3 dx c0)) * S a: point injection of amplitudes `amp` at voxels
    `idx` (duplicates add up), divided by c0 there (App. B, Alg. 1)."""
    m = np.zeros(G.shape).reshape(-1)
    np.add.at(m, idx, amp)
    m = m.reshape(G.shape)
    return 2.0 * G.dt / (3.0 * G.dx * c) * m


def forward(G: Grid, c: np.ndarray, src_idx, src_weights, wavelet, rec_idx, layer_idx=None,
            nt=None, gamma_idx=None, record_field=False, delays=None):
    """Forward iteration of Alg. 1 for the encoded source sum_i w_i s_i, or, with
    delays (whole time steps per source, Eq. 13), sum_i w_i s(t_n - delays_i dt).

    Returns f [nt, n_rec], g [nt, n_layer] (or None), and, if gamma_idx is given,
    the stored forward field on Gamma [nt, n_gamma] (the 'full' variant);
    record_field=True also returns all pressure fields [nt, nz, ny, nx].
    """
    nt = len(wavelet) if nt is None else nt
    c2 = c * c
    S = State(G.shape)
    f = np.zeros((nt, len(rec_idx)))
    g = np.zeros((nt, len(layer_idx))) if layer_idx is not None else None
    hist = np.zeros((nt, len(gamma_idx))) if gamma_idx is not None else None
    fields = np.zeros((nt,) + G.shape) if record_field else None
    w = np.asarray(src_weights, dtype=np.float64)
    src_idx = np.asarray(src_idx)
    base = injection_map(G, c, src_idx, w)            # time-independent part of S s_hat
    if delays is not None:
        delays = np.asarray(delays, dtype=np.int64)
    for n in range(nt):
        if delays is None:
            src = base * wavelet[n]
        else:                                          # source i emits s(t_n - delays_i dt)
            m = n - delays
            s_i = np.where((m >= 0) & (m < len(wavelet)), np.asarray(wavelet)[np.clip(m, 0, len(wavelet) - 1)], 0.0)
            src = injection_map(G, c, src_idx, w * s_i)
        step(G, S, c2, mass_src=src)
        pf = S.p.reshape(-1)
        f[n] = pf[rec_idx]                            # f^n = M p
        if g is not None:
            g[n] = pf[layer_idx]                      # g^n = p(dGamma)
        if hist is not None:
            hist[n] = pf[gamma_idx]
        if fields is not None:
            fields[n] = S.p
    out = [f, g]
    if gamma_idx is not None:
        out.append(hist)
    if record_field:
        out.append(fields)
    return tuple(out)


def encode_data(weights, data, delays=None, nt=None):
    """f_hat = sum_i w_i f_i for per-source data [n_src, nt_data, n_rec] (Sec. 3.2); with
    delays (whole time steps), f_hat[n] = sum_i w_i f_i[n - delays_i] (Eq. 13), zero
    where n - delays_i falls outside the data, over nt samples (default nt_data)."""
    w = np.asarray(weights, dtype=np.float64)
    data = np.asarray(data, dtype=np.float64)
    if delays is None:
        return np.tensordot(w, data, axes=1)
    nt = data.shape[1] if nt is None else nt
    out = np.zeros((nt, data.shape[2]))
    for i, d in enumerate(np.asarray(delays, dtype=np.int64)):
        for n in range(max(0, d), min(nt, d + data.shape[1])):
            out[n] += w[i] * data[i, n - d]
    return out


def adjoint_source(f, f_obs):
    """q^n = f^(Nt-n) - f_obs(T - t_n); D = 0.5 ||q||^2; Q = cumsum_n q (Alg. 1)."""
    q = f[::-1] - f_obs[::-1]
    D = 0.5 * float(np.sum(q * q))
    Q = np.cumsum(q, axis=0)
    return D, Q


def box_indices(shape, origin, size, idx):
    """Linear indices idx of a grid of `shape` (nz, ny, nx) -> linear indices of the box of
    `size` (nx', ny', nz') whose first voxel is `origin` (x0, y0, z0).  Every voxel must lie
    inside the box.  Cropping keeps the (z, y, x) order, so sorted lists stay sorted."""
    nz, ny, nx = shape
    idx = np.asarray(idx, dtype=np.int64)
    x = idx % nx
    y = (idx // nx) % ny
    z = idx // (nx * ny)
    xb, yb, zb = x - origin[0], y - origin[1], z - origin[2]
    if np.any((xb < 0) | (xb >= size[0]) | (yb < 0) | (yb >= size[1]) | (zb < 0) | (zb >= size[2])):
        raise ValueError("a voxel lies outside the TR box")
    return xb + size[0] * (yb + size[1] * zb)


def tr_grid(G: Grid, c: np.ndarray, tr_box, pml_alpha=2.0):
    """Grid and cropped sound speed of the TR box (origin, size, pml), see `gradient`."""
    origin, size, pml = tr_box
    Gb = Grid(size[0], size[1], size[2], G.dx, G.dt, G.c_ref, G.rho0, pml, pml_alpha)
    x0, y0, z0 = origin
    cb = c[z0:z0 + size[2], y0:y0 + size[1], x0:x0 + size[0]]
    if cb.shape != Gb.shape:
        raise ValueError("the TR box must lie inside the grid")
    return Gb, np.ascontiguousarray(cb)


def gradient(G: Grid, c: np.ndarray, f, f_obs, rec_idx, layer_idx, gamma_idx, g,
             pairing="literal", history=None, c_rec=None, tr_box=None, pml_alpha=2.0):
    """Misfit and sound-speed gradient of Alg. 1 (second part).

    f, f_obs: simulated and observed (encoded) traces [nt, n_rec]; g: boundary
    history [nt, n_layer] from `forward`.  Returns (D, grad) where grad has the
    grid's shape and is zero outside Gamma.  With c_rec given the raw Alg. 1
    accumulator is multiplied by dx * c_rec / 2, which makes the exact pairing
    equal dD/dc when every receiver sits in a medium of speed c_rec (without
    PML); without it the raw accumulator is returned.  tr_box = (origin (x0, y0, z0),
    size (nx', ny', nz'), pml (px, py, pz)) runs the TR re-simulation on that box only
    (its own PML of strength pml_alpha inside it); None runs it on the whole grid.
    """
    nt = f.shape[0]
    Nt = nt - 1
    c2 = c * c
    cf = c.reshape(-1)
    D, Q = adjoint_source(f, f_obs)
    gamma_idx = np.asarray(gamma_idx)
    coef = 2.0 / (G.dt * cf[gamma_idx] ** 3)
    acc = np.zeros(len(gamma_idx))

    # TR side: P(m) ~ p(t_(Nt-m)) on Gamma for m = 0, 1, 2, ...
    if history is None:
        layer_idx = np.asarray(layer_idx)
        gs = g / (3.0 * cf[layer_idx] ** 2)                # pressure -> split density
        if tr_box is None:                                 # TR on the whole grid
            GT, c2T, layT, gamT = G, c2, layer_idx, gamma_idx
        else:                                              # TR on a box enclosing Gamma
            GT, cT = tr_grid(G, c, tr_box, pml_alpha)
            c2T = cT * cT
            layT = box_indices(G.shape, tr_box[0], tr_box[1], layer_idx)
            gamT = box_indices(G.shape, tr_box[0], tr_box[1], gamma_idx)
        T = State(GT.shape)
        T.p.reshape(-1)[layT] = g[Nt]                      # initial value on dGamma
        m_done = [0]

        def tr_next():
            m = m_done[0] + 1
            if m > Nt:
                return np.zeros(len(gamma_idx))
            step(GT, T, c2T, dirichlet=(layT, gs[Nt - m]))
            m_done[0] = m
            return T.p.reshape(-1)[gamT].copy()

        p_m0 = T.p.reshape(-1)[gamT].copy()
    else:
        m_done = [0]

        def tr_next():
            m = m_done[0] + 1
            m_done[0] = m
            return history[Nt - m].copy() if m <= Nt else np.zeros(len(gamma_idx))

        p_m0 = history[Nt].copy()

    rec_idx = np.asarray(rec_idx)
    A = State(G.shape)
    p_minus = p_m0                  # P(m)
    p_zero = tr_next()              # P(m+1): the lead TR step
    if pairing == "literal":
        inject = range(1, Nt)          # adjoint step n = 1..Nt-1 injects Q^n
    elif pairing == "exact":
        inject = range(0, Nt + 1)      # adjoint step j = 0..Nt injects Q^j
    else:
        raise ValueError(pairing)
    # The k-th adjoint step (k = 0, 1, ...) is paired with the TR window
    # P(k) - 2 P(k+1) + P(k+2): for the literal loop index n = k + 1 this is
    # p+ - 2 p0 + p- = P(n+1) - 2 P(n) + P(n-1) as printed.
    for qi in inject:
        step(G, A, c2, mass_src=injection_map(G, c, rec_idx, Q[qi]))    # M^T q
        p_plus = tr_next()
        acc += coef * (p_plus - 2.0 * p_zero + p_minus) * A.p.reshape(-1)[gamma_idx]
        p_minus, p_zero = p_zero, p_plus
    grad = np.zeros(G.shape).reshape(-1)
    grad[gamma_idx] = acc
    if c_rec is not None:
        grad *= G.dx * c_rec / 2.0
    return D, grad.reshape(G.shape)


def fwi_gradient(G: Grid, c, src_idx, weights, wavelet, rec_idx, layer_idx, gamma_idx, f_obs,
                 pairing="literal", c_rec=None, full=False, delays=None, tr_box=None, pml_alpha=2.0):
    """Forward + gradient for one encoded super-shot (weights [n_src]; delays [n_src] in
    time steps for the delayed encoding of Eq. 13, f_obs then encoded with the same delays;
    tr_box: TR re-simulation on a box enclosing Gamma, see `gradient`)."""
    if full:
        f, g, hist = forward(G, c, src_idx, weights, wavelet, rec_idx, layer_idx, gamma_idx=gamma_idx,
                             delays=delays)
        return (f,) + gradient(G, c, f, f_obs, rec_idx, layer_idx, gamma_idx, g, pairing,
                               history=hist, c_rec=c_rec)
    f, g = forward(G, c, src_idx, weights, wavelet, rec_idx, layer_idx, delays=delays)
    return (f,) + gradient(G, c, f, f_obs, rec_idx, layer_idx, gamma_idx, g, pairing, c_rec=c_rec,
                           tr_box=tr_box, pml_alpha=pml_alpha)


def grid_for(wl, pml_on=True):
    """Grid of a synthetic workload object (fields nx, ny, nz, dx, dt, c_ref, rho0, pml, pml_alpha)."""
    return Grid(wl.nx, wl.ny, wl.nz, wl.dx, wl.dt, wl.c_ref, wl.rho0,
                wl.pml if pml_on else (0, 0, 0), wl.pml_alpha)
