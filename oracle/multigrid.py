"""Grid transfers of the coarse-to-fine scheme (Sec. 3.3, App. C) in plain FP64 numpy.

TEST INFRASTRUCTURE ONLY.  Only the test-suite may import this module; the
product path (fwi_resample in the CUDA library) never does.

App. C transfers fields between grids by Fourier (trigonometric) interpolation
with smoothing in Fourier space: the model is up-sampled with a Blackman window,
time series (observed data, source signals) are down-sampled with a Kaiser-window
low-pass filter, and down-sampled data are scaled by eta^(d-1).  Readings where
App. C names a routine instead of a formula (all listed in the design notes):

* every transfer is separable periodic Fourier resampling along each axis: the
  output sample i is the windowed trigonometric interpolant of the input at
  t = i N_in / N_out (same period, Matlab interpft / interpftn semantics);
* the band is |k| <= K = floor((min(N_in, N_out) - 1) / 2) (the Nyquist bins are
  dropped, which keeps the operator real);
* Blackman window w(k) = 0.42 + 0.5 cos(pi k / (K+1)) + 0.08 cos(2 pi k / (K+1)),
  equal to 1 at k = 0 and 0 just beyond the band;
* Kaiser window w(k) = I0(beta sqrt(1 - (k / (K+1))^2)) / I0(beta), beta = 4;
* rectangular window w = 1 (plain Fourier interpolation).

The oracle evaluates the resampling with FFTs (zero-padding or truncating the
windowed spectrum, inverse transform at N_out, scaled by N_out / N_in); it is
pinned against the brute-force trigonometric sum.
"""
from __future__ import annotations

import math

import numpy as np

WINDOWS = {"none": 0, "blackman": 1, "kaiser": 2}


def band(n_in: int, n_out: int) -> int:
    return (min(n_in, n_out) - 1) // 2


def window(kind: str, K: int, beta: float = 4.0) -> np.ndarray:
    """w(k) for k = 0..K (the window is even in k)."""
    k = np.arange(K + 1, dtype=np.float64)
    if kind == "none":
        return np.ones(K + 1)
    if kind == "blackman":
        a = np.pi * k / (K + 1)
        return 0.42 + 0.5 * np.cos(a) + 0.08 * np.cos(2.0 * a)
    if kind == "kaiser":
        r = k / (K + 1)
        return np.i0(beta * np.sqrt(1.0 - r * r)) / np.i0(beta)
    raise ValueError(kind)


def resample_1d(u: np.ndarray, n_out: int, axis: int, kind: str = "none", beta: float = 4.0) -> np.ndarray:
    """Periodic Fourier resampling of u along `axis` to n_out samples (see module)."""
    u = np.moveaxis(np.asarray(u, dtype=np.float64), axis, -1)
    n_in = u.shape[-1]
    K = band(n_in, n_out)
    w = window(kind, K, beta)
    U = np.fft.fft(u, axis=-1)
    V = np.zeros(u.shape[:-1] + (n_out,), dtype=np.complex128)
    V[..., 0] = w[0] * U[..., 0]
    for k in range(1, K + 1):
        V[..., k] = w[k] * U[..., k]
        V[..., n_out - k] = w[k] * U[..., n_in - k]
    out = np.real(np.fft.ifft(V, axis=-1)) * (n_out / n_in)
    return np.moveaxis(out, -1, axis)


def resample(u: np.ndarray, shape_out, kind: str = "none", beta: float = 4.0) -> np.ndarray:
    """Separable resampling of an array [..] to shape_out, axis by axis."""
    out = np.asarray(u, dtype=np.float64)
    for ax, n in enumerate(shape_out):
        if out.shape[ax] != n or kind != "none":
            out = resample_1d(out, n, ax, kind, beta)
    return out


def upsample_model(u_coarse: np.ndarray, shape_fine) -> np.ndarray:
    """u_f = Fourier interpolation of u_c with Blackman smoothing (App. C)."""
    return resample(u_coarse, shape_fine, "blackman")


def downsample_series(x: np.ndarray, n_out: int, axis: int, eta: float = None, d: int = 3,
                      beta: float = 4.0) -> np.ndarray:
    """Time series to a coarser time grid: Kaiser-windowed Fourier resampling; if eta is
    given the result is scaled by eta^(d-1), as App. C requires for the data."""
    y = resample_1d(x, n_out, axis, "kaiser", beta)
    return y * eta ** (d - 1) if eta is not None else y


def trig_sum(u: np.ndarray, n_out: int, kind: str = "none", beta: float = 4.0) -> np.ndarray:
    """Brute force for a 1D signal: sum over the band of w(k) U_k exp(2 pi i k t / N_in) / N_in
    at t = i N_in / N_out (the definition the FFT evaluation must match)."""
    u = np.asarray(u, dtype=np.float64)
    n_in = len(u)
    K = band(n_in, n_out)
    w = window(kind, K, beta)
    j = np.arange(n_in)
    out = np.zeros(n_out)
    for i in range(n_out):
        t = i * n_in / n_out
        s = w[0] * u.sum()
        for k in range(1, K + 1):
            Uk = np.sum(u * np.exp(-2j * math.pi * k * j / n_in))
            s += 2.0 * w[k] * np.real(Uk * np.exp(2j * math.pi * k * t / n_in))
        out[i] = s / n_in
    return out
