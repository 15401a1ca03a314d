"""Pins of the FP64 oracle against facts fixed by the paper or by mathematics.

None of these compare the oracle with itself: each checks a closed form, an
invariant, an identity of the discrete scheme, a special case, or a value the
paper prints.  A plausible mistake in the oracle (a sign, a dropped factor, a
wrong shift direction, a wrong time pairing, a transposed axis) fails at least
one of them.
"""
import math
import os

import numpy as np
import pytest
from scipy import special

from oracle import pstd
from paper_2102_00755_b300 import synth

C_REF = 1800.0


@pytest.fixture(autouse=True, scope="module")
def _one_fft_worker():
    """The pins run small grids, where one FFT thread is fastest.  The setting lasts only
    while this module runs (pytest imports every test module before running any), so the
    parity tests' large oracle runs keep every core.  A value set by the caller stands."""
    preset = "ORACLE_WORKERS" in os.environ
    if not preset:
        os.environ["ORACLE_WORKERS"] = "1"
    yield
    if not preset:
        os.environ.pop("ORACLE_WORKERS", None)


def _grid(nx, ny, nz, dx=1e-3, pml=(0, 0, 0)):
    return pstd.Grid(nx, ny, nz, dx, synth.time_step(dx), C_REF, 1000.0, pml, 2.0)


def _kmag_kappa(G):
    k = [pstd.wavenumbers(n, G.dx) for n in (G.nx, G.ny, G.nz)]
    kx, ky, kz = k[0][None, None, :], k[1][None, :, None], k[2][:, None, None]
    km = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    a = G.c_ref * G.dt * km / 2.0
    kap = np.where(a == 0, 1.0, np.sin(a) / np.where(a == 0, 1.0, a))
    return km, kap


# ---------------------------------------------------------------------------
# k-space derivative, App. B (Eqs. 18-19)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(12, 10, 9), (9, 15, 8)])
def test_staggered_derivative_of_plane_wave(shape):
    """d+/dxi cos(k0.x) = -k0_xi kappa(k0) sin(k0.x + k0_xi dx/2), and d- with -dx/2."""
    nx, ny, nz = shape
    G = _grid(nx, ny, nz)
    m0 = (2, -3, 3)
    k0 = [2 * math.pi * m0[a] / (shape[a] * G.dx) for a in range(3)]
    X, Y, Z = synth.coords(shape)
    pos = (X * G.dx, Y * G.dx, Z * G.dx)
    phase = k0[0] * pos[0] + k0[1] * pos[1] + k0[2] * pos[2]
    g = np.cos(phase)
    kap0 = math.sin(G.c_ref * G.dt * math.sqrt(sum(k * k for k in k0)) / 2) / (
        G.c_ref * G.dt * math.sqrt(sum(k * k for k in k0)) / 2)
    assert kap0 < 0.97  # the correction is visible at this wavenumber
    gh = G.fft(g)
    for a in range(3):
        dp = G.deriv(gh, G.d_plus[a])
        dm = G.deriv(gh, G.d_minus[a])
        exp_p = -k0[a] * kap0 * np.sin(phase + k0[a] * G.dx / 2)
        exp_m = -k0[a] * kap0 * np.sin(phase - k0[a] * G.dx / 2)
        scale = abs(k0[a])
        assert np.abs(dp - exp_p).max() < 1e-10 * scale
        assert np.abs(dm - exp_m).max() < 1e-10 * scale


@pytest.mark.parametrize("shape", [(8, 6, 10), (9, 7, 5), (16, 12, 9)])
def test_derivative_adjoint_identity(shape):
    """<D+ a, b> = -<a, D- b> for every axis, even and odd sizes (Nyquist bin kept)."""
    nx, ny, nz = shape
    G = _grid(nx, ny, nz)
    rng = np.random.default_rng(1)
    a = rng.standard_normal(G.shape)
    b = rng.standard_normal(G.shape)
    for ax in range(3):
        lhs = np.sum(G.deriv(G.fft(a), G.d_plus[ax]) * b)
        rhs = -np.sum(a * G.deriv(G.fft(b), G.d_minus[ax]))
        assert abs(lhs - rhs) <= 1e-11 * abs(lhs) + 1e-9


def test_derivative_output_is_real_with_nyquist():
    """The staggered multipliers are Hermitian, so nothing is lost by taking the real part."""
    G = _grid(8, 6, 4)
    g = np.random.default_rng(2).standard_normal(G.shape)
    for ax in range(3):
        full = np.fft.ifftn(G.d_plus[ax] * np.fft.fftn(g))
        assert np.abs(full.imag).max() < 1e-12 * np.abs(full.real).max()


# ---------------------------------------------------------------------------
# Homogeneous propagator, closed form per Fourier mode (App. B: exact for a
# homogeneous medium at c = c_ref)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("c", [1800.0, 1500.0])
def test_homogeneous_closed_form(c):
    """Without PML and with uniform c each Fourier mode obeys
    p_n - 2 cos(th) p_(n-1) + p_(n-2) = c^2 beta (s_n - s_(n-1)) e_src,
    cos(th) = 1 - 2 (c/c_ref)^2 sin^2(c_ref dt |k| / 2), beta = 2 dt / (dx c),
    so p_n = sum_m F_m U_(n-m)(cos th) with Chebyshev polynomials U."""
    G = _grid(10, 12, 9)
    nt = 40
    cc = np.full(G.shape, c)
    src = np.array([3 + 10 * (4 + 12 * 2)])
    s = synth.ricker(nt, G.dt, 0.3e6)
    f, _, fields = pstd.forward(G, cc, src, [1.0], s, np.array([0]), record_field=True)
    km, _ = _kmag_kappa(G)
    a = G.c_ref * G.dt * km / 2
    cos_th = 1.0 - 2.0 * (c / G.c_ref) ** 2 * np.sin(a) ** 2
    e = np.zeros(G.shape)
    e.reshape(-1)[src] = 1.0
    e_hat = np.fft.fftn(e)
    beta = 2.0 * G.dt / (G.dx * c)
    ds = np.diff(np.concatenate([[0.0], s]))
    for n in (0, 1, 5, 17, 39):
        ph = np.zeros(G.shape, dtype=complex)
        for m in range(n + 1):
            ph += c * c * beta * ds[m] * e_hat * special.eval_chebyu(n - m, cos_th)
        p_exact = np.real(np.fft.ifftn(ph))
        ref = np.abs(fields[n]).max()
        assert ref > 0
        assert np.abs(fields[n] - p_exact).max() < 1e-11 * ref, n


@pytest.mark.parametrize("c", [1800.0, 1500.0])
def test_uniform_absorption_closed_form(c):
    """With the PML multiplier Lambda the same at every voxel and on every axis (a uniformly
    absorbing medium), Alg. 1's nesting v <- Lambda (Lambda v - dt/rho0 d+ p), rho <-
    Lambda (Lambda rho - dt rho0 d- v) + source gives, per Fourier mode, the pressure
    after step n as P_n = lam^(n+1) Q_n with lam = Lambda^2, where Q_n obeys the lossless
    recurrence of the closed form above driven by s_n / lam^(n+1) instead of s_n: the
    Lambda factors of the two half-steps cancel in the second difference.  Applying Lambda
    once instead of twice, or adding the source inside the outer multiplication, breaks it."""
    G = _grid(10, 12, 9)
    nt = 40
    Lam = 0.985
    for a in range(3):
        G.lam[a] = np.full_like(G.lam[a], Lam)
        G.lam_s[a] = np.full_like(G.lam_s[a], Lam)
    lam = Lam * Lam
    cc = np.full(G.shape, c)
    src = np.array([3 + 10 * (4 + 12 * 2)])
    s = synth.ricker(nt, G.dt, 0.3e6)
    _, _, fields = pstd.forward(G, cc, src, [1.0], s, np.array([0]), record_field=True)
    km, _ = _kmag_kappa(G)
    a = G.c_ref * G.dt * km / 2
    cos_th = 1.0 - 2.0 * (c / G.c_ref) ** 2 * np.sin(a) ** 2
    e = np.zeros(G.shape)
    e.reshape(-1)[src] = 1.0
    e_hat = np.fft.fftn(e)
    beta = 2.0 * G.dt / (G.dx * c)
    sig = np.asarray(s) / lam ** (np.arange(nt) + 1.0)
    dsig = np.diff(np.concatenate([[0.0], sig]))
    for n in (0, 1, 5, 17, 39):
        qh = np.zeros(G.shape, dtype=complex)
        for m in range(n + 1):
            qh += c * c * beta * dsig[m] * e_hat * special.eval_chebyu(n - m, cos_th)
        p_exact = lam ** (n + 1) * np.real(np.fft.ifftn(qh))
        ref = np.abs(fields[n]).max()
        assert ref > 0
        assert np.abs(fields[n] - p_exact).max() < 1e-11 * ref, n
    # the absorption is visible: the lossless field is larger by lam^-(n+1) at the end
    assert lam ** nt < 0.31


# ---------------------------------------------------------------------------
# Point-source Green's function (physical scale of the source conversion, App. B)
# ---------------------------------------------------------------------------
def test_point_source_greens_function():
    """A point pressure source s converted to a mass source by 2 dt / (3 dx c0)
    per split component is a monopole of mass rate 2 dx^2 s / c0, so in free
    space p(r, t) = dx^2 s'(t - r/c) / (2 pi c r); p_n sits at t_n + dt/2."""
    n, dx, c, f0, nt = 48, 1e-3, 1500.0, 0.15e6, 170
    G = _grid(n, n, n, dx)
    cc = np.full(G.shape, c)
    ctr = n // 2
    src = np.array([ctr + n * (ctr + n * ctr)])
    offs = [(6, 0, 0), (0, 0, -6), (4, 4, 3)]
    recs = np.array([(ctr + o[0]) + n * ((ctr + o[1]) + n * (ctr + o[2])) for o in offs])
    s = synth.ricker(nt, G.dt, f0)
    f, _ = pstd.forward(G, cc, src, [1.0], s, recs)
    t = np.arange(nt) * G.dt + G.dt / 2
    t0 = 1.5 / f0
    for k, o in enumerate(offs):
        r = math.sqrt(sum(x * x for x in o)) * dx
        tau = t - r / c - t0
        ap = 2 * math.pi ** 2 * f0 ** 2 * tau
        a = (math.pi * f0 * tau) ** 2
        sdot = (-2 * ap - (1 - 2 * a) * ap) * np.exp(-a)
        an = dx ** 2 * sdot / (2 * math.pi * c * r)
        rel = np.linalg.norm(f[:, k] - an) / np.linalg.norm(an)
        amp = np.dot(f[:, k], an) / np.dot(an, an)
        assert rel < 0.04, (k, rel)
        assert abs(amp - 1.0) < 0.03, (k, amp)


# ---------------------------------------------------------------------------
# Energy invariant of the leapfrog scheme (PML off) and PML absorption
# ---------------------------------------------------------------------------
def _apply_L(G, p):
    """L p = sum_xi D-_xi D+_xi p = F^-1{ -kappa^2 |k|^2 F p } (closed form of the product)."""
    km, kap = _kmag_kappa(G)
    return np.real(np.fft.ifftn(-(kap ** 2) * km ** 2 * np.fft.fftn(p)))


def test_energy_conserved_without_pml():
    """E_(n+1/2) = sum (p_(n+1) - p_n)^2 / c^2 - dt^2 sum p_(n+1) L p_n is exactly
    conserved once the source is silent (heterogeneous c, W = diag(1/c^2))."""
    G = _grid(12, 10, 11)
    rng = np.random.default_rng(3)
    c = 1500.0 + 200.0 * rng.random(G.shape)
    nt = 60
    s = np.zeros(nt)
    s[:12] = synth.ricker(12, G.dt, 0.4e6, t0=6 * G.dt)
    src = np.array([5 + 12 * (5 + 10 * 5)])
    _, _, fields = pstd.forward(G, c, src, [1.0], s, np.array([0]), record_field=True)
    E = []
    for n in range(14, nt - 1):
        d = fields[n + 1] - fields[n]
        E.append(np.sum(d * d / c ** 2) - G.dt ** 2 * np.sum(fields[n + 1] * _apply_L(G, fields[n])))
    E = np.array(E)
    assert E[0] > 0
    assert np.abs(E - E[0]).max() < 1e-11 * E[0]


def test_pml_profile_properties():
    """Lambda = 1 in the interior, in (0, 1) inside the layer, decreasing towards the edge."""
    n, P = 30, 8
    for stag in (False, True):
        lam = pstd.pml_profile(n, P, 2.0, C_REF, 1e-3, synth.time_step(1e-3), stag)
        assert np.all(lam[P:n - 1 - P] == 1.0)
        assert np.all((lam > 0) & (lam <= 1))
        assert np.all(np.diff(lam[:P + 1]) >= 0) and np.all(np.diff(lam[n - 1 - P:]) <= 0)
        assert lam[0] < 0.9 and lam[-1] < 0.9


def test_pml_absorbs():
    """With the PML on, the field energy left after the pulse has crossed the
    domain is a small fraction of its peak; without it, nothing leaves."""
    out = {}
    for P in (0, 8):
        G = _grid(32, 32, 32, pml=(P, P, P))
        c = np.full(G.shape, 1500.0)
        nt = 150
        s = synth.ricker(nt, G.dt, 0.3e6)
        src = np.array([16 + 32 * (16 + 32 * 16)])
        _, _, fields = pstd.forward(G, c, src, [1.0], s, np.array([0]), record_field=True)
        e = np.array([np.sum(fields[n] ** 2) for n in range(nt)])
        out[P] = e[-1] / e.max()
    assert out[8] < 0.02 and out[0] > 0.2


# ---------------------------------------------------------------------------
# Reciprocity (symmetric W and L): trace(B <- A) c_A = trace(A <- B) c_B
# ---------------------------------------------------------------------------
def test_reciprocity_heterogeneous():
    G = _grid(12, 11, 10)
    rng = np.random.default_rng(4)
    c = 1450.0 + 300.0 * rng.random(G.shape)
    nt = 50
    s = synth.ricker(nt, G.dt, 0.35e6)
    A = 2 + 12 * (3 + 11 * 2)
    B = 9 + 12 * (7 + 11 * 6)
    fa, _ = pstd.forward(G, c, np.array([A]), [1.0], s, np.array([B]))
    fb, _ = pstd.forward(G, c, np.array([B]), [1.0], s, np.array([A]))
    cA, cB = c.reshape(-1)[A], c.reshape(-1)[B]
    assert abs(cA - cB) > 10
    lhs, rhs = fa[:, 0] * cA, fb[:, 0] * cB
    assert np.abs(lhs - rhs).max() < 1e-10 * np.abs(lhs).max()


# ---------------------------------------------------------------------------
# Gradient: finite differences (exact pairing, no PML, layer = Gamma)
# ---------------------------------------------------------------------------
def _smooth_direction(wl, rng):
    X, Y, Z = synth.coords((wl.nx, wl.ny, wl.nz))
    d = np.zeros(wl.shape)
    for _ in range(3):
        kx, ky, kz = rng.integers(0, 3, size=3)
        ph = rng.uniform(0, 2 * math.pi, size=3)
        d += np.cos(2 * math.pi * kx * X / wl.nx + ph[0]) * np.cos(2 * math.pi * ky * Y / wl.ny + ph[1]) \
            * np.cos(2 * math.pi * kz * Z / wl.nz + ph[2])
    m = np.zeros(wl.n_vox)
    m[wl.gamma_idx] = 1.0
    d *= m.reshape(wl.shape)
    return d / np.abs(d).max()


def _misfit(G, wl, c, f_obs):
    f, _ = pstd.forward(G, c, wl.src_idx, wl.weights[0], wl.wavelet, wl.rec_idx)
    return pstd.adjoint_source(f, f_obs)[0]


def test_gradient_matches_finite_differences_exact_pairing():
    """<grad D, delta> equals the central difference of D along smooth directions
    supported in Gamma; transducers sit in water (c = c_rec) outside Gamma."""
    wl = synth.small_workload(14, 13, 12, 70, pml=0, layer=6, n_src=2, n_rec=20, K=1, f0=0.3e6)
    G = pstd.grid_for(wl, pml_on=False)
    gam = np.zeros(wl.n_vox, bool)
    gam[wl.gamma_idx] = True
    assert not gam[wl.src_idx].any() and not gam[wl.rec_idx].any()
    assert len(wl.layer_idx) == len(wl.gamma_idx)            # layer covers Gamma
    assert np.all(wl.c_model.reshape(-1)[wl.rec_idx] == wl.c_rec)
    f_obs, _ = pstd.forward(G, wl.c_true, wl.src_idx, wl.weights[0], wl.wavelet, wl.rec_idx)
    _, D, grad = pstd.fwi_gradient(G, wl.c_model, wl.src_idx, wl.weights[0], wl.wavelet, wl.rec_idx,
                                   wl.layer_idx, wl.gamma_idx, f_obs, pairing="exact", c_rec=wl.c_rec)
    rng = np.random.default_rng(11)
    h = 1e-2
    for _ in range(3):
        d = _smooth_direction(wl, rng)
        fd = (_misfit(G, wl, wl.c_model + h * d, f_obs) - _misfit(G, wl, wl.c_model - h * d, f_obs)) / (2 * h)
        an = float(np.sum(grad * d))
        assert abs(fd) > 0
        assert abs(an - fd) < 1e-6 * abs(fd), (an, fd)


def test_literal_pairing_converges_to_exact():
    """Alg. 1 as printed pairs the adjoint one step later than the exact discrete
    adjoint; the two gradients agree to O(dt): halving dt halves their distance."""
    rel = []
    for refine in (1, 2):
        dx = 1e-3
        dt = synth.time_step(dx) / refine
        nt = 50 * refine
        wl = synth.small_workload(12, 12, 10, nt, pml=0, layer=6, n_src=1, n_rec=16, K=1, f0=0.25e6)
        wl.dt = dt
        wl.wavelet = synth.ricker(nt, dt, 0.25e6)
        G = pstd.grid_for(wl, pml_on=False)
        f_obs, _ = pstd.forward(G, wl.c_true, wl.src_idx, wl.weights[0], wl.wavelet, wl.rec_idx)
        out = {}
        for pairing in ("literal", "exact"):
            out[pairing] = pstd.fwi_gradient(G, wl.c_model, wl.src_idx, wl.weights[0], wl.wavelet,
                                             wl.rec_idx, wl.layer_idx, wl.gamma_idx, f_obs,
                                             pairing=pairing, c_rec=wl.c_rec)[2]
        rel.append(np.linalg.norm(out["literal"] - out["exact"]) / np.linalg.norm(out["exact"]))
    assert rel[0] < 0.5
    assert 1.6 < rel[0] / rel[1] < 2.6, rel


# ---------------------------------------------------------------------------
# Time reversal (Sec. 3.1, Sec. 4.3 / Table 2)
# ---------------------------------------------------------------------------
def test_tr_equals_stored_field_when_layer_covers_gamma():
    wl = synth.small_workload(14, 12, 12, 60, pml=3, layer=6, n_src=2, n_rec=20, K=1)
    assert len(wl.layer_idx) == len(wl.gamma_idx)
    G = pstd.grid_for(wl)
    f_obs, _ = pstd.forward(G, wl.c_true, wl.src_idx, wl.weights[0], wl.wavelet, wl.rec_idx)
    args = (G, wl.c_model, wl.src_idx, wl.weights[0], wl.wavelet, wl.rec_idx, wl.layer_idx,
            wl.gamma_idx, f_obs)
    for pairing in ("literal", "exact"):
        _, D1, g_tr = pstd.fwi_gradient(*args, pairing=pairing)
        _, D2, g_full = pstd.fwi_gradient(*args, pairing=pairing, full=True)
        assert D1 == D2
        assert np.abs(g_tr - g_full).max() < 1e-12 * np.abs(g_full).max()


def test_tr_error_decreases_with_layer_thickness():
    """Like Table 2: the TR gradient approaches the stored-field gradient as the layer thickens."""
    errs = []
    for L in (1, 2):
        wl = synth.small_workload(22, 22, 20, 90, pml=3, layer=L, n_src=2, n_rec=24, K=1, seed=5,
                                  gamma_frac=0.3)
        assert len(wl.layer_idx) < len(wl.gamma_idx)
        G = pstd.grid_for(wl)
        f_obs, _ = pstd.forward(G, wl.c_true, wl.src_idx, wl.weights[0], wl.wavelet, wl.rec_idx)
        args = (G, wl.c_model, wl.src_idx, wl.weights[0], wl.wavelet, wl.rec_idx, wl.layer_idx,
                wl.gamma_idx, f_obs)
        g_tr = pstd.fwi_gradient(*args)[2]
        g_full = pstd.fwi_gradient(*args, full=True)[2]
        errs.append(np.linalg.norm(g_tr - g_full) / np.linalg.norm(g_full))
    assert errs[1] < 0.5 * errs[0], errs


# TR re-simulation on a box enclosing Gamma (Sec. 3.1)
def _tr_box_case():
    wl = synth.small_workload(36, 36, 30, 90, pml=4, n_src=3, n_rec=30, K=1, layer=3, seed=5, f0=0.4e6,
                              gamma_frac=0.25)
    G = pstd.grid_for(wl)
    w = wl.weights[0]
    f_obs = pstd.forward(G, wl.c_true, wl.src_idx, w, wl.wavelet, wl.rec_idx)[0]
    f, g, hist = pstd.forward(G, wl.c_model, wl.src_idx, w, wl.wavelet, wl.rec_idx, wl.layer_idx,
                              gamma_idx=wl.gamma_idx)

    def grad(**kw):
        return pstd.gradient(G, wl.c_model, f, f_obs, wl.rec_idx, wl.layer_idx, wl.gamma_idx, g,
                             c_rec=wl.c_rec, **kw)[1]
    return wl, grad, hist


def test_tr_box_covering_the_grid_is_the_whole_grid_tr():
    """A box equal to the grid, with the grid's PML, is the whole-grid TR bit for bit
    (the cropping and index mapping are the identity)."""
    wl, grad, _ = _tr_box_case()
    box = ((0, 0, 0), (wl.nx, wl.ny, wl.nz), wl.pml)
    assert np.array_equal(grad(tr_box=box), grad())


def test_tr_box_equals_stored_field_when_layer_covers_gamma():
    """With the boundary layer covering all of Gamma the TR values on Gamma are the imposed
    forward values, on any box: the box gradient equals the stored-field gradient.  A wrong
    mapping of the layer or Gamma into the box breaks this."""
    wl = synth.small_workload(20, 20, 18, 60, pml=3, layer=6, n_src=2, n_rec=20, K=1, seed=3)
    assert len(wl.layer_idx) == len(wl.gamma_idx)
    G = pstd.grid_for(wl)
    f_obs, _ = pstd.forward(G, wl.c_true, wl.src_idx, wl.weights[0], wl.wavelet, wl.rec_idx)
    args = (G, wl.c_model, wl.src_idx, wl.weights[0], wl.wavelet, wl.rec_idx, wl.layer_idx,
            wl.gamma_idx, f_obs)
    box = synth.tr_box(wl, 1, 2)
    assert box[1] != (wl.nx, wl.ny, wl.nz) and box[0] != (0, 0, 0)
    for pairing in ("literal", "exact"):
        _, D1, g_box = pstd.fwi_gradient(*args, pairing=pairing, tr_box=box)
        _, D2, g_full = pstd.fwi_gradient(*args, pairing=pairing, full=True)
        assert D1 == D2
        assert np.abs(g_box - g_full).max() < 1e-12 * np.abs(g_full).max()


def test_tr_box_converges_to_whole_grid_tr_as_margin_grows():
    """The box only changes what lies outside the boundary layer; the non-local k-space
    operator feels it across the layer.  Growing the margin between Gamma and the box's PML
    brings the box gradient monotonically closer to the whole-grid TR gradient, and its
    error against the stored-field gradient stays that of the whole-grid TR."""
    wl, grad, hist = _tr_box_case()
    g_tr = grad()
    g_full = grad(history=hist)
    e_tr = np.linalg.norm(g_tr - g_full) / np.linalg.norm(g_full)
    diffs = []
    for m in (0, 2, 4, 6):
        box = synth.tr_box(wl, m, 3)
        g_box = grad(tr_box=box)
        diffs.append(np.linalg.norm(g_box - g_tr) / np.linalg.norm(g_tr))
        e_box = np.linalg.norm(g_box - g_full) / np.linalg.norm(g_full)
        assert abs(e_box - e_tr) < 0.05 * e_tr, (m, e_box, e_tr)
    assert all(b < a for a, b in zip(diffs, diffs[1:])), diffs
    assert diffs[-1] < 0.01


# ---------------------------------------------------------------------------
# Source encoding (Sec. 3.2, App. E)
# ---------------------------------------------------------------------------
def test_encoded_forward_is_linear():
    wl = synth.small_workload(12, 10, 10, 40, pml=3, n_src=3, n_rec=12, K=1)
    G = pstd.grid_for(wl)
    w = np.array([1.0, -1.0, 1.0])
    f_enc, g_enc = pstd.forward(G, wl.c_model, wl.src_idx, w, wl.wavelet, wl.rec_idx, wl.layer_idx)
    f_sum = 0
    g_sum = 0
    for i in range(3):
        e = np.zeros(3)
        e[i] = 1.0
        fi, gi = pstd.forward(G, wl.c_model, wl.src_idx, e, wl.wavelet, wl.rec_idx, wl.layer_idx)
        f_sum = f_sum + w[i] * fi
        g_sum = g_sum + w[i] * gi
    assert np.abs(f_enc - f_sum).max() < 1e-12 * np.abs(f_enc).max()
    assert np.abs(g_enc - g_sum).max() < 1e-12 * np.abs(g_enc).max()


def test_encoding_unbiased_over_all_sign_patterns():
    """E[w_i w_j] = delta_ij: the mean of the encoded gradient over all 2^3 Rademacher
    patterns equals the sum of the single-source gradients (App. E)."""
    wl = synth.small_workload(12, 11, 10, 40, pml=3, n_src=3, n_rec=14, K=1, layer=1)
    G = pstd.grid_for(wl)
    f_i = []
    for i in range(3):
        e = np.zeros(3)
        e[i] = 1.0
        f_i.append(pstd.forward(G, wl.c_true, wl.src_idx, e, wl.wavelet, wl.rec_idx)[0])
    f_i = np.stack(f_i)

    def grad_for(w):
        f_obs = pstd.encode_data(w, f_i)
        return pstd.fwi_gradient(G, wl.c_model, wl.src_idx, w, wl.wavelet, wl.rec_idx,
                                 wl.layer_idx, wl.gamma_idx, f_obs)

    total = 0
    for i in range(3):
        e = np.zeros(3)
        e[i] = 1.0
        total = total + grad_for(e)[2]
    mean = 0
    Dmean = 0
    for bits in range(8):
        w = np.array([1.0 if (bits >> i) & 1 else -1.0 for i in range(3)])
        _, D, g = grad_for(w)
        mean = mean + g / 8
        Dmean += D / 8
    assert np.abs(mean - total).max() < 1e-10 * np.abs(total).max()
    Dsum = sum(grad_for(np.eye(3)[i])[1] for i in range(3))
    assert abs(Dmean - Dsum) < 1e-10 * Dsum


def test_adjoint_source_definitions():
    """q^n = f^(Nt-n) - f_obs^(Nt-n), D = 0.5 sum q^2, Q^n = sum_(m<=n) q^m (Alg. 1)."""
    rng = np.random.default_rng(5)
    f = rng.standard_normal((7, 3))
    fo = rng.standard_normal((7, 3))
    D, Q = pstd.adjoint_source(f, fo)
    Nt = 6
    acc = np.zeros(3)
    tot = 0.0
    for n in range(7):
        q = f[Nt - n] - fo[Nt - n]
        tot += 0.5 * float(q @ q)
        acc = acc + q
        assert np.allclose(Q[n], acc, rtol=0, atol=1e-14)
    assert abs(D - tot) < 1e-13


# ---------------------------------------------------------------------------
# Values the paper prints (tests/golden/paper_setup.txt)
# ---------------------------------------------------------------------------
def _golden():
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_setup.txt")
    vals = {}
    with open(path) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split()
                vals[k] = float(v)
    return vals


def test_paper_time_step():
    g = _golden()
    dt = synth.time_step(g["dx_m"], g["c_max"], g["cfl"])
    assert round(dt * 1e9, 1) == g["dt_ns"]


def test_paper_grid_and_pml_rule():
    """221 x 221 x 111 mm at 0.5 mm is 442 x 442 x 222 voxels (Sec. 4.1); the App. B
    PML rule (10..20 cells, smallest largest prime factor) pads it to FFT-friendly sizes."""
    g = _golden()
    n = [int(round(g[k] / g["dx_mm"])) for k in ("domain_x_mm", "domain_y_mm", "domain_z_mm")]
    assert n == [int(g["nx"]), int(g["ny"]), int(g["nz"])]
    for m in n:
        P = synth.optimal_pml(m)
        assert 10 <= P <= 20
        tot = m + 2 * P
        for p in (7, 11, 13, 17, 19, 23, 29, 31, 37, 41, 43, 47):
            assert tot % p != 0


# ---------------------------------------------------------------------------
# Closed-form traces used for full-size parity (App. B, homogeneous medium)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape,c", [((12, 10, 9), 1800.0), ((9, 15, 8), 1500.0), ((16, 16, 12), 1800.0)])
def test_closed_form_traces_match_time_stepping(shape, c):
    """The per-mode recurrence summed at receiver offsets (half spectrum in x, with
    wrap-around offsets) equals the oracle's time-stepping forward traces."""
    from oracle import closed_form
    nx, ny, nz = shape
    G = _grid(nx, ny, nz)
    nt = 60
    rng = np.random.default_rng(5)
    src = int(rng.integers(0, nx * ny * nz))
    rec = rng.choice(nx * ny * nz, size=7, replace=False)
    s = synth.ricker(nt, G.dt, 0.3e6)
    f, _ = pstd.forward(G, np.full(G.shape, c), np.array([src]), [1.0], s, rec)
    cf = closed_form.homogeneous_traces(shape, G.dx, G.dt, C_REF, c, src, rec, s, nt)
    assert np.abs(f).max() > 0
    assert np.abs(cf - f).max() < 1e-11 * np.abs(f).max()


# ---------------------------------------------------------------------------
# Delayed source encoding (Eq. 13, App. D): whole-step delays
# ---------------------------------------------------------------------------
def _delay_setup():
    G = _grid(12, 10, 9)
    nt = 50
    rng = np.random.default_rng(8)
    c = 1500.0 + 40.0 * rng.random(G.shape)
    src = np.array([5 + 12 * (4 + 10 * 4), 2 + 12 * (7 + 10 * 2), 9 + 12 * (1 + 10 * 6)])
    rec = rng.choice(12 * 10 * 9, size=6, replace=False)
    s = synth.ricker(nt, G.dt, 0.4e6)
    return G, nt, c, src, rec, s


def test_delayed_source_emits_later():
    """One source delayed by d steps: s(t - d dt) gives the undelayed traces d samples later,
    and exact zeros before (the field starts from rest)."""
    G, nt, c, src, rec, s = _delay_setup()
    f0, _ = pstd.forward(G, c, src[:1], [1.0], s, rec)
    f7, _ = pstd.forward(G, c, src[:1], [1.0], s, rec, delays=[7])
    assert np.all(f7[:7] == 0.0)
    assert np.abs(f0).max() > 0
    assert np.abs(f7[7:] - f0[:-7]).max() < 1e-12 * np.abs(f0).max()


def test_delayed_encoding_is_shifted_superposition():
    """p_hat(t) = sum_i w_i p_i(t - d_i tau) by linearity and time invariance (App. D)."""
    G, nt, c, src, rec, s = _delay_setup()
    w = np.array([1.0, -1.0, 1.0])
    d = np.array([0, 5, 11])
    f_hat, _ = pstd.forward(G, c, src, w, s, rec, delays=d)
    ref = np.zeros_like(f_hat)
    for i in range(3):
        fi, _ = pstd.forward(G, c, src[i:i + 1], [1.0], s, rec)
        ref[d[i]:] += w[i] * fi[:nt - d[i]]
    assert np.abs(f_hat - ref).max() < 1e-12 * np.abs(ref).max()


def test_zero_delays_are_conventional_encoding():
    G, nt, c, src, rec, s = _delay_setup()
    w = np.array([1.0, -1.0, -1.0])
    fa, _ = pstd.forward(G, c, src, w, s, rec)
    fb, _ = pstd.forward(G, c, src, w, s, rec, delays=[0, 0, 0])
    assert np.abs(fa - fb).max() < 1e-13 * np.abs(fa).max()


def test_delayed_data_encoding_closed_form():
    """data_i[n][r] = (i + 1)(n + 1) + r: f_hat[n][r] = sum over sources with
    0 <= n - d_i < nt_data of w_i ((i + 1)(n - d_i + 1) + r)."""
    n_src, nt_d, n_rec, nt = 3, 6, 2, 10
    data = np.array([[[(i + 1) * (n + 1) + r for r in range(n_rec)] for n in range(nt_d)] for i in range(n_src)],
                    dtype=float)
    w, d = [1.0, -1.0, 1.0], [0, 2, 5]
    out = pstd.encode_data(w, data, delays=d, nt=nt)
    assert out.shape == (nt, n_rec)
    # n = 7: source 0 has ended (7 >= 6), source 1 at 5: -(2*6 + r), source 2 at 2: 3*3 + r
    assert list(out[7]) == [-12.0 + 9.0, -13.0 + 10.0]
    # n = 0: only source 0: 1*1 + r
    assert list(out[0]) == [1.0, 2.0]
    assert np.allclose(pstd.encode_data(w, data), pstd.encode_data(w, data, delays=[0, 0, 0]))


# ---------------------------------------------------------------------------
# Stochastic L-BFGS (Alg. 2)
# ---------------------------------------------------------------------------
def _spd(n, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return Q @ np.diag(np.linspace(1.0, 20.0, n)) @ Q.T, rng.standard_normal(n)


def test_two_loop_secant_condition():
    """Secant condition of the BFGS update: after each new pair (s, y), H y = s for that
    pair, whatever the earlier pairs and the initial scaling."""
    from oracle import slbfgs
    A, _ = _spd(8, 1)
    rng = np.random.default_rng(2)
    S, Y = [], []
    for k in range(8):
        s = rng.standard_normal(8)
        assert slbfgs.push_pair(S, Y, s, A @ s, 64)
        h = slbfgs.two_loop(Y[-1], S, Y, 0.7)
        assert np.allclose(h, S[-1], rtol=1e-10, atol=1e-12)


def test_two_loop_equals_dense_bfgs_update():
    """The two-loop recursion equals the dense BFGS inverse update
    H+ = (I - rho s y') H (I - rho y s') + rho s s' applied pair by pair from h0 I."""
    from oracle import slbfgs
    A, g = _spd(6, 3)
    rng = np.random.default_rng(4)
    S, Y = [], []
    H = 0.3 * np.eye(6)
    for _ in range(4):
        s = rng.standard_normal(6)
        y = A @ s
        slbfgs.push_pair(S, Y, s, y, 64)
        rho = 1.0 / (y @ s)
        V = np.eye(6) - rho * np.outer(y, s)
        H = V.T @ H @ V + rho * np.outer(s, s)
    assert np.allclose(slbfgs.two_loop(g, S, Y, 0.3), H @ g, rtol=1e-10, atol=1e-12)


def test_history_limit_and_curvature_skip():
    from oracle import slbfgs
    S, Y = [], []
    for k in range(5):
        slbfgs.push_pair(S, Y, np.array([1.0, k]), np.array([1.0, 0.5]), 3)
    assert len(S) == 3 and S[0][1] == 2.0
    assert not slbfgs.push_pair(S, Y, np.array([1.0, 0.0]), np.array([-1.0, 0.0]), 3)
    assert len(S) == 3


def test_slbfgs_exact_gradients_reach_quadratic_minimum():
    """theta = 0 (exact energy and gradient): the iterates converge to A^-1 b."""
    from oracle import slbfgs
    A, b = _spd(10, 5)
    est = lambda u, th, n: (0.5 * u @ A @ u - b @ u, A @ u - b)
    u_hat, Js, _ = slbfgs.slbfgs(np.zeros(10), est, nu=1.0, n_evl=60, m=64)
    assert np.linalg.norm(u_hat - np.linalg.solve(A, b)) < 1e-8 * np.linalg.norm(np.linalg.solve(A, b))


def test_slbfgs_projection_and_averaging():
    """Bounds are enforced after every step, and after the first energy increase the
    returned estimate is the w(i) = i^3 weighted mean of the later iterates."""
    from oracle import slbfgs
    rng = np.random.default_rng(6)
    A, b = _spd(5, 7)
    def est(u, th, n):               # noisy gradient, same noise for the same n
        e = np.random.default_rng(n).standard_normal(5)
        return 0.5 * u @ A @ u - b @ u + 0.1 * (e @ u), A @ u - b + 0.1 * e
    u_hat, Js, us = slbfgs.slbfgs(rng.standard_normal(5), est, nu=0.5, n_evl=40, m=8, u_min=-0.2, u_max=0.2)
    assert all(np.all(u >= -0.2) and np.all(u <= 0.2) for u in us)
    first = next(i for i in range(1, len(Js)) if Js[i] > Js[i - 1])     # 0-based iteration index
    idx = range(first + 1, len(us))
    w = np.array([(i + 1) ** 3 for i in idx], dtype=float)
    assert np.allclose(u_hat, sum(wi * us[i] for wi, i in zip(w, idx)) / w.sum())


# ---------------------------------------------------------------------------
# Grid transfers of the coarse-to-fine scheme (Sec. 3.3, App. C)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n_in,n_out,kind", [(11, 21, "blackman"), (21, 11, "kaiser"), (16, 33, "none"),
                                              (24, 16, "none"), (9, 9, "blackman")])
def test_resampling_matches_trigonometric_sum(n_in, n_out, kind):
    """The FFT evaluation equals the brute-force windowed trigonometric sum."""
    from oracle import multigrid
    u = np.random.default_rng(n_in * 31 + n_out).standard_normal(n_in)
    fast = multigrid.resample_1d(u, n_out, 0, kind)
    slow = multigrid.trig_sum(u, n_out, kind)
    assert np.allclose(fast, slow, rtol=1e-12, atol=1e-12)


def test_fourier_interpolation_is_exact_for_band_limited_signals():
    """Rectangular window: a trigonometric polynomial inside the band is reproduced exactly
    at the fine sample positions, in 3D and for odd and even sizes."""
    from oracle import multigrid
    def f(shape, scale):
        z, y, x = np.meshgrid(*[np.arange(n) * scale[a] for a, n in enumerate(shape)], indexing="ij")
        return (1.0 + np.cos(2 * np.pi * 2 * x / shape[2] / scale[2]) * np.sin(2 * np.pi * 1 * y / shape[1] / scale[1])
                + 0.5 * np.cos(2 * np.pi * 3 * z / shape[0] / scale[0] + 0.3))
    shape_c, shape_f = (9, 12, 11), (17, 24, 21)
    uc = f(shape_c, (1.0, 1.0, 1.0))
    uf = f(shape_f, tuple(c / n for c, n in zip(shape_c, shape_f)))
    assert np.allclose(multigrid.resample(uc, shape_f, "none"), uf, atol=1e-12)


def test_windows_dc_gain_and_attenuation():
    """DC is kept (w(0) = 1), a pure cosine of band index k comes out scaled by w(k),
    and a component beyond the coarse band is removed by down-sampling."""
    from oracle import multigrid
    n = 40
    t = np.arange(n)
    for kind in ("blackman", "kaiser"):
        K = multigrid.band(n, 80)
        w = multigrid.window(kind, K)
        assert abs(w[0] - 1.0) < 1e-15
        k = 5
        out = multigrid.resample_1d(3.0 + np.cos(2 * np.pi * k * t / n), 80, 0, kind)
        ref = 3.0 + w[k] * np.cos(2 * np.pi * k * np.arange(80) / 80)
        assert np.allclose(out, ref, atol=1e-12)
    hi = np.cos(2 * np.pi * 15 * t / n)            # above the band of a 20-sample output
    assert np.abs(multigrid.downsample_series(hi, 20, 0)).max() < 1e-12


def test_data_scaling_eta():
    from oracle import multigrid
    x = np.ones(30)
    assert np.allclose(multigrid.downsample_series(x, 15, 0, eta=2.0), 4.0)
