"""Host-side checks of the C ABI: the library loads, exports every entry point that
include/fwi.h declares, and rejects bad problems at plan creation (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2102_00755_b300 import build as fbuild
from paper_2102_00755_b300 import fwi, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    fbuild.build()
    return fwi.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "fwi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fwi_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(L):
    names = _declared()
    assert len(names) >= 9
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(fwi.C_SYMBOLS)


def test_status_strings(L):
    for s in range(8):
        assert fwi.fwi_status_string(s)
    assert "unstable" in fwi.fwi_status_string(fwi.FWI_EUNSTABLE)


def _problem(wl, **over):
    keep = [np.ascontiguousarray(a, dtype=np.int32) for a in (wl.src_idx, wl.rec_idx, wl.layer_idx, wl.gamma_idx)]
    wav = np.ascontiguousarray(wl.wavelet, dtype=np.float32)
    P = fwi.fwi_problem()
    P.nx, P.ny, P.nz = wl.nx, wl.ny, wl.nz
    P.pml[0], P.pml[1], P.pml[2] = wl.pml
    P.dx, P.dt, P.c_ref, P.rho0, P.pml_alpha, P.c_rec = wl.dx, wl.dt, wl.c_ref, wl.rho0, wl.pml_alpha, 0.0
    P.nt, P.n_src, P.n_rec, P.n_layer, P.n_gamma = wl.nt, *[len(k) for k in keep]
    ip = ctypes.POINTER(ctypes.c_int32)
    P.src_idx, P.rec_idx, P.layer_idx, P.gamma_idx = [k.ctypes.data_as(ip) for k in keep]
    P.wavelet = wav.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    P.pairing, P.max_shots, P.sims_per_launch = 0, 2, 0
    for k, v in over.items():
        setattr(P, k, v)
    return P, (keep, wav)


def test_plan_create_reports_workspace(L):
    wl = synth.small_workload(24, 20, 18, 40)
    P, keep = _problem(wl)
    st, plan, nbytes = fwi.fwi_plan_create(P)
    assert st == fwi.FWI_OK and nbytes > 0
    N = wl.n_vox
    assert nbytes > 2 * 2 * 6 * N * 4          # 2K simulation states of six fields at least
    assert fwi.fwi_plan_voxel_steps(plan, 2, 1) == 2 * N * (3 * wl.nt - 3)
    assert fwi.fwi_plan_voxel_steps(plan, 1, 0) == N * wl.nt
    fwi.fwi_plan_destroy(plan)


@pytest.mark.parametrize("field,value", [
    ("nx", 1), ("nt", 2), ("max_shots", 0), ("max_shots", 9), ("dx", 0.0), ("pairing", 5),
    ("c_rec", -1.0)])
def test_plan_create_rejects_bad_scalars(L, field, value):
    wl = synth.small_workload(24, 20, 18, 40)
    P, keep = _problem(wl, **{field: value})
    st, plan, _ = fwi.fwi_plan_create(P)
    assert st == fwi.FWI_EINVAL


def test_plan_create_rejects_bad_lists(L):
    wl = synth.small_workload(24, 20, 18, 40)
    bad = synth.Workload(**{**wl.__dict__})
    bad.rec_idx = wl.rec_idx.copy()
    bad.rec_idx[0] = wl.n_vox          # out of range
    P, keep = _problem(bad)
    assert fwi.fwi_plan_create(P)[0] == fwi.FWI_EINVAL
    bad = synth.Workload(**{**wl.__dict__})
    bad.gamma_idx = wl.gamma_idx[::-1].copy()   # not increasing
    P, keep = _problem(bad)
    assert fwi.fwi_plan_create(P)[0] == fwi.FWI_EINVAL
    bad = synth.Workload(**{**wl.__dict__})
    bad.layer_idx = np.array([wl.src_idx[0]], np.int32)   # layer voxel outside Gamma
    P, keep = _problem(bad)
    assert fwi.fwi_plan_create(P)[0] == fwi.FWI_EINVAL


def test_plan_create_rejects_unsupported_sizes(L):
    wl = synth.small_workload(24, 20, 18, 40)
    P, keep = _problem(wl, nx=21)        # 21 = 3 * 7: prime factor 7
    # keep indices valid for the smaller grid
    st, plan, _ = fwi.fwi_plan_create(P)
    assert st in (fwi.FWI_ENOTSUP, fwi.FWI_EINVAL)


def test_binding_fails_loudly_without_library(monkeypatch):
    monkeypatch.setattr(fwi, "_lib", None)
    monkeypatch.setattr(fwi, "LIB_PATH", "/nonexistent/libfwi.so")
    with pytest.raises(ImportError):
        fwi.lib()


def test_tr_box_validation_and_workspace(L):
    """fwi_plan_set_tr_box (Sec. 3.1's TR on a box enclosing Gamma) checks the box on the
    host and reports the new workspace size: the whole-grid TR states go, the box plan's
    workspace and the cropped c0 come in.  No device memory is touched."""
    wl = synth.small_workload(36, 36, 30, 40, pml=4, n_src=3, n_rec=30, K=2, layer=3, seed=5, gamma_frac=0.25)
    P, keep = _problem(wl)
    st, plan, nbytes = fwi.fwi_plan_create(P)
    assert st == fwi.FWI_OK
    origin, size, pml = synth.tr_box(wl, 2, 3)
    st, nb_box = fwi.fwi_plan_set_tr_box(plan, origin, size, pml)
    assert st == fwi.FWI_OK
    state = 2 * 6 * wl.n_vox * 4                    # K = 2 whole-grid TR states of six fields
    assert nb_box < nbytes - state // 2
    assert fwi.fwi_plan_voxel_steps(plan, 2, 1) == 2 * ((2 * wl.nt - 2) * wl.n_vox +
                                                      (wl.nt - 1) * size[0] * size[1] * size[2])
    # calling again replaces the box; the grid itself is a valid box
    st, nb_full = fwi.fwi_plan_set_tr_box(plan, (0, 0, 0), (wl.nx, wl.ny, wl.nz), wl.pml)
    assert st == fwi.FWI_OK and nb_full > nb_box
    bad = [((30, 0, 0), size, pml),                 # box leaves the grid
           (origin, size, (9, 9, 9)),               # Gamma inside the box's PML
           ((0, 0, 0), (12, 12, 12), pml),          # Gamma outside the box
           (origin, size, (-1, 3, 3))]
    for o, s, p in bad:
        assert fwi.fwi_plan_set_tr_box(plan, o, s, p)[0] == fwi.FWI_EINVAL, (o, s, p)
    fwi.fwi_plan_destroy(plan)


def test_per_shot_models_validation_and_workspace(L):
    """per_shot_models = 1 keeps one c0^2 field and one set of sparse coefficients per
    super-shot (K of them); any other value than 0 or 1 is rejected."""
    wl = synth.small_workload(24, 20, 18, 40)
    P, keep = _problem(wl)
    st, plan, one = fwi.fwi_plan_create(P)
    assert st == fwi.FWI_OK
    fwi.fwi_plan_destroy(plan)
    P, keep = _problem(wl, per_shot_models=1)
    st, plan, each = fwi.fwi_plan_create(P)
    assert st == fwi.FWI_OK
    assert each - one >= (P.max_shots - 1) * wl.n_vox * 4      # the extra c0^2 fields at least
    fwi.fwi_plan_destroy(plan)
    P, keep = _problem(wl, per_shot_models=2)
    assert fwi.fwi_plan_create(P)[0] == fwi.FWI_EINVAL


def test_launch_count_follows_the_schedule(L):
    """fwi_plan_launches (the bench's gpu_launches claim) from the host: per time step 4
    launches per stream group (8 with split planes); the two-step kernels add the gradient
    term inside the mass kernel, the warp-owned kernels need one accumulation launch per
    iteration; a TR box adds its crop and preparation."""
    import ctypes as C
    wl = synth.small_workload(32, 32, 32, 40, pml=4, n_src=3, n_rec=24, K=4, layer=2, gamma_frac=0.25)
    P, keep = _problem(wl, max_shots=4)
    st, plan, _ = fwi.fwi_plan_create(P)
    assert st == fwi.FWI_OK

    def launches(**sched):
        s = fwi.fwi_schedule(sched.get("specialized", 2), 0, 32, sched.get("split_plane", 0),
                             sched.get("stream_groups", 1))
        assert L.fwi_plan_set_schedule(plan, C.byref(s)) == fwi.FWI_OK
        return fwi.fwi_plan_launches(plan, 4, 0), fwi.fwi_plan_launches(plan, 4, 1)

    nt = wl.nt
    f1, g1 = launches(stream_groups=1)
    f4, g4 = launches(stream_groups=4)
    assert f1 == 3 + 4 * nt and f4 == 3 + 4 * 4 * nt
    # backward with one group: misfit x2, TR init, lead step, (nt - 2) iterations of 4, one final
    # accumulation, the scatter (two-step kernels: no per-iteration accumulation)
    assert g1 - f1 == 2 + 1 + 4 + 4 * (nt - 2) + 1 + 1
    fw, gw = launches(specialized=1, stream_groups=1)          # warp-owned kernels
    assert fw == f1 and gw - g1 == (nt - 2) - 1
    st, _ = fwi.fwi_plan_set_tr_box(plan, *synth.tr_box(wl, 1, 2))
    assert st == fwi.FWI_OK
    fb, gb = launches(stream_groups=1)
    assert fb == f1 and gb - g1 == 3 + 4 * (nt - 2)            # crop + prepare x2, separate TR launches
    fwi.fwi_plan_destroy(plan)


def test_plan_create_survives_malformed_problems(L):
    """Host validation under random problems, valid ones with up to two corruptions (a bad
    size, count, scalar, enum, an index out of range, an unsorted Gamma, a layer voxel
    outside Gamma): every answer is a defined status, nothing crashes, and an accepted
    problem gives a plan whose workspace size, voxel-step and launch counts and TR-box
    validation can be queried (no GPU needed)."""
    from hypothesis import HealthCheck, given, settings
    from hypothesis import strategies as st

    statuses = {fwi.FWI_OK, fwi.FWI_EINVAL, fwi.FWI_ENOMEM, fwi.FWI_ENOTSUP}
    sizes = st.sampled_from([2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 14, 15, 16, 20])
    corruptions = ["nx", "nt", "pml", "max_shots", "pairing", "spl", "psm", "dx", "dt", "c_ref",
                   "src_range", "rec_range", "gamma_order", "layer_outside", "gamma_empty"]
    seen = {"ok": 0, "box_ok": 0}

    @settings(max_examples=int(os.environ.get("FWI_FUZZ_EXAMPLES", "500")), deadline=None, suppress_health_check=list(HealthCheck))
    @given(n=st.tuples(sizes, sizes, sizes), nt=st.integers(3, 6), seed=st.integers(0, 2 ** 16),
           max_shots=st.integers(1, 8), pairing=st.integers(0, 1), spl=st.integers(0, 3), psm=st.integers(0, 1),
           bad=st.lists(st.sampled_from(corruptions), max_size=2),
           box=st.tuples(*[st.integers(-1, 12)] * 7), whole=st.booleans())
    def check(n, nt, seed, max_shots, pairing, spl, psm, bad, box, whole):
        rng = np.random.default_rng(seed)
        nx, ny, nz = n
        nvox = nx * ny * nz
        pml = [int(rng.integers(0, m // 2 + 1)) for m in n]
        src = rng.integers(0, nvox, size=int(rng.integers(1, 5))).astype(np.int32)
        rec = rng.integers(0, nvox, size=int(rng.integers(1, 5))).astype(np.int32)
        gam = np.unique(rng.integers(0, nvox, size=int(rng.integers(1, 9)))).astype(np.int32)
        lay = gam[rng.random(len(gam)) < 0.5].copy()
        dx, dt, c_ref = 1e-3, 1e-7, 1500.0
        wav = np.ones(nt + 8, np.float32)
        for b in bad:
            if b == "nx": nx = int(rng.choice([-1, 0, 1, 7 * 11, 1 << 20]))
            if b == "nt": nt = int(rng.choice([-1, 0, 2]))
            if b == "pml": pml[int(rng.integers(0, 3))] = int(rng.choice([-1, 100]))
            if b == "max_shots": max_shots = int(rng.choice([-1, 0, 64]))
            if b == "pairing": pairing = int(rng.choice([-1, 2]))
            if b == "spl": spl = -1
            if b == "psm": psm = int(rng.choice([-1, 2]))
            if b == "dx": dx = float(rng.choice([0.0, -1.0, float("nan")]))
            if b == "dt": dt = float(rng.choice([0.0, -1.0, float("nan")]))
            if b == "c_ref": c_ref = float(rng.choice([0.0, -1.0, float("nan")]))
            if b == "src_range": src[0] = int(rng.choice([-1, nvox]))
            if b == "rec_range": rec[-1] = int(rng.choice([-1, nvox]))
            if b == "gamma_order" and len(gam) > 1: gam = gam[::-1].copy()
            if b == "layer_outside": lay = np.append(lay, np.int32(nvox - 1 if nvox - 1 not in gam else -1))
            if b == "gamma_empty": gam = gam[:0]
        keep = [np.ascontiguousarray(a, dtype=np.int32) for a in (src, rec, gam, lay)]
        P = fwi.fwi_problem()
        P.nx, P.ny, P.nz, P.nt = nx, ny, nz, nt
        P.pml[0], P.pml[1], P.pml[2] = pml
        P.dx, P.dt, P.c_ref, P.rho0, P.pml_alpha, P.c_rec = dx, dt, c_ref, 1000.0, 2.0, 0.0
        P.n_src, P.n_rec, P.n_gamma, P.n_layer = [len(k) for k in keep]
        ip = ctypes.POINTER(ctypes.c_int32)
        P.src_idx, P.rec_idx, P.gamma_idx, P.layer_idx = [k.ctypes.data_as(ip) for k in keep]
        P.wavelet = wav.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        P.pairing, P.max_shots, P.sims_per_launch, P.per_shot_models = pairing, max_shots, spl, psm
        status, plan, nbytes = fwi.fwi_plan_create(P)
        assert status in statuses
        if status != fwi.FWI_OK:
            return
        seen["ok"] += 1
        assert nbytes > 0
        for K in (1, max_shots):
            assert fwi.fwi_plan_voxel_steps(plan, K, 1) > 0
            assert L.fwi_plan_launches(plan, K, 1) > 0
        if whole:                        # the whole grid as the box, no PML: always valid
            box = (0, 0, 0, nx, ny, nz, 0)
        s_box, ws_box = fwi.fwi_plan_set_tr_box(plan, box[0:3], box[3:6], (box[6],) * 3)
        assert s_box in statuses and (s_box == fwi.FWI_OK or not whole)
        if s_box == fwi.FWI_OK:
            seen["box_ok"] += 1
            assert ws_box > 0 and fwi.fwi_plan_voxel_steps(plan, 1, 1) > 0
        fwi.fwi_plan_destroy(plan)

    check()
    assert seen["ok"] > 50 and seen["box_ok"] > 0, seen
