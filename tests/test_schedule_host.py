"""Host logic of FFT schedule selection: the autotuner's candidate list, the C ABI's
schedule validation per grid, and the schedule cache (no GPU: plans without a workspace)."""
import json
import types

import numpy as np
import pytest

from paper_2102_00755_b300 import autotune
from paper_2102_00755_b300 import build as fbuild
from paper_2102_00755_b300 import fwi, synth

from .test_abi import _problem


@pytest.fixture(scope="module")
def L():
    fbuild.build()
    return fwi.lib()


def _plan(L, nx, ny, nz, max_shots=2):
    wl = synth.small_workload(nx, ny, nz, 12, pml=3, n_src=3, n_rec=8, K=1, layer=1, seed=3)
    P, keep = _problem(wl, max_shots=max_shots)
    st, plan, _ = fwi.fwi_plan_create(P)
    assert st == fwi.FWI_OK
    return types.SimpleNamespace(handle=plan, keep=keep)


def test_candidate_list_is_unique_and_consistent():
    keys = [tuple(c[k] for k in autotune.KNOBS) for c in autotune.CANDIDATES]
    assert len(keys) == len(set(keys))
    for c in autotune.CANDIDATES:
        assert set(c) == set(autotune.KNOBS)
        if c["specialized"] >= 1:
            assert c["radix_order"] == 0          # radix orders only steer the runtime schedules
        if c["stream_groups"] > 1:
            assert c["specialized"] == 2
        assert not (c["split_plane"] == 1 and c["specialized"] == 1)
    assert any(c["split_plane"] == 1 for c in autotune.CANDIDATES)
    assert {c["stream_groups"] for c in autotune.CANDIDATES} == {1, 2, 4}


def test_default_schedules_follow_the_plane_size(L):
    p128 = _plan(L, 128, 128, 16)
    s = autotune.get_schedule(p128)
    assert (s["specialized"], s["split_plane"]) == (2, 0)
    fwi.fwi_plan_destroy(p128.handle)
    p480 = _plan(L, 480, 480, 8)        # a 480^2 plane does not fit one CTA: split planes
    s = autotune.get_schedule(p480)
    assert (s["specialized"], s["split_plane"]) == (2, 1)
    fwi.fwi_plan_destroy(p480.handle)


def test_schedule_validation(L):
    p = _plan(L, 128, 128, 16)
    before = autotune.get_schedule(p)
    bad = [dict(before, z_tile=8), dict(before, stream_groups=3), dict(before, specialized=3),
           dict(before, radix_order=-1), dict(before, split_plane=2)]
    for b in bad:
        assert autotune.set_schedule(p, b) == fwi.FWI_EINVAL
        assert autotune.get_schedule(p) == before
    # every candidate is either taken or refused as unsupported, and a refusal keeps the old one
    taken = 0
    for c in autotune.CANDIDATES:
        st = autotune.set_schedule(p, c)
        assert st in (fwi.FWI_OK, fwi.FWI_ENOTSUP)
        if st == fwi.FWI_OK:
            taken += 1
            assert autotune.get_schedule(p) == c
        else:
            assert autotune.get_schedule(p) != c
    assert taken >= 2
    fwi.fwi_plan_destroy(p.handle)


def test_cache_round_trip(L, tmp_path, monkeypatch):
    path = tmp_path / "schedules.json"
    monkeypatch.setenv("FWI_SCHEDULE_CACHE", str(path))
    p = _plan(L, 64, 64, 16)
    assert not autotune.apply_cached(p, 64, 64, 16, 1)
    want = dict(specialized=2, radix_order=0, z_tile=16, split_plane=0, stream_groups=1)
    path.write_text(json.dumps({autotune.key_of(64, 64, 16, 1): {"schedule": want, "ms": 1.0}}))
    assert autotune.apply_cached(p, 64, 64, 16, 1)
    assert autotune.get_schedule(p) == want
    assert not autotune.apply_cached(p, 64, 64, 32, 1)
    fwi.fwi_plan_destroy(p.handle)
