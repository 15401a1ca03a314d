"""Host logic of the serving loop (admission, memory, continuous batching) with fake slots
in place of device plans: no GPU."""
import numpy as np
import pytest
import torch

from paper_2102_00755_b300 import serve


class _Event:
    def __init__(self, slot):
        self.slot = slot

    def query(self):
        # a launch completes after its level's number of polls
        self.slot.polls += 1
        return self.slot.polls >= self.slot.level.c["polls"]


class _Plan:
    def __init__(self, slot):
        self.slot = slot
        self.closed = False

    def voxel_steps(self, K, gradient):
        return 1000 * (3 if gradient else 1)

    def close(self):
        self.closed = True
        _FakeSlot.closed += 1


class _FakeSlot:
    """Stands in for serve._Slot: the same attributes the server uses."""
    made = []
    closed = 0
    log = []

    def __init__(self, level, device, pairing, use_graphs):
        self.level = level
        self.plan = _Plan(self)
        self.busy = False
        self.bytes = level.c["bytes"]
        self.done_event = _Event(self)
        self.polls = 0
        _FakeSlot.made.append(self)

    def launch(self, kind, weights):
        self.polls = 0
        _FakeSlot.log.append(("launch", self.level.name, kind, id(self)))


@pytest.fixture
def fake(monkeypatch):
    _FakeSlot.made, _FakeSlot.closed, _FakeSlot.log = [], 0, []
    monkeypatch.setattr(serve, "_Slot", _FakeSlot)
    monkeypatch.setattr(serve.Server, "_slot_bytes", lambda self, lv: lv.c["bytes"])
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "empty_cache", lambda *a, **k: None)
    return _FakeSlot


def _level(name, bytes_, polls):
    # the server only passes a level through to its slots; the fake reads `c` as its spec
    return serve.Level(name=name, wl=None, c={"bytes": bytes_, "polls": polls})


def _req(rid, level, kind="gradient", arrival=0.0):
    return serve.Request(rid, level, kind, np.ones(4, np.float32), arrival)


def test_requests_overlap_up_to_the_inflight_cap(fake):
    srv = serve.Server([_level("A", 10, polls=5)], device="cpu", max_inflight=3, mem_budget=1000)
    out = srv.run([_req(i, "A") for i in range(7)], realtime=False, poll_s=0.0)
    assert out["stats"]["requests"] == 7 and out["stats"]["gradients"] == 7
    # three slots were made (the cap), later requests reuse them as they free up
    assert len(fake.made) == 3
    assert sum(1 for e in fake.log if e[0] == "launch") == 7
    # the first three were admitted before any completed: continuous batching, not a queue
    first = sorted(out["results"], key=lambda r: r.admitted)[:3]
    assert max(r.admitted for r in first) < min(r.done for r in out["results"])
    assert [r.rid for r in out["results"]] == list(range(7))
    assert out["stats"]["gvoxel_steps_per_s"] > 0


def test_memory_budget_limits_slots_and_releases_idle_levels(fake):
    big, small = _level("big", 60, polls=3), _level("small", 30, polls=3)
    srv = serve.Server([big, small], device="cpu", max_inflight=8, mem_budget=100)
    reqs = [_req(0, "small"), _req(1, "small"), _req(2, "small"), _req(3, "big"), _req(4, "small")]
    out = srv.run(reqs, realtime=False, poll_s=0.0)
    st = out["stats"]
    assert st["requests"] == 5
    # three small slots fit (90 of 100); the big request waits for memory, is refused while
    # small ones run, then gets memory once the idle small slots are released
    # one request (the big one) had to wait; it is counted once however long it polled
    assert st["refused_for_memory"] == 1
    assert fake.closed >= 1
    assert srv.reserved <= 100
    order = [e[1] for e in fake.log]
    assert order.index("big") == 3


def test_forward_and_gradient_kinds_and_fifo_admission(fake):
    srv = serve.Server([_level("A", 10, polls=2)], device="cpu", max_inflight=1, mem_budget=100)
    reqs = [_req(0, "A", "forward", 0.0), _req(1, "A", "gradient", 0.0), _req(2, "A", "forward", 0.0)]
    out = srv.run(reqs, realtime=False, poll_s=0.0)
    assert [e[2] for e in fake.log] == ["forward", "gradient", "forward"]
    assert out["stats"]["gradients"] == 1
    res = out["results"]
    assert res[0].done <= res[1].admitted and res[1].done <= res[2].admitted   # one in flight at a time
