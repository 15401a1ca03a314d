"""Serving loop: requests of two grid levels arriving faster than they finish are
admitted as slots free up, overlap on the device, and each result is the same as
when the request runs alone."""
import numpy as np
import pytest
import torch

from paper_2102_00755_b300 import build as fbuild
from paper_2102_00755_b300 import fwi, serve, synth

pytestmark = pytest.mark.gpu


def _levels():
    a = synth.small_workload(32, 32, 24, 60, pml=4, n_src=8, n_rec=24, K=1, seed=21)
    b = synth.small_workload(48, 40, 30, 80, pml=5, n_src=8, n_rec=32, K=1, seed=22)
    return [serve.make_level("A", a), serve.make_level("B", b)]


def test_mixed_stream_equals_alone_and_overlaps():
    fbuild.build()
    levels = _levels()
    reqs = serve.poisson_stream(["A", "B"], [1, 1], n=12, rate=500.0, n_src=8, seed=5)
    srv = serve.Server(levels, max_inflight=4)
    out = srv.run(reqs, keep_outputs=True)
    res = out["results"]
    st = out["stats"]
    assert st["requests"] == 12 and st["p50_s"] > 0 and st["p99_s"] >= st["p50_s"]
    # continuous batching: some request was admitted while another was still running
    spans = sorted((r.admitted, r.done) for r in res)
    assert any(spans[k + 1][0] < spans[k][1] for k in range(len(spans) - 1))
    srv.close()
    # each request alone, on a fresh plan, default stream
    by_name = {lv.name: lv for lv in levels}
    for req, r in zip(sorted(reqs, key=lambda q: q.rid), res):
        lv = by_name[req.level]
        plan = fwi.Plan.from_workload(lv.wl, max_shots=1)
        w = torch.tensor(req.weights[None], dtype=torch.float32, device="cuda")
        if req.kind == "forward":
            tr = plan.forward(lv.c, w)
            assert torch.equal(tr, r.traces), req.rid
        else:
            tr = torch.empty_like(r.traces)
            D, g = plan.gradient(lv.c, w, lv.raw_observed, encoded=False, traces=tr)
            assert torch.equal(tr, r.traces) and torch.equal(D, r.misfit) and torch.equal(g, r.grad), req.rid
        plan.close()


def test_admission_respects_memory_budget():
    fbuild.build()
    levels = _levels()
    reqs = serve.poisson_stream(["B"], [1], n=6, rate=1000.0, n_src=8, seed=6, p_gradient=1.0)
    probe = serve.Server(levels)
    one = probe._slot_bytes(levels[1])
    probe.close()
    srv = serve.Server(levels, max_inflight=8, mem_budget=int(2.5 * one))
    out = srv.run(reqs)
    assert out["stats"]["requests"] == 6
    assert max(len(v) for v in srv.pool.values()) <= 2        # never more slots than memory allows
    assert srv.refused_for_memory > 0
    srv.close()
