"""The multi-GPU form (replicas only: an independent encoded gradient estimate per rank, the
job timed as the slowest rank) as two gloo ranks on the CPU."""
import importlib.util
import os
import socket

import numpy as np
import torch.multiprocessing as mp

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(_ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench = _bench()
        from paper_2102_00755_b300 import synth
        wl = synth.small_workload(12, 11, 10, 8, pml=2, n_src=6, n_rec=4, K=3, layer=1, seed=5)
        w = bench.replica_weights(wl.weights, rank)
        local_ms = 10.0 + 7.5 * rank                       # rank 1 is the slow one
        job = bench.job_time_ms(local_ms, world, device="cpu")
        rate = bench.whole_job_rate(1000.0, world, 4, job)
        dist.barrier()
        out.put((rank, w, job, rate))
    finally:
        dist.destroy_process_group()


def test_two_replicas_time_the_slowest_rank_and_draw_their_own_encodings():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.SimpleQueue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world):
        r, w, job, rate = out.get()
        res[r] = (w, job, rate)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    # both ranks agree on the job time (the max) and on the whole-job rate
    assert res[0][1] == res[1][1] == 17.5
    assert res[0][2] == res[1][2] == 1000.0 * 2 * 4 / 17.5e-3
    # rank 0 keeps the workload's encoding, rank 1 draws its own Rademacher super-shots
    from paper_2102_00755_b300 import synth
    wl = synth.small_workload(12, 11, 10, 8, pml=2, n_src=6, n_rec=4, K=3, layer=1, seed=5)
    assert np.array_equal(res[0][0], wl.weights)
    w1 = res[1][0]
    assert w1.shape == wl.weights.shape and set(np.unique(w1)) <= {-1.0, 1.0}
    assert not np.array_equal(w1, wl.weights)


def test_single_rank_needs_no_process_group():
    bench = _bench()
    assert bench.job_time_ms(12.5, 1) == 12.5
    assert bench.whole_job_rate(2.0, 1, 3, 1000.0) == 6.0
