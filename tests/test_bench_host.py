"""Host logic of bench.py: algorithmic bytes per kernel and the validity rules of the
reported DRAM traffic (no GPU)."""
import importlib.util
import os

import pytest

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(_ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_algorithmic_bytes_count_fields_and_half_spectra(bench):
    """A half spectrum of nx/2+1 complex FP32 per nx reals; FP32 fields 4 B per voxel."""
    nx = 128
    hf = 8.0 * 65 / 128
    assert bench.alg_bytes_per_voxel("zpass_momentum", nx) == pytest.approx(3 * hf)
    assert bench.alg_bytes_per_voxel("zpass_mass", nx) == pytest.approx(6 * hf)
    # three velocity components read + written (24 B) on top of five half spectra
    assert bench.alg_bytes_per_voxel("plane_momentum", nx) - 5 * hf == pytest.approx(24.0)
    # three densities read + written and c0^2 read (28 B) on top of four half spectra
    assert bench.alg_bytes_per_voxel("plane_mass", nx) - 4 * hf == pytest.approx(28.0)
    step = sum(bench.alg_bytes_per_voxel(k, nx) for k in
               ("zpass_momentum", "plane_momentum", "zpass_mass", "plane_mass"))
    assert step == pytest.approx(125.125)


def test_traffic_only_for_the_captured_launches(bench):
    # the capture ran one stream group (every simulation of a phase in each launch), the launch
    # shape the headline roofline times
    sched = {"specialized": 2, "radix_order": 0, "z_tile": 32, "split_plane": 0, "stream_groups": 1}
    per_sim = bench.TRAFFIC_PER_SIM["bytes"]["plane_mass"]
    assert bench.traffic_per_launch("plane_mass", (128, 128, 64), sched, 6.0) == pytest.approx(6.0 * per_sim)
    assert bench.traffic_per_launch("plane_mass", (128, 128, 64), dict(sched, stream_groups=4), 1.5) is None
    # the plane kernels do not see the z tile; the z passes do
    z16 = dict(sched, z_tile=16)
    assert bench.traffic_per_launch("plane_mass", (128, 128, 64), z16, 1.0) == pytest.approx(per_sim)
    assert bench.traffic_per_launch("zpass_mass", (128, 128, 64), z16, 1.0) is None
    # other kernels' builds or grids: no figure
    assert bench.traffic_per_launch("plane_mass", (128, 128, 64), dict(sched, specialized=1), 1.0) is None
    assert bench.traffic_per_launch("plane_mass", (128, 128, 64), dict(sched, split_plane=1), 1.0) is None
    assert bench.traffic_per_launch("plane_mass", (160, 160, 80), sched, 1.0) is None
