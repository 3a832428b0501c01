"""Host arithmetic of the benchmark line (no GPU): the algorithmic byte model of each kernel
family and the roofline fraction built from it."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_state_bytes_per_node():
    # label, excess, sink residual + down flow + 4 hard flows (+ 2 soft pair values)
    _, s_soft = bench.algorithmic_bytes(1, 50, 0, 0)
    _, s_hard = bench.algorithmic_bytes(1, 0, 0, 0)
    assert s_soft == 4 * (3 + 1 + 4 + 2) == 40
    assert s_hard == 4 * (3 + 1 + 4) == 32


def test_family_bytes():
    N = 512 * 512 * 384
    by, S = bench.algorithmic_bytes(N, 50, tiles_per_sweep=1000, scans_per_sweep=0.5)
    assert by["sweep"] == 4 * N * 0.5 + 1000 * 1024 * (S + 8)
    assert by["bfs"] == (16 + 4 * 7) * N       # 44 B per node with soft arcs
    assert by["cut"] == (8 + 4 * 7) * N
    assert by["build"] == (4 + S) * N
    by0, S0 = bench.algorithmic_bytes(N, 0, 0, 0)
    assert by0["bfs"] == (16 + 4 * 5) * N and by0["sweep"] == 0


def test_job_throughput_and_roofline_units():
    # 100.66 M nodes per solve at 1.834 s: 54.9 Mnodes/s
    assert abs(bench.job_throughput(1, 100663296, 3, 3 * 1834.729) - 54.865) < 0.01
    # 0.456 ms per tiled sweep moving 398.9 MB: 874 GB/s
    by = 398911296.0
    assert abs(by / (0.45645 / 1e3) / 1e9 - 873.9) < 0.1


def test_convex_sweep_model():
    # delta 9, f(t) = 4 t^2: k_0 = 4 and k_1..k_8 = 8, so 8 layers d >= 1 and the pair layer
    t = [4 * d * d for d in range(1, 10)]
    nl, arcs, per_node = bench.convex_sweep_model(t)
    assert nl == 8
    assert arcs == 3 + 4 * (2 + 1 + 16) == 79   # sink, down, up; per direction hard out/in, pair, 8 x 2 layer arcs
    assert per_node == 20 + 8 * 79 == 652
    # the linear profile has the pair layer only; the hinge profile 7 (t - 1)^+ one layer d = 1
    assert bench.convex_sweep_model([3, 6, 9]) == (0, 3 + 4 * 3, 20 + 8 * 15)
    assert bench.convex_sweep_model([0, 7, 14])[:2] == (1, 3 + 4 * (2 + 0 + 2))
    assert bench.convex_sweep_model([]) == (0, 3 + 4 * 2, 20 + 8 * 11)


def test_convex_traffic_is_gated_by_the_kernel_source():
    entry = bench.MEASURED_TRAFFIC["k_cv_push_relabel"]
    if entry["source_sha"] == bench._source_sha("k_cv_push_relabel"):
        assert bench.measured_traffic("k_cv_push_relabel", 1000) == entry["bytes_per_unit"] * 1000
    else:
        assert bench.measured_traffic("k_cv_push_relabel", 1000) is None
