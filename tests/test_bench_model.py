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
