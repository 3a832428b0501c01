"""The multi-GPU path of the benchmark is independent replicas (the solve of one volume is not
sharded): ranks only meet for a barrier and the maximum of their timings. Its host logic runs
here as world-size-2 gloo process groups on CPU, and the reference arm's rank gating as plain
subprocesses."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r timed (10 r + 1, 5 - r) ms: the job time is the slowest rank's
        got = bench.max_over_ranks([10 * rank + 1, 5 - rank])
        dist.barrier()
        out.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    results = dict(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert results == {0: [11.0, 5.0], 1: [11.0, 5.0]}


def test_max_over_ranks_without_group_is_identity():
    assert bench.max_over_ranks([3, 4.5]) == [3.0, 4.5]


def test_job_throughput_counts_every_rank():
    # two replicas of 100 M nodes, 3 steps each, slowest rank 6 s: 100 Mnodes/s for the job
    assert bench.job_throughput(2, 100_000_000, 3, 6000.0) == pytest.approx(100.0)
    assert bench.job_throughput(1, 100_000_000, 3, 6000.0) == pytest.approx(50.0)


@pytest.mark.parametrize("rank", [0, 1])
def test_reference_arm_runs_on_rank_zero_only(rank):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank))
    res = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "small", "--steps", "1",
                          "--warmup", "1"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.strip()]
    if rank:
        assert lines == []
    else:
        assert len(lines) == 1
        line = json.loads(lines[0])
        assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
        assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
