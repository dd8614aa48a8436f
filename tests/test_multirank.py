"""The N > 1 path of the benchmark (replicas: one domain per rank, no data-path
collective, the slowest rank's time, whole-job throughput printed by rank 0)
with world_size 2 on the CPU gloo backend, and the reference arm under
torchrun (rank 0 alone works and prints)."""
import json
import multiprocessing as mp
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    dist.barrier()
    t = bench.max_over_ranks(times[rank], dist, world, "cpu")
    out.put((rank, t, bench.job_mlups(world, 1000, 50, t)))
    dist.barrier()
    dist.destroy_process_group()


def test_slowest_rank_sets_the_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [1.25, 3.5]
    ps = [ctx.Process(target=_rank, args=(r, 2, port, times, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks see the maximum; the job rate counts both ranks' nodes
    assert [r[1] for r in res] == [3.5, 3.5]
    assert abs(res[0][2] - 2 * 1000 * 50 / 3.5 / 1e6) < 1e-15


def test_single_rank_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.0, None, 1, "cpu") == 2.0
    assert bench.job_mlups(1, 4096 * 4096, 1000, 0.4353) == pytest.approx(38543.5, rel=1e-4)


def test_reference_arm_under_torchrun_prints_once():
    """`bench.py --impl reference` launched as the driver launches N = 2:
    rank 0 times the oracle and prints one JSON line, rank 1 exits 0."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
