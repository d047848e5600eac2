"""The N > 1 bookkeeping of bench.py on the CPU, as world_size-2 gloo ranks
(no GPU): every rank times its own sequence, the job's time is the slowest
rank's, and only rank 0 prints. The data path itself has no collective
(independent sequences, weak scaling)."""
import json
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


def _rank(rank, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE="2")
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=2)
    try:
        # rank r took 10 + 5 r ms: the job took 15 ms
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist)
        q.put((rank, ms, bench.job_throughput(2, 100, 10, 4, ms * 1e-3)))
    finally:
        dist.destroy_process_group()


def test_slowest_rank_times_the_job():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks agree on the maximum; throughput counts both ranks' work
    assert [g[1] for g in got] == [15.0, 15.0]
    assert all(g[2] == pytest.approx(2 * 100 * 10 * 4 / 0.015) for g in got)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None) == 3.5
    assert bench.job_throughput(1, 40962, 100, 10, 0.064) == pytest.approx(40962 * 100 * 10 / 0.064)


def test_reference_arm_under_torchrun_prints_once():
    """Launched like the N = 2 driver run: rank 0 alone times the oracle and
    prints its line, the other rank exits 0 without work."""
    port = _free_port()
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
                        "--nproc-per-node", "2", "--master-addr", "127.0.0.1",
                        "--master-port", str(port), os.path.join(ROOT, "bench.py"),
                        "--impl", "reference", "--workload", "tiny", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0
