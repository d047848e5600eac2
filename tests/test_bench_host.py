"""Host-side checks of bench.py's bookkeeping (no GPU): the algorithmic work
per stage that the roofline divides by, and the guard that reports a kernel's
measured DRAM traffic only while its sources are the ones that were measured."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402
from paper_2602_22212_gb300 import inputs as I  # noqa: E402


def test_stage_work_at_the_benchmark_size():
    """Per vertex-frame the forward is 2 H^2 (D - 1) + 2 x 7 H FLOP (17.3 k at
    H = 64, D = 3) and the backward twice that, 34.56 k (51.8 k for forward +
    backward, the recompute inside the backward kernel not counted); the
    preconditioner reads and writes 8 B and Adam moves 28 B per grid parameter."""
    p = I.preset("paper")
    N, T = 40962, 100
    H, D, NO, Z, M = 64, 3, 7, 6, 4
    K = Z + 2 * M
    w = bench.stage_work(p, N, T, 20000 * T, (H, D, K, Z, NO), "tc", "bf16", 10000)
    rows = N * T
    assert w["decode"][0] == "tensor" and w["decode"][1] == (2 * H * H * 2 + 2 * NO * H) * rows
    assert w["mlp_bwd"][1] == 34560 * rows
    assert abs((w["decode"][1] + w["mlp_bwd"][1]) / rows - 51.8e3) < 0.1e3
    n = sum(r ** 3 * p["F"] for r in p["res"]) + 4 ** 3 * 2
    assert w["precond"] == ("hbm", (8 + 28) * n, "B")
    assert w["adam"] == ("hbm", 28 * 10000, "B")
    w32 = bench.stage_work(p, N, T, 20000 * T, (H, D, K, Z, NO), "fp32", "fp32", 10000)
    assert w32["decode"][0] == "alu" and w32["precond"][0] == "alu"


def test_measured_traffic_follows_the_sources(monkeypatch):
    rec = bench.MEASURED_TRAFFIC[("mlp_bwd_tc2_kernel", "paper")]
    assert rec["bytes"] is None or rec["bytes"] > 0
    if rec["bytes"] is not None:
        assert bench.measured_traffic("mlp_bwd_tc2_kernel", "paper") in (rec["bytes"], None)
    monkeypatch.setattr(bench, "sources_sha", lambda kernel: "0" * 64)
    assert bench.measured_traffic("mlp_bwd_tc2_kernel", "paper") is None
    assert bench.measured_traffic("mlp_bwd_tc2_kernel", "profile") is None
    assert bench.measured_traffic("decode_tc_kernel", "paper") is None


def test_sources_hash_covers_the_kernel_files():
    import hashlib
    csrc = os.path.join(ROOT, "paper_2602_22212_gb300", "csrc")
    h = hashlib.sha256()
    for f in bench.KERNEL_SOURCES["mlp_bwd_tc2_kernel"]:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    assert bench.sources_sha("mlp_bwd_tc2_kernel") == h.hexdigest()
    # the committed record matches the committed sources
    rec = bench.MEASURED_TRAFFIC[("mlp_bwd_tc2_kernel", "paper")]
    if rec["sha256"] is not None:
        assert rec["sha256"] == h.hexdigest()


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` times the FP64 oracle on the host cores and
    prints one JSON line with the arm's keys (tiny workload here)."""
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "tiny", "--steps", "1", "--warmup", "3"],
                         capture_output=True, text=True, timeout=300, check=True).stdout
    lines = [l for l in out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "e2e",
              "cpu_baseline"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["steps"] == 1 and d["warmup"] == 3
