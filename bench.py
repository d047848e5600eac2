#!/usr/bin/env python
"""fwd+bwd+step vertex-frames/s of the Neu-PiG optimisation iteration on GB300.

One step = one full iteration through the C ABI (npg_iteration): latent-grid
lookup, time modulation, MLP decode + rigid transform for every vertex and
frame, bidirectional Chamfer nearest neighbours, loss, hand-written backward,
Sobolev preconditioner on every grid level and Adam.

Workload (default "paper"): capsule figure remeshed to N = 40962 vertices,
T = 100 frames of 20000 noisy points, 8-level grid 16 -> 256 with 4 features,
MLP 3 x 64 LeakyReLU; synthetic, seeded. Its per-iteration working set (grid,
gradient, moments: ~3 GB) is far larger than L2, so no L2 flush is needed
between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16|fp32]
                  [--graph|--no-graph] [--impl npg|reference]

The default form is the metric's headline: BF16 tensor-core MLP, tensor-core
preconditioner, the iteration replayed from a CUDA graph (`value`); the plain
FP32 per-sequence form (FP32 SIMT MLP and preconditioner, eager) is timed on
the same sequence and state beside it (`plain_fp32`, with the ratio).

With N > 1 (torchrun, one rank per GPU) every rank optimises its own sequence
(independent problems: weak scaling, no data-path collective); value counts
the vertex-frames of all ranks over the slowest rank's time.
--impl reference times the FP64 CPU oracle on the host cores instead, each
step a bounded sample of the same workload extrapolated to a full iteration.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fwd+bwd+step vertex-frames/s at T=100, N=40962; batched BF16 vs plain FP32"
UNIT = "vertex-frames/s"
FP32_LANES_PER_SM = 128  # FP32 FMA units per SM (Blackwell)


def fp32_peak_tflops(sms, mhz):
    """FP32 peak from unit counts: SMs x FMA lanes x 2 FLOP x SM clock."""
    return sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of a
# kernel at the default workload, from a one-pass ncu capture, with the
# SHA-256 of the sources that define the kernel at capture time: a changed
# source reports null traffic until the counters are taken again.
KERNEL_SOURCES = {
    "mlp_bwd_tc2_kernel": ("k_mlp_tc64.cu", "mlp_tc_common.cuh", "tc_sm100.cuh",
                           "npg_device.cuh"),
}
MEASURED_TRAFFIC = {
    ("mlp_bwd_tc2_kernel", "paper"): {"bytes": 78841344 + 1164800,
                                      "sha256": "e4c2c2ce952c704c6e0fccee2fd1baee4e9d4e37a32856dcdbc65e882bfab34b"},
}


def sources_sha(kernel):
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2602_22212_gb300", "csrc")
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(kernel, workload):
    rec = MEASURED_TRAFFIC.get((kernel, workload))
    if not rec or rec["bytes"] is None or kernel not in KERNEL_SOURCES:
        return None
    return rec["bytes"] if sources_sha(kernel) == rec["sha256"] else None


def max_over_ranks(x, dist):
    """The maximum of a per-rank scalar over all ranks (x itself without a
    process group); on the process group's device (CUDA for NCCL)."""
    if dist is None:
        return float(x)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, N, T, steps, seconds):
    """Whole-job vertex-frames/s: every rank processes its own N x T sequence
    (weak scaling), timed by the slowest rank."""
    return world * N * T * steps / seconds


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return dict(hbm=d["hbm_gbs"], bf16=d["bf16_tflops"], bf16_sus=d["bf16_tflops_sustained"],
                    src="measured")
    return dict(hbm=6800.0, bf16=1900.0, bf16_sus=1700.0, src="fallback")


def workload(name, seed=0):
    from paper_2602_22212_gb300 import inputs as I
    p = I.preset(name)
    seq = I.make_sequence(p, seed=seed)
    return p, seq


def make_cfg(npg, p, precision, graph, stream, e_max, precond):
    return npg.make_config(p["L"], p["res"], p["F"], p["H"], p["D"], slope=p["slope"],
                           precision=npg.BF16_MLP if precision == "bf16" else npg.FP32,
                           e_max=e_max, use_graph=graph, stream=stream,
                           w_iso=p.get("w_iso", 100.0),
                           precond_mode=npg.PRECOND_TC if precond == "tc" else npg.PRECOND_FP32)


# ----------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.f = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for k, n in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ----------------------------------------------------------------- algorithmic work

def stage_work(p, N, T, MT, mlp_dims, precond="fp32", precision="fp32", mlp_len=0):
    """Algorithmic bytes / FLOPs per launch of each stage (formulas per stage below)."""
    H, D, K, Z, NO = mlp_dims
    L, F = p["L"], p["F"]
    rows = N * T
    # per vertex-frame: the forward's hidden and output layers (the first layer
    # is factorised into per-vertex U and per-frame V); the backward is twice
    # that (input and weight gradients), the forward recompute inside the
    # backward kernel is not counted as algorithmic work
    fwd_row = 2 * H * H * (D - 1) + 2 * NO * H
    bwd_row = 2 * fwd_row
    res = p["res"]
    dct_flops = sum(12 * r ** 4 * F for r in res) + 12 * 4 ** 4 * 2
    dct_bytes = sum(6 * 8 * r ** 3 * F for r in res) + 6 * 8 * 4 ** 3 * 2
    n_params = sum(r ** 3 * F for r in res) + 4 ** 3 * 2
    mlp_kind = "tensor" if precision == "bf16" else "alu"
    return {
        "nn_x": ("alu", None, "FLOP"),
        "nn_p": ("alu", None, "FLOP"),
        "decode": (mlp_kind, fwd_row * rows, "FLOP"),
        "mlp_bwd": (mlp_kind, bwd_row * rows, "FLOP"),
        # the grid levels' Adam steps run inside the preconditioner stage (each
        # level's DCT passes and Adam on one of four concurrent stream lanes);
        # the adam stage is the MLP's. Algorithmic bytes per grid parameter: read and
        # write of the gradient for Eq. 9 (8 B) and Adam's read of p, g~, m, v
        # and write of p, m, v (28 B). The six DCT passes move 48 B per value
        # (implementation traffic, `dct_bytes`).
        "precond": (("hbm", 36 * n_params, "B") if precond == "tc"
                    else ("alu", dct_flops, "FLOP")),
        "adam": ("hbm", 28 * mlp_len, "B"),
        "encode": ("hbm", N * (8 * L * F + 8 * 2) * 4 + N * 16 * 2, "B"),
        "scatter": ("hbm", N * (8 * L * F + 8 * 2) * 4 * 2, "B"),
    }


# ----------------------------------------------------------------- CPU oracle sample

def cpu_info():
    """Host CPU model and logical core count (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "hardware", "cpu part")):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return {"model": model, "nproc": os.cpu_count()}


def oracle_timed(p, seq, frames):
    """The oracle sample on one host thread and on all of them."""
    import oracle as O
    n0 = O.set_threads()
    out = {}
    try:
        for label, n in (("one", 1), ("all", os.cpu_count() or 1)):
            used = O.set_threads(n)
            v, s, desc = oracle_sample(p, seq, frames=frames)
            out[label] = (v, s, desc, used)
    finally:
        O.set_threads(n0)
    return out


def oracle_sample(p, seq, frames=1, level=1):
    """Time the FP64 oracle on a bounded sample of the workload and extrapolate
    one full iteration: `frames` frames of the per-frame work (decode, Chamfer
    by brute force, loss and reverse pass) and the preconditioner (CG) + Adam
    on one grid level, scaled to all levels by node count x sqrt(1 + 12 lambda)
    (CG iterations grow with the square root of the condition number)."""
    import oracle as O
    cfg = O.make_cfg(L=p["L"], res=p["res"], F=p["F"], H=p["H"], D=p["D"], slope=p["slope"],
                     w_iso=p.get("w_iso", 100.0))
    sub = seq.offsets[:frames + 1]
    prob = O.Problem(cfg, seq.x, seq.n, seq.faces, seq.points[:sub[-1]], sub, 0)
    from paper_2602_22212_gb300 import inputs as I
    rng = np.random.default_rng(0)
    grid = rng.normal(scale=0.01, size=O.grid_len(cfg))
    mlp = I.mlp_init(O.k_in(cfg), p["H"], p["D"], O.n_out(cfg), seed=0,
                     zero_last=False).astype(np.float64)
    t0 = time.perf_counter()
    O.loss_full(prob, grid, mlp, 1, 10)
    t_frames = time.perf_counter() - t0
    r = p["res"][level]
    lam = [0.4 * 1.5 ** l for l in range(p["L"])]
    g = rng.normal(size=r ** 3 * p["F"])
    t0 = time.perf_counter()
    pc, _ = O.precondition(r, p["F"], lam[level], g)
    O.adam(np.zeros_like(g), pc, np.zeros_like(g), np.zeros_like(g), 0.01, 1)
    t_lvl = time.perf_counter() - t0
    scale = sum((rr / r) ** 3 * np.sqrt((1 + 12 * lam[l]) / (1 + 12 * lam[level]))
                for l, rr in enumerate(p["res"]))
    t_iter = t_frames / frames * seq.T + t_lvl * scale
    desc = (f"{frames} frame(s) of N={seq.N}, M={int(seq.offsets[1])} (decode, brute-force "
            f"Chamfer, loss, reverse pass: {t_frames:.2f} s) + CG preconditioner and Adam on "
            f"the {r}^3 x {p['F']} level ({t_lvl:.2f} s), extrapolated to T={seq.T} and all "
            f"{p['L']} levels")
    return seq.N * seq.T / t_iter, t_frames + t_lvl, desc


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    p, seq = workload(args.workload)
    cores = O.set_threads(os.cpu_count() or 1)
    for _ in range(args.warmup):
        oracle_sample(p, seq)
    vals, secs = [], 0.0
    desc = ""
    for _ in range(args.steps):
        v, s, desc = oracle_sample(p, seq)
        vals.append(v)
        secs += s
    value = float(np.mean(vals))
    host = cpu_info()
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_dict(p, seq, "f64 CPU oracle", False),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": desc, "cpu_model": host["model"], "nproc": host["nproc"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def run_micro(args):
    """Standalone preconditioner call (six DCT passes) on one r^3 x 4 grid
    level: the small case for kernel profiles. Each call also builds its
    tables on the host, allocates scratch and synchronises, so ms_per_call is
    an upper bound on the kernels' time; the in-step stage timing of the
    benchmark proper is the kernel figure."""
    import torch
    from paper_2602_22212_gb300 import build, npg
    build.build()
    r, F = args.micro_res, 4
    stream = torch.cuda.Stream()
    g = torch.randn(r ** 3 * F, device="cuda")
    out = torch.empty_like(g)
    fn = npg.npg_precondition_tc if args.micro == "precond_tc" else npg.npg_precondition
    lam = 0.4 * 1.5 ** 7
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            fn(g, out, r, F, lam, stream=stream)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            fn(g, out, r, F, lam, stream=stream)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    nbytes = 6 * 8 * r ** 3 * F
    peaks = load_peaks()
    print(json.dumps({"micro": args.micro, "r": r, "F": F, "ms_per_call": ms,
                      "algorithmic_bytes": nbytes, "gbs_lower_bound": nbytes / ms / 1e6,
                      "hbm_peak_gbs": peaks["hbm"], "peak_source": peaks["src"]}))


def run_batch(args):
    """Uneven sequences (sizes from inputs.batch_specs: N 5k-50k, T 50-500, M
    5k-30k, sphere blobs and capsule figures) optimised as one batch: every
    iteration of all of them is one CUDA-graph launch, the sequences in
    chains (npg_batch_set_width; the chain count is swept unless given).
    value = total vertex-frames / batched iteration time; the same
    contexts run one after the other (each its own graph, synchronised in
    between) for `one_by_one`. Sequences are generated in worker processes
    (spawned before any CUDA use); generation is outside the timed region."""
    from concurrent.futures import ProcessPoolExecutor
    import multiprocessing as mp
    from paper_2602_22212_gb300 import inputs as I
    specs = I.batch_specs(args.batch, seed=0)
    with ProcessPoolExecutor(max_workers=min(len(specs), os.cpu_count() or 1),
                             mp_context=mp.get_context("spawn")) as ex:
        seqs = list(ex.map(I.make_batch_sequence, specs))
    import torch
    from paper_2602_22212_gb300 import build, npg
    build.build()
    p = dict(L=8, res=I.linear_resolutions(8, 16, 256), F=4, H=64, D=3, slope=0.01, w_iso=1.0)
    K, NO = 2 + p["F"] + 8, 7
    ctxs, streams = [], []
    for k, seq in enumerate(seqs):
        st = torch.cuda.Stream()
        cfg = make_cfg(npg, p, "bf16", True, st, 200, "tc")
        ctxs.append(npg.Context(cfg, seq, I.mlp_init(K, p["H"], p["D"], NO, seed=k),
                                device_inputs=True))
        streams.append(st)
    # each sequence's launch shapes (search-grid resolutions, decode CTAs per
    # SM) tuned to its sizes before the batch is captured
    tuned = [npg.npg_autotune(c.h, 2) for c in ctxs] if not args.no_autotune else None
    main = torch.cuda.Stream()
    vf = sum(s.N * s.T for s in seqs)

    def time_batch(batch, steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(main)
        for _ in range(steps):
            npg.npg_batch_iteration(batch)
        e1.record(main)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    # the graph's concurrency: sequences in `width` chains (1: one after the
    # other; 0: every sequence its own branch), the fastest of a short sweep
    # (its iterations are part of the warm-up)
    sweep = {}
    if args.batch_width is None:
        for w in (1, 2, 4, 0):
            b = npg.npg_batch_create([c.h for c in ctxs], main)
            npg.npg_batch_set_width(b, w)
            for _ in range(2):
                npg.npg_batch_iteration(b)
            sweep[w] = time_batch(b, 3)
            npg.npg_batch_destroy(b)
        width = min(sweep, key=sweep.get)
    else:
        width = args.batch_width
    batch = npg.npg_batch_create([c.h for c in ctxs], main)
    npg.npg_batch_set_width(batch, width)
    for _ in range(args.warmup):
        npg.npg_batch_iteration(batch)
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    l0 = sum(npg.npg_launch_count(c.h) for c in ctxs)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(main)
    for _ in range(args.steps):
        npg.npg_batch_iteration(batch)
    ev1.record(main)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    clocks = sampler.stop()
    launches = sum(npg.npg_launch_count(c.h) for c in ctxs) - l0
    # one by one: each sequence's own graph, the next one after it finishes
    for c in ctxs:
        npg.npg_iteration(c.h)  # eager + capture of the per-sequence graph
    torch.cuda.synchronize()
    steps1 = max(1, args.steps // 2)
    t0 = time.perf_counter()
    for _ in range(steps1):
        for c in ctxs:
            npg.npg_iteration(c.h)
            torch.cuda.synchronize()
    ms1 = (time.perf_counter() - t0) / steps1 * 1e3
    npg.npg_batch_destroy(batch)
    sizes = [dict(gen=s["gen"], N=q.N, T=q.T, M=s["M"]) for s, q in zip(specs, seqs)]
    print(json.dumps({
        "metric": f"batched uneven sequences: total vertex-frames/s ({len(seqs)} sequences)",
        "value": vf / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16", "data": "synthetic (seeded sphere blobs and "
        "capsule figures of uneven sizes; no dataset)",
        "config": {"workload": f"{len(seqs)} uneven sequences, {vf} vertex-frames per "
                               "iteration, 8-level grid 16->256 x F=4, MLP 3x64, w_iso=1",
                   "form": "one CUDA graph per batch iteration, the sequences in "
                           + ("one chain" if width == 1 else
                              "a branch each" if width == 0 or width >= len(seqs) else
                              f"{width} concurrent chains"),
                   "chains": width,
                   "chain_sweep_ms": {str(k): round(v, 3) for k, v in sweep.items()} or None,
                   "sequences": sizes},
        "one_by_one": {"value": vf / (ms1 * 1e-3), "unit": UNIT, "ms_per_step": ms1,
                       "timing": "host clock, each sequence's graph synchronised"},
        "autotuned": ([dict(vertex_cells=t[0], point_cells=t[1], decode_ctas_per_sm=t[2],
                            ball_rows_x=t[3], ball_rows_p=t[4]) for t in tuned]
                      if tuned else None),
        "gpu_launches": int(launches), "clocks": clocks}))
    for c in ctxs:
        c.close()


def config_dict(p, seq, form, graph):
    return {"workload": f"{p['gen']} N={seq.N} T={seq.T} M={int(seq.offsets[1])}/frame, "
                        f"{p['L']}-level grid {p['res'][0]}->{p['res'][-1]} x F={p['F']}, "
                        f"MLP {p['D']}x{p['H']}",
            "form": form, "cuda_graph": bool(graph),
            "l2": "working set (~3 GB of grid state per step) exceeds L2; no flush",
            "N": seq.N, "T": seq.T, "M": int(seq.offsets[1]), "levels": p["res"], "F": p["F"],
            "H": p["H"], "depth": p["D"], "w_iso": p.get("w_iso", 100.0)}


# ----------------------------------------------------------------- main

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="npg", choices=["npg", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16"],
                    help="bf16: the batched BF16 graph-captured form (headline); fp32: the "
                         "plain FP32 per-sequence form")
    ap.add_argument("--no-fp32-leg", action="store_true",
                    help="skip timing the plain FP32 form beside the BF16 form")
    ap.add_argument("--graph", dest="graph", action="store_true", default=None)
    ap.add_argument("--no-graph", dest="graph", action="store_false")
    ap.add_argument("--batch-width", type=int, default=None,
                    help="with --batch: chains of sequences in the batch graph (0: one branch "
                         "per sequence); default: the fastest of 1, 2, 4 and 0")
    ap.add_argument("--workload", default="paper", choices=["paper", "long", "stress", "tiny", "profile"])
    ap.add_argument("--precond", default=None, choices=["fp32", "tc"],
                    help="preconditioner DCT arithmetic (default: tc with bf16, fp32 with fp32)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--batch", type=int, default=0,
                    help="time that many uneven sequences as one batch (npg_batch_*) against "
                         "running them one by one, instead of the single-sequence step")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch shapes (no npg_autotune) in the BF16 form")
    ap.add_argument("--micro", default=None, choices=["precond_tc", "precond_fp32"],
                    help="time one kernel family alone on a standalone grid instead of the step")
    ap.add_argument("--micro-res", type=int, default=256)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)
    if args.micro:
        return run_micro(args)
    if args.batch:
        return run_batch(args)

    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2602_22212_gb300 import build, npg
    build.build()
    graph = (args.precision == "bf16") if args.graph is None else args.graph
    precond = args.precond or ("tc" if args.precision == "bf16" else "fp32")

    p, seq = workload(args.workload, seed=rank)
    stream = torch.cuda.Stream()
    from paper_2602_22212_gb300 import inputs as I
    H, D = p["H"], p["D"]
    K, Z, NO = 2 + p["F"] + 8, 2 + p["F"], 7
    mlp = I.mlp_init(K, H, D, NO, seed=rank)
    e_max = p["iters"]
    cfg = make_cfg(npg, p, args.precision, graph, stream, e_max, precond)
    ctx = npg.Context(cfg, seq, mlp, device_inputs=True)
    N, T, MT = seq.N, seq.T, int(seq.offsets[-1])
    # the batched form's launch shapes come from the project's autotuner
    # (search-grid resolutions, decode CTAs per SM); the plain form keeps the
    # defaults. Tuning runs forward and loss passes only: the optimisation
    # state is unchanged.
    tuned = None
    if args.precision == "bf16" and not args.no_autotune:
        tuned = npg.npg_autotune(ctx.h, 3)

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        ctx.iteration()
    torch.cuda.synchronize()
    # the optimisation state the timed region starts from; the stage
    # attribution and the end-to-end run restart from it, so that all three
    # see the same nearest-neighbour workload
    state0 = npg.npg_get_state(ctx.h)
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = npg.npg_launch_count(ctx.h)
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        npg.npg_iteration(ctx.h, None)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = ev0.elapsed_time(ev1)
    clocks = sampler.stop()
    launches = npg.npg_launch_count(ctx.h) - launches0
    ms = max_over_ranks(ms, dist)
    value = job_throughput(world, N, T, args.steps, ms * 1e-3)

    # per-stage attribution: the same iteration, eager, with CUDA events per stage
    sctx = ctx
    npg.npg_set_state(ctx.h, state0)
    if graph:
        cfg2 = make_cfg(npg, p, args.precision, False, stream, e_max, precond)
        sctx = npg.Context(cfg2, seq, mlp, device_inputs=True)
        if tuned is not None:
            npg.npg_autotune(sctx.h, 3)
        for _ in range(args.warmup):
            sctx.iteration()
    npg.npg_timing(sctx.h, args.steps)
    for _ in range(args.steps):
        npg.npg_iteration(sctx.h, None)
    stages = {}
    n_timed = 1
    for k, name in enumerate(npg.STAGES):
        tot, n = npg.npg_timing_read(sctx.h, k)
        stages[name] = tot / max(n, 1)
        n_timed = max(n_timed, n)
    cx, rx, cp, rp = npg.npg_search_stats(sctx.h)
    search = {"cand_per_query_x": cx / n_timed / (N * T), "rows_per_query_x": rx / n_timed / (N * T),
              "cand_per_query_p": cp / n_timed / MT, "rows_per_query_p": rp / n_timed / MT}
    npg.npg_timing(sctx.h, 0)

    # e2e: host buffers through the public API; each step uploads the step's
    # point clouds from pinned memory and reads the loss back
    e2e_steps = args.e2e_steps or max(3, args.steps // 2)
    pts_pin = torch.from_numpy(np.ascontiguousarray(seq.points)).pin_memory()
    off_pin = torch.from_numpy(np.ascontiguousarray(seq.offsets)).pin_memory()
    loss_out = np.zeros(3)
    npg.npg_set_state(ctx.h, state0)
    npg.npg_set_points(ctx.h, pts_pin, off_pin)
    npg.npg_iteration(ctx.h, loss_out)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        npg.npg_set_points(ctx.h, pts_pin, off_pin)
        npg.npg_iteration(ctx.h, loss_out)
    t_e2e = time.perf_counter() - t0
    t_e2e = max_over_ranks(t_e2e, dist)
    e2e_value = job_throughput(world, N, T, e2e_steps, t_e2e)

    peaks = load_peaks()
    # FP32 peak: unit counts at the SM clock sampled during the timed region
    # (the maximum clock when no sample was taken); the FMA probe measures the
    # same rate directly, with its own clock samples, as a cross-check
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    mhz = clocks["sm_mhz"] if clocks else 2070.0
    fp32_peak = fp32_peak_tflops(sms, mhz)
    fp32_src = (f"FP32 FMA: {sms} SMs x {FP32_LANES_PER_SM} lanes x 2 x {mhz:.0f} MHz "
                f"({'median sampled under load' if clocks else 'maximum clock'})")
    probe_sampler = ClockSampler(local)
    probe_sampler.start()
    probe = [npg.npg_fp32_fma_rate(stream) for _ in range(12)]
    probe_clk = probe_sampler.stop()
    fp32_probe = {"tflops_median": statistics.median(t for t, _ in probe),
                  "tflops_max": max(t for t, _ in probe),
                  "ms_per_launch": statistics.median(m for _, m in probe),
                  "clocks": probe_clk,
                  "derived_at_probe_clock": (fp32_peak_tflops(sms, probe_clk["sm_mhz"])
                                             if probe_clk else None)}
    work = stage_work(p, N, T, MT, (H, D, K, Z, NO), precond, args.precision, mlp.size)
    # the searches against brute force: 2 N M_t pair evaluations per frame
    # (both directions) would be needed without the grid; delivered per
    # second of the two search stages, at 8 FLOP per pair
    t_search = (stages["nn_x"] + stages["nn_p"]) * 1e-3
    bf_pairs = 2.0 * N * MT
    search["brute_force_equivalent"] = {
        "pairs": bf_pairs, "pairs_per_s": bf_pairs / t_search,
        "tflops_equivalent": 8.0 * bf_pairs / t_search / 1e12,
        "x_fp32_peak": 8.0 * bf_pairs / t_search / 1e12 / fp32_peak}
    # search work: 8 FLOP per candidate pair (3 sub, 1 mul, 2 fma, compare)
    work["nn_x"] = ("alu", 8 * search["cand_per_query_x"] * N * T, "FLOP")
    work["nn_p"] = ("alu", 8 * search["cand_per_query_p"] * MT, "FLOP")
    def roofline(stage):
        kind, amount, _ = work[stage][:3]
        dur = stages[stage] * 1e-3
        if kind == "hbm":
            ach = amount / dur / 1e9
            return {"bound": "hbm", "achieved": ach, "peak": peaks["hbm"], "unit": "GB/s",
                    "frac": ach / peaks["hbm"], "traffic": None,
                    "peak_source": f"{peaks['src']} copy bandwidth"}
        if kind == "tensor":
            ach = amount / dur / 1e12
            return {"bound": "tensor", "achieved": ach, "peak": peaks["bf16_sus"],
                    "unit": "TFLOP/s", "frac": ach / peaks["bf16_sus"], "traffic": None,
                    "peak_source": f"{peaks['src']} BF16 dense, sustained"}
        ach = amount / dur / 1e12
        return {"bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": ach / fp32_peak, "traffic": None,
                "peak_source": fp32_src}

    # the dominant kernel: the longest stage that is one kernel launch (the
    # preconditioner stage is 6 passes x levels plus Adam on concurrent lanes,
    # the search stages two kernels per direction); every stage's position is
    # listed in stage_rooflines
    wide = H > 64
    kernels = {"mlp_bwd": ("mlp_bwd_tc128_kernel" if wide else "mlp_bwd_tc2_kernel")
               if args.precision == "bf16" else
               ("wide_gemm_kernel (layered)" if wide else "mlp_bwd_fp32_kernel"),
               "decode": ("decode_tc128_kernel" if wide else "decode_tc_kernel")
               if args.precision == "bf16" else
               ("wide_gemm_kernel (layered)" if wide else "decode_fp32_kernel"),
               "encode": "encode_kernel", "scatter": "scatter_kernel"}
    dom = max(kernels, key=lambda s: stages.get(s, 0.0))
    roof = roofline(dom)
    roof["kernel"] = kernels[dom]
    roof["ms_per_launch"] = stages[dom]
    roof["traffic"] = measured_traffic(kernels[dom], args.workload)
    if dom == "mlp_bwd":
        # what the kernel also executes beyond the algorithmic backward: the
        # forward recompute of every row (not counted in `achieved`)
        roof["recompute_flop"] = work["decode"][1]
    stage_roofs = {s: {k: v for k, v in roofline(s).items() if k in ("bound", "achieved", "unit",
                                                                    "frac")}
                   for s in stages if s in work and stages[s] > 0}

    # the plain FP32 per-sequence form on the same sequence, for the ratio the
    # metric names (eager, FP32 preconditioner, from the same initial state)
    plain = None
    if args.precision == "bf16" and not args.no_fp32_leg:
        cfg3 = make_cfg(npg, p, "fp32", False, stream, e_max, "fp32")
        pctx = npg.Context(cfg3, seq, mlp, device_inputs=True)
        for _ in range(args.warmup):
            pctx.iteration()
        npg.npg_set_state(pctx.h, state0)
        steps3 = max(3, min(args.steps, 20))
        torch.cuda.synchronize()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps3):
            npg.npg_iteration(pctx.h, None)
        e1.record(stream)
        torch.cuda.synchronize()
        ms3 = e0.elapsed_time(e1)
        ms3 = max_over_ranks(ms3, dist)
        v3 = job_throughput(world, N, T, steps3, ms3 * 1e-3)
        plain = {"value": v3, "unit": UNIT, "ms_per_step": ms3 / steps3, "steps": steps3,
                 "form": "plain FP32 per-sequence (eager, FP32 preconditioner)",
                 "ratio_bf16_over_fp32": value / v3}
        pctx.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        host = cpu_info()
        res = oracle_timed(p, seq, frames=2)
        v, s, desc, used = res["all"]
        v1, s1, _, _ = res["one"]
        cpu = {"value": v, "unit": UNIT, "cores": used, "kind": "oracle", "sample": desc,
               "cpu_model": host["model"], "nproc": host["nproc"],
               "single_thread": {"value": v1, "unit": UNIT, "cores": 1,
                                 "sample_seconds": round(s1, 2)},
               "all_threads_sample_seconds": round(s, 2)}

    if rank == 0:
        form = ("batched BF16 tensor-core MLP, graph-captured" if args.precision == "bf16"
                else "plain FP32") + (" (CUDA graph)" if graph and args.precision != "bf16" else "")
        form += ", preconditioner " + ("tensor-core split BF16" if precond == "tc" else "FP32")
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16" if args.precision == "bf16" else "f32",
            "data": "synthetic (seeded capsule-figure sequence; no dataset)",
            "config": dict(config_dict(p, seq, form, graph), autotuned=(
                dict(vertex_cells=tuned[0], point_cells=tuned[1], decode_ctas_per_sm=tuned[2],
                     ball_rows_x=tuned[3], ball_rows_p=tuned[4]) if tuned else None)),
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "h2d_bytes_per_step": int(seq.points.nbytes + seq.offsets.nbytes),
                    "d2h_bytes_per_step": 24},
            "gpu_launches": int(launches),
            "roofline": roof,
            "stage_rooflines": stage_roofs,
            "stages_ms": {k: round(v, 4) for k, v in stages.items()},
            "search": {k: (round(v, 2) if isinstance(v, float) else v)
                       for k, v in search.items()},
            "plain_fp32": plain,
            "fp32_fma_probe": fp32_probe,
            "cpu_baseline": cpu,
            "clocks": clocks,
        }
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
