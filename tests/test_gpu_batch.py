"""Batched uneven sequences (npg_batch_*): several independent sequences of
different vertex, frame and point counts iterated together, each a branch of
one CUDA graph, give the same results as running each sequence on its own.

The first iteration's forward and loss are deterministic, so its loss is
compared bit for bit; later iterations follow a backward whose float atomics
sum in a varying order, and Adam's sign-like first steps turn last-bit
differences into small trajectory differences, so they are compared to 5e-2
(the same bound as graph replay against eager runs of one sequence).
"""
import time

import numpy as np
import pytest

import oracle as O
from paper_2602_22212_gb300 import inputs as I

pytestmark = pytest.mark.gpu

# (generator, subdivision, T, M per frame, seed): uneven on purpose
SPECS = [("blob", 3, 5, 1500, 0), ("figure", 4, 9, 3000, 1), ("blob", 4, 13, 5000, 2),
         ("figure", 3, 7, 2000, 3), ("blob", 2, 11, 800, 4), ("figure", 4, 6, 4000, 5)]


@pytest.fixture(scope="module")
def npg():
    from paper_2602_22212_gb300 import build
    build.build()
    from paper_2602_22212_gb300 import npg as mod
    return mod


def make_seq(gen, subdiv, T, M, seed):
    if gen == "blob":
        return I.sphere_blob(subdiv=subdiv, T=T, M=M, noise=0.005, seed=seed)
    return I.figure(subdiv=subdiv, T=T, M=M, noise_rel=0.003, seed=seed)


def contexts(npg, seqs, precision, streams, use_graph=False):
    ocfg = O.make_cfg(L=4, res=(8, 27, 45, 64), F=4, H=64, D=3, slope=0.01)
    out = []
    for k, seq in enumerate(seqs):
        mlp = I.mlp_init(O.k_in(ocfg), 64, 3, O.n_out(ocfg), seed=10 + k, zero_last=False)
        mlp[-(O.n_out(ocfg) * 64 + O.n_out(ocfg)):] *= 0.1
        cfg = npg.make_config(4, (8, 27, 45, 64), 4, 64, 3, slope=0.01, precision=precision,
                              e_max=20, w_iso=1.0, stream=streams[k], use_graph=use_graph,
                              precond_mode=npg.PRECOND_TC if precision else npg.PRECOND_FP32)
        out.append(npg.Context(cfg, seq, mlp))
    return out


@pytest.mark.parametrize("precision, width", [(0, 0), (1, 0), (1, 1), (1, 2)])
def test_batch_matches_separate_runs(npg, precision, width):
    """Every chain width (0: a branch per sequence; 1: all in one chain; 2:
    two chains of sequences assigned largest first) gives the same results."""
    import torch
    seqs = [make_seq(*s) for s in SPECS]
    S = len(seqs)
    bstreams = [torch.cuda.Stream() for _ in range(S)]
    sstreams = [torch.cuda.Stream() for _ in range(S)]
    main = torch.cuda.Stream()
    cb = contexts(npg, seqs, precision, bstreams)
    cs = contexts(npg, seqs, precision, sstreams)
    batch = npg.npg_batch_create([c.h for c in cb], main)
    npg.npg_batch_set_width(batch, width)
    try:
        for it in range(4):
            lb = np.zeros((S, 3))
            npg.npg_batch_iteration(batch, lb)
            ls = np.array([c.iteration() for c in cs])
            if it == 0:
                np.testing.assert_array_equal(lb, ls)
            else:
                np.testing.assert_allclose(lb, ls, rtol=5e-2, atol=0)
        for c in cb:
            assert npg.npg_get_epoch(c.h) == 4
            assert npg.npg_launch_count(c.h) > 0
        with pytest.raises(npg.NpgError):  # the graph is captured
            npg.npg_batch_set_width(batch, 3)
        # the contexts stay usable on their own streams after the batch
        for c in cb:
            c.forward()
            assert np.all(np.isfinite(c.loss()[0]))
    finally:
        npg.npg_batch_destroy(batch)
        for c in cb + cs:
            c.close()


def test_batch_rejects_shared_streams(npg):
    import torch
    seqs = [make_seq(*s) for s in SPECS[:2]]
    st = torch.cuda.Stream()
    cb = contexts(npg, seqs, 0, [st, st])
    try:
        with pytest.raises(npg.NpgError) as ei:
            npg.npg_batch_create([c.h for c in cb], torch.cuda.Stream())
        assert ei.value.code == npg.EINVAL
        with pytest.raises(npg.NpgError):
            npg.npg_batch_create([cb[0].h], None)
    finally:
        for c in cb:
            c.close()


def test_batch_throughput_reported(npg):
    """Sixteen small uneven sequences: one graph launch per iteration against
    sixteen graph launches one after the other (reported, and the batch must
    not be slower)."""
    import torch
    rng = np.random.default_rng(3)
    specs = [("blob" if k % 2 == 0 else "figure", int(rng.integers(2, 5)), int(rng.integers(4, 16)),
              int(rng.integers(500, 5000)), 100 + k) for k in range(16)]
    seqs = [make_seq(*s) for s in specs]
    vf = sum(s.N * s.T for s in seqs)
    streams = [torch.cuda.Stream() for _ in seqs]
    cb = contexts(npg, seqs, 1, streams)
    batch = npg.npg_batch_create([c.h for c in cb], torch.cuda.Stream())
    one_stream = torch.cuda.Stream()  # one after the other
    ones = []
    for k, seq in enumerate(seqs):
        ones.append(contexts(npg, [seq], 1, [one_stream], use_graph=True)[0])
    try:
        for _ in range(3):
            npg.npg_batch_iteration(batch)
            for c in ones:
                npg.npg_iteration(c.h)
        torch.cuda.synchronize()
        iters = 20
        t0 = time.perf_counter()
        for _ in range(iters):
            npg.npg_batch_iteration(batch)
        torch.cuda.synchronize()
        t_batch = (time.perf_counter() - t0) / iters
        t0 = time.perf_counter()
        for _ in range(iters):
            for c in ones:
                npg.npg_iteration(c.h)
        torch.cuda.synchronize()
        t_one = (time.perf_counter() - t0) / iters
        print(f"16 sequences, {vf} vertex-frames: batched {vf / t_batch:.3e} vf/s, "
              f"one by one {vf / t_one:.3e} vf/s ({t_one / t_batch:.2f}x)")
        assert t_batch <= 1.05 * t_one, (t_batch, t_one)
    finally:
        npg.npg_batch_destroy(batch)
        for c in cb + ones:
            c.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_autotune_keeps_results_exact(npg, precision):
    """npg_autotune picks each sequence's search-grid resolutions (and, for the
    BF16 form, the decode's CTAs per SM) among its candidates; the searches are
    exact at every resolution, so the first loss after tuning equals the loss
    before it bit for bit, and the tuned contexts then run as a batch."""
    import torch
    seqs = [make_seq(*s) for s in SPECS[:3]]
    streams = [torch.cuda.Stream() for _ in seqs]
    ctxs = contexts(npg, seqs, precision, streams, use_graph=bool(precision))
    for ctx in ctxs:
        ctx.forward()
        before, _ = ctx.loss()
        chosen = npg.npg_autotune(ctx.h, 2)
        assert chosen[0] >= 1 and chosen[1] >= 1
        if precision:
            assert chosen[2] in (3, 4, 6, 8)
        assert chosen[3] in (6, 12, 24, 48, 96, 192, 384) and chosen[4] in (6, 12, 24, 48, 96, 192, 384)
        ctx.forward()
        after, _ = ctx.loss()
        np.testing.assert_array_equal(after, before)
    batch = npg.npg_batch_create([c.h for c in ctxs], torch.cuda.Stream())
    out = np.zeros((len(ctxs), 3))
    for _ in range(3):
        npg.npg_batch_iteration(batch, out)
        assert np.all(np.isfinite(out))
    npg.npg_batch_destroy(batch)
    for c in ctxs:
        c.close()
