"""The BF16 tensor-core MLP path (tcgen05, FP32 accumulation) against the
FP32 path and the FP64 oracle.

BF16 keeps 8 significand bits, so each rounded activation or weight carries
a relative error up to 2^-9 = 2e-3; a 64-term dot product of such terms lands
within a few 1e-3 of its FP32 value. Tolerances:
  x-hat                 5e-3 absolute against the FP32 path (coordinates O(1))
  parameter gradients   per block (every MLP weight and bias block, every grid
                        level), from the same dL/dx-hat as the oracle, within
                        the rounding bound k u ||m|| of tests/bf16_model.py,
                        m the oracle's magnitude pass (sums of |products|): the
                        bound follows each block's cancellation
  final Chamfer         paired over 128 sequences, the mean excess over the
                        FP32 path's at most 1%
"""
import numpy as np
import pytest

import oracle as O
from paper_2602_22212_gb300 import inputs as I

from bf16_model import bf16_block_bound

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def npg():
    from paper_2602_22212_gb300 import build
    build.build()
    from paper_2602_22212_gb300 import npg as mod
    return mod


def setup(rot_mode=0, seed=1, T=8, M=4096, Fn=2, n_freq=4):
    seq = I.sphere_blob(subdiv=4, T=T, M=M, noise=0.005, seed=seed)
    ocfg = O.make_cfg(L=4, res=(8, 27, 45, 64), F=4, Fn=Fn, H=64, D=3, rot_mode=rot_mode,
                      slope=0.01, n_freq=n_freq)
    prob = O.Problem(ocfg, seq.x, seq.n, seq.faces, seq.points, seq.offsets, seq.t_key)
    return seq, ocfg, prob


def cfg_of(npg, ocfg, precision, e_max=10, **kw):
    return npg.make_config(ocfg.L, [ocfg.res[l] for l in range(ocfg.L)], ocfg.F, ocfg.H, ocfg.D,
                           slope=ocfg.slope, rot_mode=ocfg.rot_mode, e_max=e_max,
                           precision=precision, **kw)


def rand_params(ocfg, seed=2):
    rng = np.random.default_rng(seed)
    grid = rng.normal(scale=0.3, size=O.grid_len(ocfg)).astype(np.float32)
    mlp = I.mlp_init(O.k_in(ocfg), ocfg.H, ocfg.D, O.n_out(ocfg), seed=seed + 1, zero_last=False)
    mlp[-(O.n_out(ocfg) * ocfg.H + O.n_out(ocfg)):] *= 0.5
    return grid, mlp


def rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b)


@pytest.mark.parametrize("rot_mode", [0, 1, 2])
def test_bf16_decode_tracks_fp32(npg, rot_mode):
    seq, ocfg, prob = setup(rot_mode)
    grid, mlp = rand_params(ocfg)
    out = {}
    for prec in (npg.FP32, npg.BF16_MLP):
        ctx = npg.Context(cfg_of(npg, ocfg, prec), seq, mlp)
        ctx.set(npg.BUF_GRID, grid)
        ctx.forward()
        out[prec] = ctx.get(npg.BUF_XHAT).reshape(prob.T, prob.N, 3)
        ctx.close()
    d = np.abs(out[npg.BF16_MLP] - out[npg.FP32])
    assert d.max() <= 5e-3, d.max()
    disp = out[npg.FP32] - seq.x[None]
    assert rel(out[npg.BF16_MLP] - seq.x[None], disp) <= 2e-2


@pytest.mark.parametrize("subdiv", [1, 2, 3])
def test_bf16_decode_small_and_ragged_meshes(npg, subdiv):
    """Meshes of 42 vertices (fewer than a 128-row tile: every thread loads
    its own U and V rows), 162 and 642 (tiles across frame boundaries, a
    ragged last tile: the staged rows of two frames)."""
    seq = I.sphere_blob(subdiv=subdiv, T=5, M=500, noise=0.005, seed=3)
    ocfg = O.make_cfg(L=4, res=(8, 27, 45, 64), F=4, Fn=2, H=64, D=3, slope=0.01, n_freq=4)
    grid, mlp = rand_params(ocfg)
    out = {}
    for prec in (npg.FP32, npg.BF16_MLP):
        ctx = npg.Context(cfg_of(npg, ocfg, prec), seq, mlp)
        ctx.set(npg.BUF_GRID, grid)
        ctx.forward()
        out[prec] = ctx.get(npg.BUF_XHAT).reshape(seq.T, seq.N, 3)
        ctx.close()
    assert np.abs(out[npg.BF16_MLP] - out[npg.FP32]).max() <= 5e-3


def test_bf16_identity_initialisation_exact(npg):
    seq, ocfg, prob = setup(T=3, M=500)
    mlp = I.mlp_init(O.k_in(ocfg), ocfg.H, ocfg.D, O.n_out(ocfg), seed=0)
    ctx = npg.Context(cfg_of(npg, ocfg, npg.BF16_MLP), seq, mlp)
    ctx.forward()
    xh = ctx.get(npg.BUF_XHAT).reshape(3, seq.N, 3)
    for t in range(3):
        np.testing.assert_array_equal(xh[t], seq.x)
    ctx.close()


def _backprop_vs_oracle(npg, seq, ocfg, prob, **kw):
    import torch
    grid, mlp = rand_params(ocfg)
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    ref = O.loss_full(prob, f32(grid), f32(mlp), 3, 10, decide_f32=True)
    gx32 = ref["g_xhat"].astype(np.float32)
    want_g, want_m = O.backprop(prob, f32(grid), f32(mlp), f32(gx32))
    mag_g, mag_m = O.backprop(prob, f32(grid), f32(mlp), f32(gx32), magnitude=True)
    ctx = npg.Context(cfg_of(npg, ocfg, npg.BF16_MLP, **kw), seq, mlp)
    ctx.set(npg.BUF_GRID, grid)
    npg.npg_set_epoch(ctx.h, 3)
    ctx.forward()
    npg.npg_backprop(ctx.h, torch.from_numpy(gx32.reshape(-1)).cuda())
    gg = ctx.get(npg.BUF_GRID_GRAD).astype(np.float64)
    gm = ctx.get(npg.BUF_MLP_GRAD).astype(np.float64)
    H, D, K, NO = 64, 3, O.k_in(ocfg), O.n_out(ocfg)
    off = 0
    for name, n in [("W1", H * K), ("b1", H), ("W2", H * H), ("b2", H), ("W3", H * H),
                    ("b3", H), ("Wo", NO * H), ("bo", NO)]:
        sl = slice(off, off + n)
        err, bound = np.linalg.norm(gm[sl] - want_m[sl]), bf16_block_bound(mag_m[sl])
        assert err <= bound, (name, err, bound, rel(gm[sl], want_m[sl]))
        off += n
    for l in range(ocfg.L + 1):
        a = O.level_offset(ocfg, l)
        b = O.level_offset(ocfg, l + 1) if l < ocfg.L else O.grid_len(ocfg)
        err, bound = np.linalg.norm(gg[a:b] - want_g[a:b]), bf16_block_bound(mag_g[a:b])
        assert err <= bound, (l, err, bound, rel(gg[a:b], want_g[a:b]))
    ctx.close()


@pytest.mark.parametrize("rot_mode", [0, 1, 2])
def test_bf16_backprop_vs_oracle(npg, rot_mode):
    seq, ocfg, prob = setup(rot_mode)
    _backprop_vs_oracle(npg, seq, ocfg, prob)


def test_bf16_backprop_ragged_tiles(npg):
    """Tiles cut by both ends: N = 2562 leaves 2 vertices in the last block of
    16, T = 5 fills 5 of the 8 frames, and Z = 5, 2M = 6 make the last
    block's z run (2 x 5 floats) and every gamma run (5 x 6 floats) miss a
    16-byte multiple, so the staged copies take their rounded, padded form."""
    seq, ocfg, prob = setup(0, T=5, Fn=1, n_freq=3)
    assert seq.N % 16 == 2 and O.k_in(ocfg) == 11
    _backprop_vs_oracle(npg, seq, ocfg, prob, F_n=1, n_freq=3)


_FINAL_RUNS = 128
_FINAL_ITERS = 500
_final_cache = {}


def final_chamfer(npg, precision, precond, seed):
    """Mean Chamfer distance (cd_t averaged over frames and over the last 10
    iterations) after a full run from the identity initialisation on the
    articulated figure with sequence seed `seed`."""
    key = (precision, precond, seed)
    if key not in _final_cache:
        seq = I.figure(subdiv=4, T=8, M=4096, noise_rel=0.003, seed=seed)
        ocfg = O.make_cfg(L=4, res=(8, 27, 45, 64), F=4, H=64, D=3, slope=0.01, w_iso=1.0)
        mlp = I.mlp_init(O.k_in(ocfg), ocfg.H, ocfg.D, O.n_out(ocfg), seed=seed)
        ctx = npg.Context(cfg_of(npg, ocfg, precision, e_max=_FINAL_ITERS, w_iso=1.0,
                                 precond_mode=precond), seq, mlp)
        tail = []
        for k in range(_FINAL_ITERS):
            ctx.iteration()
            if k >= _FINAL_ITERS - 10:
                tail.append(ctx.get(npg.BUF_CD).mean())
        ctx.close()
        _final_cache[key] = float(np.mean(tail))
    return _final_cache[key]


@pytest.mark.parametrize("precond", [0, 1])
def test_bf16_final_chamfer_within_one_percent_of_fp32(npg, precond):
    """Full 500-iteration runs (the paper's schedules are 250 and 1000) on
    128 articulated-figure sequences, FP32 against BF16 (with the FP32 or the
    tensor-core preconditioner). A single run's final Chamfer is not
    reproducible to 1%, even in FP32: the gradient's float atomics sum in a
    varying order and Adam's sign-like steps carry their last-bit differences
    into a different trajectory (a heavy-tailed spread per run, up to ~18%).
    So the comparison is paired per sequence and averaged over enough
    sequences that the mean's standard error (~0.45%) is well inside the 1%:
    the BF16 runs' mean relative excess over FP32 must be at most 1% (measured:
    -1.15% and -1.33%, standard errors 0.51% and 0.50%). The isometry weight
    is 1: on this synthetic data w_iso = 100 makes the isometry term dominate
    L_def and the paper's per-level learning rates diverge."""
    ratios = []
    for seed in range(_FINAL_RUNS):
        f = final_chamfer(npg, npg.FP32, 0, seed)
        b = final_chamfer(npg, npg.BF16_MLP, precond, seed)
        ratios.append(b / f - 1.0)
    ratios = np.array(ratios)
    se = ratios.std(ddof=1) / np.sqrt(len(ratios))
    print("BF16/FP32 - 1 per sequence:", np.round(ratios, 4), "mean %.4f se %.4f" % (
        ratios.mean(), se))
    assert ratios.mean() <= 0.01, (ratios.mean(), se)
