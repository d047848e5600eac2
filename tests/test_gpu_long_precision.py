"""Precision of the long-sequence workload against the FP64 oracle: the
capsule figure with N = 20000 vertices, T = 1000 frames of M = 10000 points,
an 8-level grid 16 -> 256 with F = 4 and a 3 x 128 MLP, optimised for its 300
iterations in the BF16 form (tcgen05 MLP, tensor-core preconditioner, CUDA
graph). At the final parameters, the loss, the per-frame Chamfer distances
and every parameter block's gradient are evaluated on the ten frames
{0, 111, ..., 999} by the GPU (BF16 and FP32 forms) and by the oracle (FP64,
FP64 nearest-neighbour decisions). Those frames have t~ = k / 9, so a
ten-frame sequence of them has the same time encoding as the full one; its
keyframe is frame 555 (index 5) and e = e_max, where every confidence weight
is 1.

The errors are printed (they are the precision report) and bounded:
  cd_t           the Chamfer terms: BF16 within 1e-2 relative, FP32 within 1e-5
  loss           FP32 within 1e-5; BF16 within 2e-2: near convergence the
                 isometry term is a mean of |edge length - keyframe length|
                 over differences of a few 1e-4, about the size of the BF16
                 decode's error in x-hat, so it carries most of the loss error
  gradients      BF16 within the rounding bound of tests/bf16_model.py per
                 block; FP32 within 1e-2 per block: at a converged state the
                 gradient is a sum of strongly cancelling terms, and the FP32
                 and FP64 forms take some |.| signs of Eq. 13 and some nearest
                 neighbours differently where the two candidates are within
                 rounding of each other (the arithmetic itself is checked to
                 1e-4 from a shared dL/dx-hat in the other parity tests)
"""
import numpy as np
import pytest

import oracle as O
from paper_2602_22212_gb300 import inputs as I

from bf16_model import bf16_block_bound

pytestmark = pytest.mark.gpu

FRAMES = [111 * k for k in range(10)]


@pytest.fixture(scope="module")
def npg():
    from paper_2602_22212_gb300 import build
    build.build()
    from paper_2602_22212_gb300 import npg as mod
    return mod


def subset(seq, frames, t_key):
    pts = [seq.points[seq.offsets[t]:seq.offsets[t + 1]] for t in frames]
    off = np.cumsum([0] + [len(p) for p in pts]).astype(np.int64)

    class Sub:
        pass
    s = Sub()
    s.x, s.n, s.faces, s.N = seq.x, seq.n, seq.faces, seq.N
    s.points, s.offsets, s.T, s.t_key = np.concatenate(pts), off, len(frames), t_key
    return s


def test_long_sequence_precision_against_fp64(npg):
    import torch
    p = I.preset("long")
    seq = I.make_sequence(p, seed=0)
    H, D, K, NO = p["H"], p["D"], 2 + p["F"] + 8, 7
    mlp0 = I.mlp_init(K, H, D, NO, seed=0)
    stream = torch.cuda.Stream()
    cfg = npg.make_config(p["L"], p["res"], p["F"], H, D, slope=p["slope"],
                          precision=npg.BF16_MLP, e_max=p["iters"], use_graph=True,
                          stream=stream, w_iso=p["w_iso"], precond_mode=npg.PRECOND_TC)
    ctx = npg.Context(cfg, seq, mlp0, device_inputs=True)
    first = ctx.iteration()
    for _ in range(p["iters"] - 1):
        last = ctx.iteration()
    cd_full = ctx.get(npg.BUF_CD)
    grid = ctx.get(npg.BUF_GRID)
    mlp = ctx.get(npg.BUF_MLP)
    ctx.close()
    print(f"\nlong BF16 run: loss {first[0]:.4e} -> {last[0]:.4e} over {p['iters']} iterations; "
          f"mean Chamfer of the last forward {cd_full.mean():.4e}")
    assert last[1] < first[1]

    sub = subset(seq, FRAMES, 5)
    ocfg = O.make_cfg(L=p["L"], res=p["res"], F=p["F"], H=H, D=D, slope=p["slope"],
                      w_iso=p["w_iso"])
    prob = O.Problem(ocfg, sub.x, sub.n, sub.faces, sub.points, sub.offsets, sub.t_key)
    g64 = grid.astype(np.float64)
    m64 = mlp.astype(np.float64)
    ref = O.loss_full(prob, g64, m64, p["iters"], p["iters"], decide_f32=False)
    mag_g, mag_m = O.backprop(prob, g64, m64, ref["g_xhat"], magnitude=True)
    report = {}
    for name, prec in (("bf16", npg.BF16_MLP), ("fp32", npg.FP32)):
        c = npg.make_config(p["L"], p["res"], p["F"], H, D, slope=p["slope"], precision=prec,
                            e_max=p["iters"], w_iso=p["w_iso"],
                            precond_mode=npg.PRECOND_TC if prec == npg.BF16_MLP
                            else npg.PRECOND_FP32)
        sc = npg.Context(c, sub, mlp)
        sc.set(npg.BUF_GRID, grid)
        npg.npg_set_epoch(sc.h, p["iters"])
        sc.forward()
        loss, cd = sc.loss()
        sc.backward()
        gg = sc.get(npg.BUF_GRID_GRAD).astype(np.float64)
        gm = sc.get(npg.BUF_MLP_GRAD).astype(np.float64)
        sc.close()
        rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
        blocks = {}
        o = 0
        for bn, n in [("W1", H * K), ("b1", H), ("W2", H * H), ("b2", H), ("W3", H * H),
                      ("b3", H), ("Wo", NO * H), ("bo", NO)]:
            blocks[bn] = (rel(gm[o:o + n], ref["g_mlp"][o:o + n]),
                          float(np.linalg.norm(gm[o:o + n] - ref["g_mlp"][o:o + n])),
                          bf16_block_bound(mag_m[o:o + n]))
            o += n
        for l in range(ocfg.L + 1):
            a = O.level_offset(ocfg, l)
            b = O.level_offset(ocfg, l + 1) if l < ocfg.L else O.grid_len(ocfg)
            blocks[f"grid{l}"] = (rel(gg[a:b], ref["g_grid"][a:b]),
                                  float(np.linalg.norm(gg[a:b] - ref["g_grid"][a:b])),
                                  bf16_block_bound(mag_g[a:b]))
        report[name] = dict(
            loss_rel=abs(loss[0] - ref["loss"]) / ref["loss"],
            ldef_rel=abs(loss[1] - ref["L_def"]) / ref["L_def"],
            liso_rel=abs(loss[2] - ref["L_iso"]) / ref["L_iso"],
            cd_rel_max=float(np.max(np.abs(cd - ref["cd"]) / ref["cd"])),
            mean_cd_rel=abs(cd.mean() - ref["cd"].mean()) / ref["cd"].mean(),
            grad_rel=blocks)
        r = report[name]
        print(f"{name}: loss rel err {r['loss_rel']:.3e} (L_def {r['ldef_rel']:.3e}, "
              f"L_iso {r['liso_rel']:.3e}), cd_t max rel err {r['cd_rel_max']:.3e}, "
              f"mean cd rel err {r['mean_cd_rel']:.3e}")
        print("  gradient rel err per block: " +
              ", ".join(f"{k} {v[0]:.2e}" for k, v in blocks.items()))
    b, f = report["bf16"], report["fp32"]
    print("  (L_def, L_iso of the oracle: %.4e, %.4e)" % (ref["L_def"], ref["L_iso"]))
    assert b["cd_rel_max"] <= 1e-2 and b["loss_rel"] <= 2e-2
    assert f["loss_rel"] <= 1e-5 and f["cd_rel_max"] <= 1e-5
    for k, (relerr, err, bound) in b["grad_rel"].items():
        assert err <= bound, (k, relerr, err, bound)
    for k, (relerr, err, bound) in f["grad_rel"].items():
        assert relerr <= 1e-2, (k, relerr)
