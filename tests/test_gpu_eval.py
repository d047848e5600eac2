"""Evaluation metrics on the GPU (npg_evaluate) against the FP64 oracle's
definitions (oracle.evaluate), on the GPU's own x-hat.

Tolerances: cd, nc and corr 1e-5 relative (FP32 distances and normals,
FP64 sums); precision and recall within 2 / N (F-score 4 / N), since a
distance within FP32 rounding of the threshold may fall on either side of it.
"""
import numpy as np
import pytest

import oracle as O
from paper_2602_22212_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def npg():
    from paper_2602_22212_gb300 import build
    build.build()
    from paper_2602_22212_gb300 import npg as mod
    return mod


def setup(npg, rot_mode, seed):
    seq = I.figure(subdiv=4, T=6, M=3000, noise_rel=0.003, seed=seed)
    ocfg = O.make_cfg(L=4, res=(8, 27, 45, 64), F=4, H=64, D=3, rot_mode=rot_mode, slope=0.01)
    cfg = npg.make_config(4, (8, 27, 45, 64), 4, 64, 3, slope=0.01, rot_mode=rot_mode)
    return seq, ocfg, cfg


def test_identity_frame_is_perfect(npg):
    """From the identity initialisation every frame decodes to the reference
    mesh, which is the keyframe's ground truth: (0, 1, 1, 1, 1, 0) there."""
    seq, ocfg, cfg = setup(npg, 0, 1)
    mlp = I.mlp_init(O.k_in(ocfg), 64, 3, O.n_out(ocfg), seed=0)
    ctx = npg.Context(cfg, seq, mlp)
    ctx.forward()
    m = npg.npg_evaluate(ctx.h, seq.gt_frames.astype(np.float32))
    k = seq.t_key
    assert m[k, 0] == 0.0 and m[k, 5] == 0.0
    np.testing.assert_array_equal(m[k, 1:4], [1.0, 1.0, 1.0])
    assert abs(m[k, 4] - 1.0) <= 1e-6
    np.testing.assert_allclose(m[-1], m[:-1].mean(0), rtol=1e-12)
    ctx.close()


@pytest.mark.parametrize("rot_mode", [0, 1])
def test_metrics_match_oracle(npg, rot_mode):
    import torch
    seq, ocfg, cfg = setup(npg, rot_mode, 2)
    rng = np.random.default_rng(3)
    mlp = I.mlp_init(O.k_in(ocfg), 64, 3, O.n_out(ocfg), seed=4, zero_last=False)
    mlp[-(O.n_out(ocfg) * 64 + O.n_out(ocfg)):] *= 0.05
    ctx = npg.Context(cfg, seq, mlp)
    ctx.set(npg.BUF_GRID, rng.normal(scale=0.3, size=O.grid_len(ocfg)).astype(np.float32))
    ctx.forward()
    T, N = seq.T, seq.N
    xh = ctx.get(npg.BUF_XHAT).reshape(T, N, 3).astype(np.float64)
    gt = seq.gt_frames.astype(np.float32)
    for tau_rel in (0.005, 0.02):
        got = npg.npg_evaluate(ctx.h, gt, tau_rel)
        dev = npg.npg_evaluate(ctx.h, torch.from_numpy(gt).cuda(), tau_rel)
        np.testing.assert_array_equal(got, dev)
        want = O.evaluate(xh, gt.astype(np.float64), seq.faces, tau_rel)
        for c in (0, 4, 5):
            np.testing.assert_allclose(got[:T, c], want[:, c], rtol=1e-5)
        for c in (1, 2):
            np.testing.assert_allclose(got[:T, c], want[:, c], atol=2.0 / N)
        np.testing.assert_allclose(got[:T, 3], want[:, 3], atol=4.0 / N)
        assert np.all(want[:, 3] > 0) or tau_rel == 0.005
    ctx.close()


def test_keyframe_selection_matches_oracle(npg):
    """Keyframe selection (npg_select_keyframe) against oracle.select_keyframe
    on the same FP32 clouds, from host and from device memory: extents within
    1e-12 relative (FP64 sums in another order), the same frame unless two
    weighted extents agree within that tolerance."""
    import torch
    rng = np.random.default_rng(11)
    seq = I.figure(subdiv=3, T=13, M=2500, noise_rel=0.003, seed=4)
    sizes = rng.integers(1, 3000, size=9)
    sizes[3] = 1
    ragged = [(rng.normal(size=(n, 3)) * rng.uniform(0.2, 0.9)).astype(np.float32) for n in sizes]
    cases = [(seq.points.astype(np.float32), seq.offsets.astype(np.int64)),
             (np.concatenate(ragged), np.cumsum([0] + list(sizes)).astype(np.int64)),
             (ragged[0], np.array([0, len(ragged[0])], np.int64))]
    for pts, off in cases:
        for bias in (0.0, 0.5, 1.0):
            want_t, want_e = O.select_keyframe(pts.astype(np.float64), off, bias)
            T = len(off) - 1
            tt = np.arange(T) / (T - 1) if T > 1 else np.full(1, 0.5)
            w = 1.0 - bias * np.abs(tt - 0.5)
            for dev in (False, True):
                if dev:
                    got_t, got_e = npg.npg_select_keyframe(torch.from_numpy(pts).cuda(),
                                                           torch.from_numpy(off).cuda(), bias)
                else:
                    got_t, got_e = npg.npg_select_keyframe(pts, off, bias)
                np.testing.assert_allclose(got_e, want_e, rtol=1e-12)
                if got_t != want_t:
                    s = w * want_e
                    assert abs(s[got_t] - s[want_t]) <= 1e-12 * s[want_t], (got_t, want_t)

