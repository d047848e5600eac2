"""The torch.autograd.Function over the C ABI (forward + loss, and the
hand-written adjoint as its backward) against central finite differences of
the GPU's own loss.

Finite differences see every dependence of L on the parameters, while the
adjoint follows the paper's stop-gradients (confidence weights, keyframe edge
lengths). The test therefore runs where those are constant: at e = e_max the
confidence exponent 1 - sqrt(e / e_max) is 0, so every w_t = 1, and w_iso = 0
(the isometry term and the stop-gradients are checked against the oracle's
analytic gradient, which holds them fixed, in test_gpu_parity.py). FD steps of
1e-3 (grid) and 1e-4 (MLP): the derivative along the gradient and along random-sign combinations
of the 256 largest gradient entries (grid and MLP), and of the 32 single
parameters with the largest gradients (derivatives far below the FP32
rounding of one loss evaluation carry no information).
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


@pytest.mark.parametrize("rot_mode", [0, 1, 2])
def test_autograd_function_matches_central_differences(npg, rot_mode):
    import torch
    seq = I.sphere_blob(subdiv=4, T=8, M=4096, noise=0.005, seed=5)
    ocfg = O.make_cfg(L=4, res=(8, 27, 45, 64), F=2, H=64, D=2, rot_mode=rot_mode, slope=0.01)
    rng = np.random.default_rng(6)
    grid0 = rng.normal(scale=0.2, size=O.grid_len(ocfg))
    mlp0 = I.mlp_init(O.k_in(ocfg), ocfg.H, ocfg.D, O.n_out(ocfg), seed=7, zero_last=False)
    mlp0[-(O.n_out(ocfg) * ocfg.H + O.n_out(ocfg)):] *= 0.3
    e_max = 10
    cfg = npg.make_config(ocfg.L, [ocfg.res[l] for l in range(ocfg.L)], ocfg.F, ocfg.H, ocfg.D,
                          slope=ocfg.slope, rot_mode=rot_mode, e_max=e_max, w_iso=0.0)
    ctx = npg.Context(cfg, seq, mlp0)
    npg.npg_set_epoch(ctx.h, e_max)
    fn = npg.npg_loss_fn()
    dev = torch.device("cuda")
    grid = torch.tensor(grid0, dtype=torch.float32, device=dev, requires_grad=True)
    mlp = torch.tensor(mlp0, dtype=torch.float32, device=dev, requires_grad=True)
    loss = fn.apply(grid, mlp, ctx.h)
    loss.backward()
    gg = grid.grad.double().cpu().numpy()
    gm = mlp.grad.double().cpu().numpy()
    assert np.linalg.norm(gg) > 0 and np.linalg.norm(gm) > 0

    def L(g, m):
        with torch.no_grad():
            return float(fn.apply(torch.tensor(g, dtype=torch.float32, device=dev),
                                  torch.tensor(m, dtype=torch.float32, device=dev), ctx.h))

    for name, g0, gvec in (("grid", grid0, gg), ("mlp", mlp0, gm)):
        # an MLP parameter moves whole frames (an output-layer weight moves
        # every vertex), and nearest-neighbour choices that switch within the
        # step make the loss only piecewise smooth: smaller steps there
        eps = 1e-3 if name == "grid" else 1e-4
        def Ld(d, h):
            if name == "grid":
                return (L(g0 + h * d, mlp0) - L(g0 - h * d, mlp0)) / (2 * h)
            return (L(grid0, g0 + h * d) - L(grid0, g0 - h * d)) / (2 * h)
        gn = np.linalg.norm(gvec)
        # along the gradient: the derivative is |g|
        fd = Ld(gvec / gn, eps)
        assert abs(fd - gn) <= 2e-3 * gn, (name, "gradient direction", fd, gn)
        # random-sign combinations of the 256 largest entries
        top = np.argsort(-np.abs(gvec))[:256]
        for k in range(3):
            d = np.zeros_like(g0)
            d[top] = rng.choice([-1.0, 1.0], size=len(top))
            d /= np.linalg.norm(d)
            fd, an = Ld(d, eps), float(gvec @ d)
            assert abs(fd - an) <= 1e-2 * abs(an) + 2e-3 * gn, (name, k, fd, an)
        # single parameters: the 32 with the largest gradients (a derivative
        # below the loss's FP32 rounding would say nothing); the whole step
        # lands on one parameter (an output bias turns every vertex of every
        # frame), so nearest-neighbour switches weigh more: 10% of the entry
        for k in top[:32]:
            d = np.zeros_like(g0)
            d[k] = 1.0
            fd = Ld(d, eps)
            assert abs(fd - gvec[k]) <= 1e-1 * abs(gvec[k]) + 2e-3 * gn, (name, k, fd, gvec[k])
    ctx.close()
