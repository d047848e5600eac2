"""Pins of the FP64 oracle against things other than itself.

Each test pins one part of the oracle to a closed form, an invariant the paper
states, a library routine computing the same textbook quantity, a hand-worked
example (tests/golden/) or brute force / finite differences, so that a dropped
term, a wrong sign or index or a transposed operand fails at least one test.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2602_22212_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def small_cfg(rot_mode=0, slope=0.01, F=2, L=2, res=(3, 5), H=8, D=2):
    return O.make_cfg(L=L, res=res, F=F, Fn=2, rn=4, H=H, D=D, rot_mode=rot_mode, slope=slope)


# ---------------------------------------------------------------- Sec. 3.2

def test_trilinear_matches_scipy_regular_grid_interpolator():
    """Sec. 3.2: trilinear lookup == scipy's linear RegularGridInterpolator."""
    from scipy.interpolate import RegularGridInterpolator
    rng = np.random.default_rng(1)
    for r in (2, 3, 7, 16):
        cfg = O.make_cfg(L=1, res=(r,), F=3, Fn=1, rn=2)
        G = rng.normal(size=(r, r, r, 3))            # [iz, iy, ix, f]
        gn = np.zeros(2 * 2 * 2 * 1)
        grid = np.concatenate([G.ravel(), gn])
        ax = np.linspace(-1, 1, r)
        x = rng.uniform(-1, 1, size=(200, 3))
        x[:5] = [[-1, -1, -1], [1, 1, 1], [1, -1, 1], [0, 0, 0], [-1, 1, 0.3]]
        z = O.encode(cfg, x, np.zeros_like(x), grid)[:, 1:]
        for f in range(3):
            ip = RegularGridInterpolator((ax, ax, ax), G[..., f], method="linear")
            ref = ip(x[:, ::-1])  # (z, y, x) order
            np.testing.assert_allclose(z[:, f], ref, rtol=0, atol=1e-12)


def test_trilinear_weights_partition_of_unity_and_node_values():
    rng = np.random.default_rng(2)
    for r in (2, 5, 9):
        for _ in range(50):
            p = rng.uniform(-1, 1, 3)
            idx, w = O.trilinear(r, p)
            assert abs(w.sum() - 1.0) < 1e-14
            assert np.all(w >= -1e-15) and np.all(idx >= 0) and np.all(idx < r ** 3)
        # at a node, the node's own weight is 1
        k = (1, r - 1, 0)
        p = np.array([-1 + 2 * k[0] / (r - 1), -1 + 2 * k[1] / (r - 1), -1 + 2 * k[2] / (r - 1)])
        idx, w = O.trilinear(r, p)
        node = (k[2] * r + k[1]) * r + k[0]
        assert abs(w[list(idx).index(node)] - 1.0) < 1e-12 if node in idx else False


def test_level_mean_reproduces_affine_field():
    """Eq. 1: averaging L levels that all hold the same affine field gives it back."""
    rng = np.random.default_rng(3)
    res = (2, 4, 9)
    F = 2
    cfg = O.make_cfg(L=3, res=res, F=F, Fn=2, rn=4)
    A = rng.normal(size=(F, 3))
    b = rng.normal(size=F)
    parts = []
    for r in res:
        ax = np.linspace(-1, 1, r)
        Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")
        P = np.stack([X, Y, Z], -1).reshape(-1, 3)
        parts.append((P @ A.T + b).ravel())
    An = rng.normal(size=(2, 3))
    ax = np.linspace(-1, 1, 4)
    Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")
    P = np.stack([X, Y, Z], -1).reshape(-1, 3)
    parts.append((P @ An.T).ravel())
    grid = np.concatenate(parts)
    assert len(grid) == O.grid_len(cfg)
    x = rng.uniform(-1, 1, size=(100, 3))
    n = rng.normal(size=(100, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    z = O.encode(cfg, x, n, grid)
    np.testing.assert_allclose(z[:, 2:], x @ A.T + b, atol=1e-12)
    np.testing.assert_allclose(z[:, :2], n @ An.T, atol=1e-12)


# ---------------------------------------------------------------- Sec. 3.3

def test_time_embedding_golden():
    g = _gold("time_embedding.json")
    cfg = small_cfg()
    gam = O.time_embedding(cfg, g["T"])
    for t, row in g["rows"].items():
        np.testing.assert_allclose(gam[int(t)], row, atol=1e-15)
    # T = 1 means t~ = 0
    np.testing.assert_allclose(O.time_embedding(cfg, 1)[0], g["rows"]["0"], atol=0)


@pytest.mark.parametrize("slope", [0.0, 0.01, 0.2])
def test_mlp_matches_torch_nn(slope):
    """Sec. 3.3, Eq. 4: the oracle MLP == a torch.nn FP64 stack with the same weights."""
    torch = pytest.importorskip("torch")
    cfg = O.make_cfg(L=1, res=(3,), F=4, H=16, D=3, slope=slope)
    K, H, No = O.k_in(cfg), 16, O.n_out(cfg)
    mlp = I.mlp_init(K, H, 3, No, seed=5, zero_last=False).astype(np.float64)
    rng = np.random.default_rng(6)
    y = rng.normal(size=(37, K))
    o = O.mlp_forward(cfg, mlp, y)
    layers = []
    dims = [(H, K), (H, H), (H, H), (No, H)]
    off = 0
    for li, (fo, fi) in enumerate(dims):
        lin = torch.nn.Linear(fi, fo).double()
        with torch.no_grad():
            lin.weight.copy_(torch.from_numpy(mlp[off:off + fo * fi].reshape(fo, fi)))
            off += fo * fi
            lin.bias.copy_(torch.from_numpy(mlp[off:off + fo]))
            off += fo
        layers.append(lin)
        if li < 3:
            layers.append(torch.nn.LeakyReLU(slope) if slope > 0 else torch.nn.ReLU())
    assert off == len(mlp) == O.mlp_len(cfg)
    ref = torch.nn.Sequential(*layers)(torch.from_numpy(y)).detach().numpy()
    np.testing.assert_allclose(o, ref, rtol=1e-13, atol=1e-14)


# ---------------------------------------------------------------- Sec. 3.4

def test_quaternion_rotation_matches_scipy():
    """Eq. 5-6: R((1+q_w, q_x, q_y, q_z)/norm) == scipy's quaternion rotation; d = tanh(0.1 d)."""
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(7)
    cfg = small_cfg(rot_mode=0)
    for _ in range(50):
        o = rng.normal(scale=0.7, size=7)
        R, d = O.rotation_translation(cfg, o)
        q = np.array([1 + o[0], o[1], o[2], o[3]])
        ref = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        np.testing.assert_allclose(R, ref, atol=1e-14)
        np.testing.assert_allclose(R.T @ R, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(R) - 1) < 1e-14
        np.testing.assert_allclose(d, np.tanh(0.1 * o[4:]), atol=1e-16)
    R, d = O.rotation_translation(cfg, np.array([0, 0, 0, 0, 10.0, -10.0, 0]))
    np.testing.assert_array_equal(R, np.eye(3))
    np.testing.assert_allclose(d, [0.7615941559557649, -0.7615941559557649, 0.0], atol=1e-16)
    # 90 degrees about z maps e_x to e_y: q = (cos 45, 0, 0, sin 45)
    c = np.sqrt(0.5)
    R, _ = O.rotation_translation(cfg, np.array([c - 1, 0, 0, c, 0, 0, 0]))
    np.testing.assert_allclose(R @ [1, 0, 0], [0, 1, 0], atol=1e-15)


def test_expmap_rotation_matches_scipy_and_quaternion():
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(8)
    ce = small_cfg(rot_mode=1)
    cq = small_cfg(rot_mode=0)
    for scale in (1e-7, 1e-3, 5e-3, 2e-2, 0.5, 2.0):
        for _ in range(10):
            w = rng.normal(size=3)
            w *= scale / np.linalg.norm(w)
            o = np.concatenate([w, rng.normal(size=3)])
            R, d = O.rotation_translation(ce, o)
            np.testing.assert_allclose(R, Rotation.from_rotvec(w).as_matrix(), atol=2e-15)
            np.testing.assert_allclose(d, np.tanh(0.1 * o[3:]), atol=1e-16)
            th = np.linalg.norm(w)
            a = w / th
            oq = np.array([np.cos(th / 2) - 1, *(np.sin(th / 2) * a), 0, 0, 0])
            Rq, _ = O.rotation_translation(cq, oq)
            np.testing.assert_allclose(R, Rq, atol=2e-15)


def test_cayley_rotation_matches_its_definition():
    """Rotation ablation (Sec. 4): the Cayley transform R = (I - K)^-1 (I + K),
    K = [w]x, here by a linear solve, against the oracle's closed form; R is
    orthonormal with det 1, the identity at w = 0, and a rotation by
    2 atan(|w|) about w (the Cayley transform's angle)."""
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(9)
    cc = small_cfg(rot_mode=2)
    R0, _ = O.rotation_translation(cc, np.zeros(6))
    np.testing.assert_array_equal(R0, np.eye(3))
    for scale in (1e-6, 0.1, 1.0, 5.0):
        for _ in range(10):
            w = rng.normal(size=3)
            w *= scale / np.linalg.norm(w)
            o = np.concatenate([w, rng.normal(size=3)])
            R, d = O.rotation_translation(cc, o)
            K = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
            want = np.linalg.solve(np.eye(3) - K, np.eye(3) + K)
            np.testing.assert_allclose(R, want, atol=1e-14)
            np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-14)
            assert abs(np.linalg.det(R) - 1.0) < 1e-13
            ang = 2 * np.arctan(np.linalg.norm(w))
            rv = w / np.linalg.norm(w) * ang
            np.testing.assert_allclose(R, Rotation.from_rotvec(rv).as_matrix(), atol=1e-13)
            np.testing.assert_allclose(d, np.tanh(0.1 * o[3:]), atol=1e-16)


def test_identity_at_initialisation():
    """Sec. 3.1: zero grids and a zeroed last layer give x-hat == x exactly."""
    seq = I.random_cloud_sequence(T=3)
    for rot in (0, 1, 2):
        cfg = small_cfg(rot_mode=rot)
        grid = np.zeros(O.grid_len(cfg))
        mlp = I.mlp_init(O.k_in(cfg), cfg.H, cfg.D, O.n_out(cfg), seed=0)
        z = O.encode(cfg, seq.x, seq.n, grid)
        xh = O.decode(cfg, seq.x.astype(np.float64), z, O.time_embedding(cfg, 3), mlp)
        for t in range(3):
            np.testing.assert_array_equal(xh[t], seq.x.astype(np.float64))


# ---------------------------------------------------------------- Sec. 3.5 Chamfer

def test_nn_matches_kdtree_and_tie_rule():
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(9)
    q = rng.uniform(-1, 1, size=(300, 3))
    c = rng.uniform(-1, 1, size=(500, 3))
    idx, d = O.nn(q, c)
    dd, ii = cKDTree(c).query(q)
    np.testing.assert_array_equal(idx, ii)
    np.testing.assert_allclose(d, dd ** 2, rtol=1e-12)
    # FP32 decision on float inputs: same answer except within float rounding
    qf, cf = q.astype(np.float32).astype(np.float64), c.astype(np.float32).astype(np.float64)
    i32, d32 = O.nn(qf, cf, decide_f32=True)
    i64, d64 = O.nn(qf, cf, decide_f32=False)
    bad = i32 != i64
    assert np.all(np.abs(d32[bad] - d64[bad]) <= 1e-6)
    # exact duplicates: the lowest index wins in both precisions
    c2 = np.concatenate([c[:10], c[:10]])
    for f32 in (False, True):
        i2, _ = O.nn(c2[:10] + 1e-3, c2, decide_f32=f32)
        assert np.all(i2 < 10)


def test_chamfer_invariants():
    rng = np.random.default_rng(10)
    X = rng.uniform(-1, 1, size=(1, 50, 3))
    off = np.array([0, 50])
    assert O.chamfer(X, off, X[0])[4][0] == 0.0
    P = rng.uniform(-1, 1, size=(70, 3))
    cd = O.chamfer(X, np.array([0, 70]), P)[4][0]
    cd_sw = O.chamfer(P[None], np.array([0, 50]), X[0])[4][0]
    assert abs(cd - cd_sw) < 1e-14
    perm = rng.permutation(70)
    assert abs(O.chamfer(X, np.array([0, 70]), P[perm])[4][0] - cd) < 1e-14
    s = np.array([0.3, -0.2, 0.1])
    assert abs(O.chamfer(X + s, np.array([0, 70]), P + s)[4][0] - cd) < 1e-12
    from scipy.spatial import cKDTree
    ref = np.mean(cKDTree(P).query(X[0])[0] ** 2) + np.mean(cKDTree(X[0]).query(P)[0] ** 2)
    assert abs(cd - ref) < 1e-13


def test_chamfer_from_given_indices_and_thread_count():
    """cd from given nearest-neighbour choices: with the cKDTree choices it is
    the Chamfer distance; any other choice only raises it. The brute-force
    search returns the same indices on 1 and on all host threads."""
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(14)
    X = rng.uniform(-1, 1, size=(2, 60, 3))
    P = rng.uniform(-1, 1, size=(130, 3))
    off = np.array([0, 70, 130])
    nnx = np.stack([cKDTree(P[off[t]:off[t + 1]]).query(X[t])[1] for t in range(2)])
    nnp = np.concatenate([cKDTree(X[t]).query(P[off[t]:off[t + 1]])[1] for t in range(2)])
    cd = O.chamfer_from_nn(X, off, P, nnx, nnp)
    for t in range(2):
        Pt = P[off[t]:off[t + 1]]
        ref = (np.mean(cKDTree(Pt).query(X[t])[0] ** 2) +
               np.mean(cKDTree(X[t]).query(Pt)[0] ** 2))
        assert abs(cd[t] - ref) < 1e-13
    worse = O.chamfer_from_nn(X, off, P, (nnx + 1) % 70 % 60, (nnp + 1) % 60)
    assert np.all(worse > cd)
    n0 = O.set_threads()
    try:
        O.set_threads(1)
        one = O.chamfer(X, off, P)
        O.set_threads(max(n0, 4))
        many = O.chamfer(X, off, P)
    finally:
        O.set_threads(n0)
    for a, b in zip(one, many):
        np.testing.assert_array_equal(a, b)


# ---------------------------------------------------------------- Sec. 3.5 weights, iso

def test_confidence_weights_golden_and_invariants():
    g = _gold("confidence_weights.json")
    for case in g["cases"]:
        w = O.conf_weights(np.array(g["cd"]), g["t_key"], case["e"], case["e_max"])
        np.testing.assert_allclose(w, case["w"], rtol=1e-14)
    rng = np.random.default_rng(11)
    cd = rng.uniform(0, 1, size=9)
    w = O.conf_weights(cd, 4, 3, 10)
    assert w[4] == 1.0
    assert np.all(np.diff(w[4:]) <= 0) and np.all(np.diff(w[:5]) >= 0)


def test_iso_golden_and_rigid_invariance():
    from scipy.spatial.transform import Rotation
    g = _gold("isometry_edge.json")
    xh = np.array(g["xhat"])
    e = np.array(g["edges"], dtype=np.int32)
    lref = O.edge_lengths(xh, g["t_key"], e)
    assert abs(O.iso(xh, e, lref) - g["L_iso"]) < 1e-15
    seq = I.random_cloud_sequence()
    ed = O.edges(seq.faces)
    assert len(ed) == 120  # icosphere subdiv 1: E = 3F/2
    x = seq.x.astype(np.float64)
    frames = np.stack([x @ Rotation.random(random_state=k).as_matrix().T + k * 0.1
                       for k in range(4)])
    lref = O.edge_lengths(frames, 2, ed)
    assert O.iso(frames, ed, lref) < 1e-14


# ---------------------------------------------------------------- gradient (FD)

def _fd_problem(rot_mode, seed=0):
    seq = I.random_cloud_sequence(T=3, M=[25, 31, 18], seed=seed)
    cfg = small_cfg(rot_mode=rot_mode)
    prob = O.Problem(cfg, seq.x, seq.n, seq.faces, seq.points, seq.offsets, seq.t_key)
    rng = np.random.default_rng(seed + 100)
    grid = rng.normal(scale=0.3, size=O.grid_len(cfg))
    mlp = I.mlp_init(O.k_in(cfg), cfg.H, cfg.D, O.n_out(cfg), seed=seed,
                     zero_last=False).astype(np.float64) * 1.5
    return prob, grid, mlp


@pytest.mark.parametrize("rot_mode", [0, 1, 2])
def test_gradient_matches_central_differences(rot_mode):
    """Hand-written reverse mode == central FD of the same loss (FP64,
    stop-grad inputs held fixed as Eq. 11-13 prescribe)."""
    prob, grid, mlp = _fd_problem(rot_mode)
    full = O.loss_full(prob, grid, mlp, e=3, e_max=10)
    w = full["w"]
    lref = O.edge_lengths(full["xhat"], prob.t_key, prob.edges)
    L0, gg, gm, _ = O.loss_grad(prob, grid, mlp, w, lref)
    assert abs(L0 - full["loss"]) < 1e-15
    np.testing.assert_array_equal(gg, full["g_grid"])
    eps = 1e-6
    num_g = np.zeros_like(grid)
    for k in range(len(grid)):
        if gg[k] == 0.0:  # node not touched by any vertex: check a few only
            if k % 17:
                continue
        gp, gmn = grid.copy(), grid.copy()
        gp[k] += eps
        gmn[k] -= eps
        num_g[k] = (O.loss_grad(prob, gp, mlp, w, lref, want_grad=False)[0] -
                    O.loss_grad(prob, gmn, mlp, w, lref, want_grad=False)[0]) / (2 * eps)
    num_m = np.zeros_like(mlp)
    for k in range(len(mlp)):
        mp, mm = mlp.copy(), mlp.copy()
        mp[k] += eps
        mm[k] -= eps
        num_m[k] = (O.loss_grad(prob, grid, mp, w, lref, want_grad=False)[0] -
                    O.loss_grad(prob, grid, mm, w, lref, want_grad=False)[0]) / (2 * eps)
    mask = (gg != 0) | (np.arange(len(grid)) % 17 == 0)
    assert np.linalg.norm(gg[mask] - num_g[mask]) <= 1e-6 * np.linalg.norm(gg[mask])
    assert np.linalg.norm(gm - num_m) <= 1e-6 * np.linalg.norm(gm)
    assert np.linalg.norm(gg) > 0 and np.linalg.norm(gm) > 0


def test_learned_time_embedding_closed_forms():
    """The learned embedding of the time-encoding ablation (Sec. 4),
    gamma(t) = psi_t(t~) = W act(a t~ + b) + c with Ht hidden units: with one
    linear hidden unit (slope 1, a = 1, b = 0) gamma_k = W_k t~ + c_k; with a
    ReLU unit a = -1, b = 1/2 it is W_k max(0, 1/2 - t~) + c_k."""
    T, M = 5, 2
    for slope, a, b, h in ((1.0, 1.0, 0.0, lambda t: t),
                           (0.0, -1.0, 0.5, lambda t: max(0.0, 0.5 - t))):
        cfg = O.make_cfg(L=1, res=(3,), F=1, H=4, D=1, n_freq=M, slope=slope, time_enc=3,
                         time_hidden=1)
        nt = O.time_params(cfg)
        assert nt == 2 + 2 * M + 2 * M
        Wk = np.array([1.0, -2.0, 0.25, 3.0])
        ck = np.array([0.5, 0.0, -1.0, 2.0])
        tail = np.concatenate([[a], [b], Wk, ck])
        mlp = np.concatenate([np.zeros(O.mlp_len(cfg) - nt), tail])
        g = O.time_embedding(cfg, T, mlp)
        for t in range(T):
            np.testing.assert_allclose(g[t], Wk * h(t / (T - 1)) + ck, rtol=0, atol=1e-15)


def test_learned_time_embedding_gradient_matches_central_differences():
    """Reverse mode through psi_t (and through everything else) == central FD
    of the same loss, every parameter of the decoder and of psi_t."""
    seq = I.random_cloud_sequence(T=3, M=[25, 31, 18], seed=4)
    cfg = O.make_cfg(L=2, res=(3, 5), F=2, Fn=2, rn=4, H=8, D=2, slope=0.01, time_enc=3,
                     time_hidden=6)
    prob = O.Problem(cfg, seq.x, seq.n, seq.faces, seq.points, seq.offsets, seq.t_key)
    rng = np.random.default_rng(104)
    grid = rng.normal(scale=0.3, size=O.grid_len(cfg))
    nt = O.time_params(cfg)
    dec = I.mlp_init(O.k_in(cfg), cfg.H, cfg.D, O.n_out(cfg), seed=4, zero_last=False) * 1.5
    mlp = np.concatenate([dec.astype(np.float64), rng.normal(scale=0.8, size=nt)])
    assert len(mlp) == O.mlp_len(cfg)
    full = O.loss_full(prob, grid, mlp, e=3, e_max=10)
    w = full["w"]
    lref = O.edge_lengths(full["xhat"], prob.t_key, prob.edges)
    L0, gg, gm, _ = O.loss_grad(prob, grid, mlp, w, lref)
    eps = 1e-6
    num_m = np.zeros_like(mlp)
    for k in range(len(mlp)):
        mp, mm = mlp.copy(), mlp.copy()
        mp[k] += eps
        mm[k] -= eps
        num_m[k] = (O.loss_grad(prob, grid, mp, w, lref, want_grad=False)[0] -
                    O.loss_grad(prob, grid, mm, w, lref, want_grad=False)[0]) / (2 * eps)
    assert np.linalg.norm(gm - num_m) <= 1e-6 * np.linalg.norm(gm)
    tail = slice(len(mlp) - nt, len(mlp))
    assert np.linalg.norm(gm[tail]) > 0
    assert np.linalg.norm(gm[tail] - num_m[tail]) <= 1e-6 * np.linalg.norm(gm[tail])


def test_backprop_magnitude_bounds_the_gradient():
    """The magnitude companion of the reverse pass sums |each product|: it
    bounds every gradient value from above (triangle inequality), equals it
    where a value is made of one product (the output bias of a single row), and
    scales with |dL/dx-hat|."""
    prob, grid, mlp = _fd_problem(0)
    rng = np.random.default_rng(21)
    gx = rng.normal(size=(prob.T, prob.N, 3))
    gg, gm = O.backprop(prob, grid, mlp, gx)
    mg, mm = O.backprop(prob, grid, mlp, gx, magnitude=True)
    assert np.all(np.abs(gg) <= mg * (1 + 1e-12) + 1e-300)
    assert np.all(np.abs(gm) <= mm * (1 + 1e-12) + 1e-300)
    assert np.sum(mm) > 1.5 * np.sum(np.abs(gm))  # the sums do cancel
    mg2, mm2 = O.backprop(prob, grid, mlp, -3.0 * gx, magnitude=True)
    np.testing.assert_allclose(mg2, 3.0 * mg, rtol=1e-12)
    np.testing.assert_allclose(mm2, 3.0 * mm, rtol=1e-12)
    one = np.zeros_like(gx)
    one[1, 2] = gx[1, 2]
    _, gm1 = O.backprop(prob, grid, mlp, one)
    _, mm1 = O.backprop(prob, grid, mlp, one, magnitude=True)
    NO = O.n_out(prob.cfg)
    np.testing.assert_allclose(mm1[-NO:], np.abs(gm1[-NO:]), rtol=1e-14)


# ---------------------------------------------------------------- Eq. 9

def _lattice_laplacian(r):
    import networkx as nx
    G = nx.grid_graph(dim=[r, r, r])  # nodes (ix, iy, iz) in dim order given
    order = sorted(G.nodes(), key=lambda p: (p[2], p[1], p[0]))
    Lap = nx.laplacian_matrix(G, nodelist=order).toarray().astype(np.float64)
    return Lap


@pytest.mark.parametrize("r,lam", [(2, 0.4), (3, 0.6), (4, 2.0), (5, 0.4), (6, 6.8)])
def test_preconditioner_matches_dense_solve(r, lam):
    """Eq. 9: (I + lambda L)^-2 g by CG == a dense direct solve with the
    lattice Laplacian built by networkx."""
    F = 2
    rng = np.random.default_rng(r)
    g = rng.normal(size=r ** 3 * F)
    out, its = O.precondition(r, F, lam, g)
    Lap = _lattice_laplacian(r)
    A = np.eye(r ** 3) + lam * Lap
    for ch in range(F):
        ref = np.linalg.solve(A @ A, g[ch::F])
        np.testing.assert_allclose(out[ch::F], ref, rtol=0, atol=1e-11 * np.abs(ref).max())


def test_preconditioner_invariants():
    r, F = 7, 3
    rng = np.random.default_rng(12)
    g = rng.normal(size=r ** 3 * F)
    out, _ = O.precondition(r, F, 0.0, g)
    np.testing.assert_allclose(out, g, atol=1e-14)
    c = np.tile([1.5, -2.0, 0.25], r ** 3)
    out, _ = O.precondition(r, F, 3.0, c)
    np.testing.assert_allclose(out, c, atol=1e-11)
    u, v = rng.normal(size=r ** 3), rng.normal(size=r ** 3)
    Pu, _ = O.precondition(r, 1, 1.7, u)
    Pv, _ = O.precondition(r, 1, 1.7, v)
    assert abs(u @ Pv - v @ Pu) < 1e-10 * abs(u @ Pv)


# ---------------------------------------------------------------- Adam

def test_adam_matches_torch_and_first_step():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(13)
    p0 = rng.normal(size=40)
    grads = [rng.normal(size=40) for _ in range(6)]
    p, m, v = p0.copy(), np.zeros(40), np.zeros(40)
    tp = torch.tensor(p0.copy(), requires_grad=True)
    opt = torch.optim.Adam([tp], lr=0.01)
    for s, g in enumerate(grads, start=1):
        p, m, v = O.adam(p, g, m, v, lr=0.01, step=s)
        tp.grad = torch.tensor(g)
        opt.step()
        if s == 1:
            np.testing.assert_allclose(p, p0 - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-14)
    np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-12, atol=1e-14)


# ---------------------------------------------------------------- whole iteration

def test_iteration_decreases_chamfer():
    seq = I.sphere_blob(subdiv=2, T=4, M=300, seed=3)
    cfg = O.make_cfg(L=2, res=(5, 9), F=2, H=16, D=2, slope=0.0)
    prob = O.Problem(cfg, seq.x, seq.n, seq.faces, seq.points, seq.offsets, seq.t_key)
    st = O.State(prob, np.zeros(O.grid_len(cfg)),
                 I.mlp_init(O.k_in(cfg), 16, 2, O.n_out(cfg), seed=1))
    lr = [0.005 * 2.5 ** l for l in range(cfg.L)] + [0.005]
    lam = [0.4 * 1.5 ** l for l in range(cfg.L)] + [0.4]
    # the weighted loss itself may rise as delta -> 0 lifts w_conf towards 1
    # (Eq. 11); the unweighted Chamfer distance is what must fall
    cds = [O.iteration(prob, st, 20, lr, 1e-3, lam)["cd"].mean() for _ in range(8)]
    assert cds[-1] < cds[0]
    assert st.e == 8


def _dct_precondition(r, F, lam, g):
    """(I + lam L)^-2 g per channel through scipy's orthonormal 3-D DCT-II: the
    Neumann lattice Laplacian is diagonal there with eigenvalues
    sum_axes (2 - 2 cos(pi k / r)). Independent of the oracle's CG solve."""
    from scipy.fft import dctn, idctn
    k = np.arange(r)
    mu1 = 2.0 - 2.0 * np.cos(np.pi * k / r)
    mu = mu1[:, None, None] + mu1[None, :, None] + mu1[None, None, :]
    out = np.empty_like(g)
    for ch in range(F):
        x = g[ch::F].reshape(r, r, r)
        out[ch::F] = idctn(dctn(x, norm="ortho") / (1.0 + lam * mu) ** 2, norm="ortho").ravel()
    return out


def test_iteration_first_adam_step_hand_worked():
    """One whole iteration (Sec. 3.5: Eq. 9, then Adam with the per-level rates
    of the implementation details) from zero Adam moments at e = 5.

    Hand-worked: with m = v = 0 the update of step s is
      dp = -lr (1 - b1)/(1 - b1^s) g / (sqrt((1 - b2)/(1 - b2^s)) |g| + eps),
    i.e. |dp| = lr * 0.5221178227 for s = e + 1 = 6 (it would be 0.5454892500
    for s = e = 5), against the sign of g. So every grid value of level l
    (0-based, coarsest first) must move by exactly 0.005 * 2.5^l * 0.52211782
    against the *preconditioned* gradient, the normal grid by 0.005 * 0.52211782,
    the MLP by 1e-3 * 0.52211782 against its raw gradient. The preconditioned
    gradient is recomputed here by a DCT solve with lambda_l = 0.4 * 1.5^l: it
    moves nodes whose raw gradient is 0 and flips the sign of others, so a raw
    gradient passed to Adam, a level index off by one or the step count e
    fails a check."""
    seq = I.sphere_blob(subdiv=2, T=3, M=300, seed=5)
    cfg = O.make_cfg(L=2, res=(5, 9), F=2, H=16, D=2, slope=0.01)
    prob = O.Problem(cfg, seq.x, seq.n, seq.faces, seq.points, seq.offsets, seq.t_key)
    rng = np.random.default_rng(7)
    grid0 = rng.normal(scale=0.05, size=O.grid_len(cfg))
    mlp0 = I.mlp_init(O.k_in(cfg), 16, 2, O.n_out(cfg), seed=3, zero_last=False)
    st = O.State(prob, grid0, mlp0)
    st.e = 5
    lr = [0.005 * 2.5 ** l for l in range(cfg.L)] + [0.005]
    lam = [0.4 * 1.5 ** l for l in range(cfg.L)] + [0.4]
    # eps far below every |g| checked, so that |dp| is lr * 0.52211782 to 1e-6
    out = O.iteration(prob, st, 20, lr, 1e-3, lam, eps=1e-14)
    assert st.e == 6
    ratio = 0.5221178227443565
    moved_zero, flipped = 0, 0
    for l in range(cfg.L + 1):
        r = cfg.res[l] if l < cfg.L else cfg.rn
        F = cfg.F if l < cfg.L else cfg.Fn
        o, n = O.level_offset(cfg, l), r ** 3 * F
        g = out["g_grid"][o:o + n]
        gt = out["g_grid_pc"][o:o + n]
        want_gt = _dct_precondition(r, F, lam[l], g)
        np.testing.assert_allclose(gt, want_gt, rtol=0, atol=1e-10 * np.abs(want_gt).max())
        d = st.grid[o:o + n] - grid0[o:o + n]
        big = np.abs(gt) > max(1e-7, 1e-4 * np.abs(gt).max())
        assert big.sum() > n // 2
        np.testing.assert_allclose(np.abs(d[big]), lr[l] * ratio, rtol=1e-6)
        assert np.all(np.sign(d[big]) == -np.sign(gt[big]))
        moved_zero += int(np.sum(big & (g == 0)))
        flipped += int(np.sum(big & (np.sign(g) * np.sign(gt) < 0)))
    assert moved_zero > 0 and flipped > 0
    gm = out["g_mlp"]
    dm = st.mlp - mlp0
    bigm = np.abs(gm) > 1e-7
    assert bigm.sum() > len(gm) // 2
    np.testing.assert_allclose(np.abs(dm[bigm]), 1e-3 * ratio, rtol=1e-5)
    assert np.all(np.sign(dm[bigm]) == -np.sign(gm[bigm]))
    # the loss is that of the parameters before the update, at e = 5
    ref = O.loss_full(prob, grid0, mlp0, 5, 20, want_grad=False)
    assert abs(out["loss"] - ref["loss"]) <= 1e-13 * abs(ref["loss"])


# ---------------------------------------------------------------- Sec. 4 metrics

def test_evaluation_metrics_invariants():
    """Identity: (cd, P, R, F, NC, corr) = (0, 1, 1, 1, 1, 0). A uniform shift s
    smaller than half the vertex spacing keeps every nearest pair on the same
    vertex: cd = 2 |s|^2, corr = |s|, NC = 1, and F = 1 below the threshold,
    0 above it. Scaling both meshes by k scales cd by k^2 and corr by k and
    leaves the rest (the threshold is relative to the bounding box)."""
    v, f = I.icosphere(3)
    rng = np.random.default_rng(0)
    gt = np.stack([v, v * 1.2 + 0.1])
    m = O.evaluate(gt, gt, f)
    np.testing.assert_array_equal(m, [[0, 1, 1, 1, 1, 0]] * 2)
    tau = 0.005 * np.linalg.norm(gt[0].max(0) - gt[0].min(0))
    for mag in (0.5 * tau, 3.0 * tau):
        s = _unit3(rng) * mag
        m = O.evaluate(gt[:1] + s, gt[:1], f)[0]
        np.testing.assert_allclose(m[0], 2 * mag ** 2, rtol=1e-9)
        np.testing.assert_allclose(m[5], mag, rtol=1e-9)
        np.testing.assert_allclose(m[4], 1.0, rtol=1e-12)
        assert m[3] == (1.0 if mag < tau else 0.0)
    xh = gt + rng.normal(scale=0.01, size=gt.shape)
    a, b = O.evaluate(xh, gt, f), O.evaluate(3.0 * xh, 3.0 * gt, f)
    np.testing.assert_allclose(b[:, 0], 9.0 * a[:, 0], rtol=1e-9)
    np.testing.assert_allclose(b[:, 5], 3.0 * a[:, 5], rtol=1e-9)
    np.testing.assert_allclose(b[:, 1:5], a[:, 1:5], rtol=1e-9)


def _unit3(rng):
    u = rng.normal(size=3)
    return u / np.linalg.norm(u)


def test_evaluation_metrics_match_kdtree_and_numpy_normals():
    """Against an independent computation: scipy cKDTree nearest neighbours
    and normals accumulated with numpy (np.add.at over face cross products)."""
    from scipy.spatial import cKDTree
    seq = I.sphere_blob(subdiv=3, T=3, M=500, seed=3)
    rng = np.random.default_rng(1)
    gt = seq.gt_frames
    xh = gt + rng.normal(scale=0.02, size=gt.shape)
    f = seq.faces
    got = O.evaluate(xh, gt, f, tau_rel=0.01)

    def normals(v):
        n = np.cross(v[f[:, 1]] - v[f[:, 0]], v[f[:, 2]] - v[f[:, 0]])
        acc = np.zeros_like(v)
        for k in range(3):
            np.add.at(acc, f[:, k], n)
        return acc / np.linalg.norm(acc, axis=1, keepdims=True)

    for t in range(gt.shape[0]):
        X, G = xh[t], gt[t]
        dx, ix = cKDTree(G).query(X)
        dg, ig = cKDTree(X).query(G)
        tau = 0.01 * np.linalg.norm(G.max(0) - G.min(0))
        P, R = np.mean(dx < tau), np.mean(dg < tau)
        nx, ng = normals(X), normals(G)
        nc = 0.5 * (np.mean(np.abs(np.sum(nx * ng[ix], 1))) + np.mean(np.abs(np.sum(ng * nx[ig], 1))))
        want = [np.mean(dx ** 2) + np.mean(dg ** 2), P, R, 2 * P * R / (P + R), nc,
                np.mean(np.linalg.norm(X - G, axis=1))]
        np.testing.assert_allclose(got[t], want, rtol=1e-9, atol=1e-15)


# ---------------------------------------------------------------- ablation variants

def test_time_encoding_variants():
    """Polynomial basis t~^j (j = 1..2M) and Gaussian Fourier mapping
    sin / cos(2 pi B_j t~), against hand values."""
    cfg = O.make_cfg(L=2, res=(4, 5), F=2, n_freq=2, time_enc=1)
    g = O.time_embedding(cfg, 5)  # t~ = 0, 1/4, 1/2, 3/4, 1
    np.testing.assert_allclose(g[1], [0.25, 0.0625, 0.015625, 0.00390625], rtol=1e-15)
    np.testing.assert_array_equal(g[0], 0.0)
    np.testing.assert_array_equal(g[4], 1.0)
    cfg = O.make_cfg(L=2, res=(4, 5), F=2, n_freq=2, time_enc=2, time_B=(1.0, 0.5))
    g = O.time_embedding(cfg, 5)
    np.testing.assert_allclose(g[0], [0, 1, 0, 1], atol=1e-15)
    # t~ = 1/4: B = 1 -> (sin pi/2, cos pi/2); B = 1/2 -> (sin pi/4, cos pi/4)
    np.testing.assert_allclose(g[1], [1, 0, 0.5 ** 0.5, 0.5 ** 0.5], atol=1e-15)
    # t~ = 1: B = 1 -> (0, 1); B = 1/2 -> (0, -1)
    np.testing.assert_allclose(g[4], [0, 1, 0, -1], atol=1e-15)


def test_stability_schedule_variants():
    """The confidence weights of the stability ablation on a hand-worked
    example: cd = (2, 1, 1.5, 3), keyframe 1, so omega = (1/2, 1, 2/3, 1/3)."""
    cd = np.array([2.0, 1.0, 1.5, 3.0])
    cum1 = np.array([0.5, 1.0, 2 / 3, 2 / 9])        # cumulative products, delta = 1
    single = np.array([0.5, 1.0, 2 / 3, 1 / 3])      # omega(t) alone
    w = lambda e, d, o: O.conf_weights(cd, 1, e, 4, d, o)
    # e~ = 0: every schedule has delta = 1
    for d in (0, 1, 2, 3, 4):
        np.testing.assert_allclose(w(0, d, 0), cum1, rtol=1e-14)
    # e~ = 1/4: delta = 1/2 (sqrt), 1 (constant), 3/4 (linear), exp(-5/4)
    for d, delta in ((0, 0.5), (1, 1.0), (2, 0.75), (3, np.exp(-1.25))):
        np.testing.assert_allclose(w(1, d, 0), cum1 ** delta, rtol=1e-14)
        np.testing.assert_allclose(w(1, d, 3), single ** delta, rtol=1e-14)
        np.testing.assert_allclose(w(1, d, 1), np.ones(4), rtol=0)
        np.testing.assert_allclose(w(1, d, 2), np.full(4, 0.5 ** delta), rtol=1e-14)
    np.testing.assert_allclose(w(1, 4, 0), 0.75 * cum1 + 0.25, rtol=1e-14)
    np.testing.assert_allclose(w(1, 4, 3), 0.75 * single + 0.25, rtol=1e-14)
    # e~ = 1: the method's delta is 0 (all weights 1), and so is the linear one
    for d in (0, 2, 4):
        np.testing.assert_allclose(w(4, d, 0), np.ones(4), rtol=1e-14)


def _frames(clouds):
    off = np.cumsum([0] + [len(c) for c in clouds])
    return np.concatenate(clouds), off


def test_keyframe_extent_closed_forms():
    """The RMS radius of an octahedron's six vertices about any centre is its
    circumradius; the radius scales with the cloud and ignores translation."""
    rng = np.random.default_rng(3)
    octa = np.concatenate([np.eye(3), -np.eye(3)])
    clouds = [0.7 * octa + np.array([0.1, -0.2, 0.3]), 0.25 * octa]
    base = rng.normal(size=(97, 3))
    clouds += [base, 2.5 * base + np.array([0.4, 0.0, -0.1])]
    _, e = O.select_keyframe(*_frames(clouds), bias=0.0)
    np.testing.assert_allclose(e[:2], [0.7, 0.25], rtol=1e-15)
    np.testing.assert_allclose(e[3], 2.5 * e[2], rtol=1e-13)


def test_keyframe_choice_and_midpoint_bias():
    """Without bias the widest frame wins (the first one on exact ties); equal
    frames go to the middle one; a wider edge frame beats the middle frame
    exactly when its weighted extent is larger: T = 3, extents (1.5, 1, 1),
    weights (1 - b/2, 1, 1 - b/2) give frame 0 for b < 2/3 and frame 1 above."""
    octa = np.concatenate([np.eye(3), -np.eye(3)])
    pts, off = _frames([s * octa for s in (0.5, 0.9, 0.3, 0.9)])
    assert O.select_keyframe(pts, off, 0.0)[0] == 1
    for T in (1, 3, 5, 9):
        pts, off = _frames([octa] * T)
        assert O.select_keyframe(pts, off, 1.0)[0] == (T - 1) // 2
    pts, off = _frames([1.5 * octa, octa, octa])
    for b, want in ((0.0, 0), (0.5, 0), (0.6, 0), (0.7, 1), (1.0, 1)):
        assert O.select_keyframe(pts, off, b)[0] == want, b
