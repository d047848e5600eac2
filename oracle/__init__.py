"""FP64 CPU oracle for the Neu-PiG optimisation iteration (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's
``cpu_baseline`` / ``--impl reference`` legs may import this package. The
product path (``libnpg.so`` and ``paper_2602_22212_gb300``) never does.

The C source ``npg_oracle.c`` restates the paper's definitions (Sec. 3.2-3.5,
Eq. 1-13 and the Adam / per-level learning-rate details) in plain FP64 loops;
this module compiles it with gcc and wraps it with ctypes, returning numpy
arrays. Every wrapper names the passage it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "npg_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAX_LEVELS = 16


class OrCfg(C.Structure):
    """Mirror of ``or_cfg`` in npg_oracle.c."""

    _fields_ = [
        ("L", C.c_int),
        ("res", C.c_int * MAX_LEVELS),
        ("F", C.c_int),
        ("Fn", C.c_int),
        ("rn", C.c_int),
        ("H", C.c_int),
        ("D", C.c_int),
        ("rot_mode", C.c_int),
        ("n_freq", C.c_int),
        ("slope", C.c_double),
        ("alpha", C.c_double),
        ("w_iso", C.c_double),
        ("time_enc", C.c_int),
        ("time_B", C.c_double * 8),
        ("conf_delta", C.c_int),
        ("conf_omega", C.c_int),
        ("Ht", C.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (no FMA contraction: the oracle's
    FP32 nearest-neighbour decision uses explicit ``fmaf`` only)."""
    if not force and os.path.exists(_LIB_PATH) and \
            os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", _SRC, "-o", tmp, "-lm"]
    # OpenMP over independent queries / rows / nodes when the compiler has it
    # (results do not depend on the thread count); plain serial C otherwise
    if subprocess.run(cmd[:-1] + ["-fopenmp", "-lm"], capture_output=True).returncode != 0:
        subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            P = C.POINTER
            d, i, l = C.c_double, C.c_int, C.c_long
            pd, pi32, pi64 = P(C.c_double), P(C.c_int32), P(C.c_int64)
            pl = P(C.c_long)
            cfg = P(OrCfg)
            sig = {
                "or_n_out": (i, [cfg]),
                "or_k_in": (i, [cfg]),
                "or_level_offset": (l, [cfg, i]),
                "or_grid_len": (l, [cfg]),
                "or_mlp_len": (l, [cfg]),
                "or_trilinear": (None, [i, pd, pl, pd]),
                "or_encode": (None, [cfg, i, pd, pd, pd, pd]),
                "or_time_embedding": (None, [cfg, i, pd]),
                "or_time_embedding_params": (None, [cfg, pd, i, pd]),
                "or_time_params": (l, [cfg]),
                "or_mlp_forward": (None, [cfg, pd, i, pd, pd]),
                "or_rotation_translation": (None, [cfg, pd, pd, pd]),
                "or_decode": (None, [cfg, i, i, pd, pd, pd, pd, pd]),
                "or_nn": (None, [i, pd, i, pd, i, pi32, pd]),
                "or_chamfer": (None, [i, i, pd, pi64, pd, i, pi32, pd, pi32, pd, pd]),
                "or_chamfer_from_nn": (None, [i, i, pd, pi64, pd, pi32, pi32, pd]),
                "or_set_threads": (i, [i]),
                "or_conf_weights": (None, [i, pd, i, d, d, pd]),
                "or_edges": (l, [i, pi32, pi32]),
                "or_edge_lengths": (None, [i, pd, i, l, pi32, pd]),
                "or_iso": (d, [i, i, pd, l, pi32, pd]),
                "or_loss_grad": (d, [cfg, i, pd, pd, i, pi64, pd, l, pi32, pd, pd, pd, pd, i,
                                     pd, pd, pd, pd, pd, pi32, pi32, pd]),
                "or_loss_full": (d, [cfg, i, pd, pd, i, pi64, pd, l, pi32, i, d, d, pd, pd, i,
                                     pd, pd, pd, pd, pd, pd, pi32, pi32, pd]),
                "or_backprop": (None, [cfg, i, pd, pd, i, pd, pd, pd, pd, pd]),
                "or_backprop_magnitude": (None, [cfg, i, pd, pd, i, pd, pd, pd, pd, pd]),
                "or_precondition": (i, [i, i, d, pd, pd, d, i]),
                "or_adam": (None, [l, pd, pd, pd, pd, d, d, d, d, i]),
                "or_iteration": (d, [cfg, i, pd, pd, i, pi64, pd, l, pi32, i, i, i, pd, pd, pd,
                                     pd, pd, pd, pd, d, pd, d, d, d, i, d, pd, pd, pd, pd]),
                "or_evaluate": (None, [i, i, pd, pd, i, pi32, d, pd]),
                "or_conf_weights_mode": (None, [i, pd, i, d, d, i, i, pd]),
                "or_select_keyframe": (i, [i, pi64, pd, d, pd]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


# ----------------------------------------------------------------- helpers

def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(C.POINTER(C.c_int32))


def _i64(a):
    a = np.ascontiguousarray(a, dtype=np.int64)
    return a, a.ctypes.data_as(C.POINTER(C.c_int64))


def _out_d(n):
    a = np.zeros(max(int(n), 1), dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def _out_i32(n):
    a = np.zeros(max(int(n), 1), dtype=np.int32)
    return a, a.ctypes.data_as(C.POINTER(C.c_int32))


def make_cfg(L, res, F, Fn=2, rn=4, H=64, D=3, rot_mode=0, n_freq=4, slope=0.01,
             alpha=0.1, w_iso=100.0, time_enc=0, time_B=None, conf_delta=0,
             conf_omega=0, time_hidden=0) -> OrCfg:
    c = OrCfg()
    c.L = int(L)
    for k, r in enumerate(res):
        c.res[k] = int(r)
    c.F, c.Fn, c.rn, c.H, c.D = int(F), int(Fn), int(rn), int(H), int(D)
    c.rot_mode, c.n_freq = int(rot_mode), int(n_freq)
    c.slope, c.alpha, c.w_iso = float(slope), float(alpha), float(w_iso)
    c.time_enc, c.conf_delta, c.conf_omega = int(time_enc), int(conf_delta), int(conf_omega)
    c.Ht = int(time_hidden)
    for j, b in enumerate(time_B if time_B is not None else []):
        c.time_B[j] = float(b)
    return c


def grid_len(cfg) -> int:
    return int(lib().or_grid_len(C.byref(cfg)))


def mlp_len(cfg) -> int:
    return int(lib().or_mlp_len(C.byref(cfg)))


def level_offset(cfg, l) -> int:
    return int(lib().or_level_offset(C.byref(cfg), int(l)))


def n_out(cfg) -> int:
    return int(lib().or_n_out(C.byref(cfg)))


def k_in(cfg) -> int:
    return int(lib().or_k_in(C.byref(cfg)))


# ----------------------------------------------------------------- wrappers

def trilinear(r, p):
    """Sec. 3.2: corner indices and trilinear weights of one query point."""
    p, pp = _d(p)
    idx = np.zeros(8, dtype=np.int64)
    w, pw = _out_d(8)
    lib().or_trilinear(int(r), pp, idx.ctypes.data_as(C.POINTER(C.c_long)), pw)
    return idx, w


def encode(cfg, x, n, grid):
    """Sec. 3.2, Eq. 1: (z_n, z_p) per vertex, N x (Fn + F)."""
    N = len(x)
    x, px = _d(x)
    n, pn = _d(n)
    g, pg = _d(grid)
    z, pz = _out_d(N * (cfg.Fn + cfg.F))
    lib().or_encode(C.byref(cfg), N, px, pn, pg, pz)
    return z.reshape(N, cfg.Fn + cfg.F)


def time_embedding(cfg, T, mlp=None):
    """Sec. 3.3, Eq. 3: T x 2M, interleaved (sin, cos) per frequency; the
    ablation's variants by cfg.time_enc (the learned one, 3, needs the
    parameter vector mlp, whose tail holds psi_t's weights)."""
    g, pg = _out_d(T * 2 * cfg.n_freq)
    if mlp is None:
        lib().or_time_embedding(C.byref(cfg), int(T), pg)
    else:
        m, pm = _d(mlp)
        lib().or_time_embedding_params(C.byref(cfg), pm, int(T), pg)
    return g.reshape(T, 2 * cfg.n_freq)


def time_params(cfg) -> int:
    """Number of psi_t parameters at the tail of the MLP vector (0 unless learned)."""
    return int(lib().or_time_params(C.byref(cfg)))


def mlp_forward(cfg, mlp, y):
    """Sec. 3.3, Eq. 4: psi(y) for each row of y."""
    y = np.atleast_2d(y)
    rows = len(y)
    y, py = _d(y)
    m, pm = _d(mlp)
    o, po = _out_d(rows * n_out(cfg))
    lib().or_mlp_forward(C.byref(cfg), pm, rows, py, po)
    return o.reshape(rows, n_out(cfg))


def rotation_translation(cfg, o):
    """Sec. 3.4, Eq. 5-6 (or the exponential map): R (3x3) and d-hat (3)."""
    o, po = _d(o)
    R, pR = _out_d(9)
    d, pdd = _out_d(3)
    lib().or_rotation_translation(C.byref(cfg), po, pR, pdd)
    return R.reshape(3, 3), d


def decode(cfg, x, z, gamma, mlp):
    """Sec. 3.3-3.4, Eq. 2-7: x-hat (T x N x 3)."""
    N, T = len(x), len(gamma)
    x, px = _d(x)
    z, pz = _d(z)
    g, pg = _d(gamma)
    m, pm = _d(mlp)
    xh, pxh = _out_d(T * N * 3)
    lib().or_decode(C.byref(cfg), N, T, px, pz, pg, pm, pxh)
    return xh.reshape(T, N, 3)


def nn(q, cand, decide_f32=False):
    """Brute-force nearest neighbour (lowest index on ties): (idx, squared dist)."""
    nq, nc = len(q), len(cand)
    q, pq = _d(q)
    c, pc = _d(cand)
    idx, pidx = _out_i32(nq)
    dist, pdist = _out_d(nq)
    lib().or_nn(nq, pq, nc, pc, int(bool(decide_f32)), pidx, pdist)
    return idx[:nq], dist[:nq]


def chamfer(xhat, off, pts, decide_f32=False):
    """Sec. 3.5 Chamfer term per frame: nn_x, d_x, nn_p, d_p, cd."""
    T, N = xhat.shape[0], xhat.shape[1]
    MT = int(off[-1])
    xh, pxh = _d(xhat)
    o, po = _i64(off)
    p, pp = _d(pts)
    nnx, pnnx = _out_i32(T * N)
    dx, pdx = _out_d(T * N)
    nnp, pnnp = _out_i32(MT)
    dp, pdp = _out_d(MT)
    cd, pcd = _out_d(T)
    lib().or_chamfer(T, N, pxh, po, pp, int(bool(decide_f32)), pnnx, pdx, pnnp, pdp, pcd)
    return (nnx.reshape(T, N), dx.reshape(T, N), nnp[:MT], dp[:MT], cd)


def chamfer_from_nn(xhat, off, pts, nn_x, nn_p):
    """Sec. 3.5, Eq. 10's cd_t for given nearest-neighbour choices (nn_x: T x N
    frame-local point indices, nn_p: one vertex index per point)."""
    T, N = xhat.shape[0], xhat.shape[1]
    xh, pxh = _d(xhat)
    o, po = _i64(off)
    p, pp = _d(pts)
    a, pa = _i32(np.asarray(nn_x).reshape(-1))
    b, pb = _i32(nn_p)
    cd, pcd = _out_d(T)
    lib().or_chamfer_from_nn(T, N, pxh, po, pp, pa, pb, pcd)
    return cd[:T]


def set_threads(n=0):
    """Host threads of the oracle's parallel loops (n <= 0 keeps the current
    setting); returns the count in effect (1 when built without OpenMP)."""
    return int(lib().or_set_threads(int(n)))


def conf_weights(cd, t_key, e, e_max, delta_mode=0, omega_mode=0):
    """Sec. 3.5, Eq. 11-12 (modes: the stability ablation's variants)."""
    T = len(cd)
    cd, pcd = _d(cd)
    w, pw = _out_d(T)
    lib().or_conf_weights_mode(T, pcd, int(t_key), float(e), float(e_max), int(delta_mode),
                               int(omega_mode), pw)
    return w


def edges(faces):
    """Unique undirected mesh edges (i < j), sorted."""
    faces, pf = _i32(faces)
    Ft = len(faces)
    out, po = _out_i32(6 * Ft)
    E = lib().or_edges(Ft, pf, po)
    return out[: 2 * E].reshape(E, 2).copy()


def edge_lengths(xhat, t, e):
    T, N = xhat.shape[0], xhat.shape[1]
    xh, pxh = _d(xhat)
    e, pe = _i32(e)
    out, po = _out_d(len(e))
    lib().or_edge_lengths(N, pxh, int(t), len(e), pe, po)
    return out[: len(e)]


def iso(xhat, e, lref):
    """Sec. 3.5, Eq. 13 with given reference lengths."""
    T, N = xhat.shape[0], xhat.shape[1]
    xh, pxh = _d(xhat)
    e, pe = _i32(e)
    lr, plr = _d(lref)
    return float(lib().or_iso(T, N, pxh, len(e), pe, plr))


class Problem:
    """The fixed inputs of one sequence (Sec. 3, problem statement)."""

    def __init__(self, cfg, x, n, faces, points, offsets, t_key):
        self.cfg = cfg
        self.x = np.ascontiguousarray(x, dtype=np.float64)
        self.n = np.ascontiguousarray(n, dtype=np.float64)
        self.N = len(self.x)
        self.off = np.ascontiguousarray(offsets, dtype=np.int64)
        self.T = len(self.off) - 1
        self.pts = np.ascontiguousarray(points, dtype=np.float64)
        self.edges = edges(faces)
        self.E = len(self.edges)
        self.t_key = int(t_key)


def loss_grad(prob: Problem, grid, mlp, w_fixed, lref, decide_f32=False, want_grad=True):
    """Eq. 8, 10, 13 with the stop-grad inputs held fixed, and its gradient."""
    c, N, T = prob.cfg, prob.N, prob.T
    _, px = _d(prob.x)
    _, pn = _d(prob.n)
    _, po = _i64(prob.off)
    _, pp = _d(prob.pts)
    _, pe = _i32(prob.edges)
    g, pg = _d(grid)
    m, pm = _d(mlp)
    w, pw = _d(w_fixed)
    lr, plr = _d(lref)
    gg, pgg = _out_d(grid_len(c))
    gm, pgm = _out_d(mlp_len(c))
    parts, pparts = _out_d(2)
    null = C.POINTER(C.c_double)()
    nulli = C.POINTER(C.c_int32)()
    L = lib().or_loss_grad(C.byref(c), N, px, pn, T, po, pp, prob.E, pe, pg, pm, pw, plr,
                           int(bool(decide_f32)), pgg if want_grad else null,
                           pgm if want_grad else null, null, null, pparts, nulli, nulli, null)
    return float(L), gg, gm, parts


def loss_full(prob: Problem, grid, mlp, e, e_max, decide_f32=False, want_grad=True):
    """The loss of iteration e with its stop-grad inputs computed from this
    forward pass (Eq. 11-13), plus gradients and intermediates (dict)."""
    c, N, T = prob.cfg, prob.N, prob.T
    MT = int(prob.off[-1])
    _, px = _d(prob.x)
    _, pn = _d(prob.n)
    _, po = _i64(prob.off)
    _, pp = _d(prob.pts)
    _, pe = _i32(prob.edges)
    g, pg = _d(grid)
    m, pm = _d(mlp)
    gg, pgg = _out_d(grid_len(c))
    gm, pgm = _out_d(mlp_len(c))
    xh, pxh = _out_d(T * N * 3)
    cd, pcd = _out_d(T)
    w, pw = _out_d(T)
    parts, pparts = _out_d(2)
    nnx, pnnx = _out_i32(T * N)
    nnp, pnnp = _out_i32(MT)
    gx, pgx = _out_d(T * N * 3)
    null = C.POINTER(C.c_double)()
    L = lib().or_loss_full(C.byref(c), N, px, pn, T, po, pp, prob.E, pe, prob.t_key, float(e),
                           float(e_max), pg, pm, int(bool(decide_f32)),
                           pgg if want_grad else null, pgm if want_grad else null, pxh, pcd,
                           pw, pparts, pnnx, pnnp, pgx if want_grad else null)
    return dict(loss=float(L), g_grid=gg, g_mlp=gm, xhat=xh.reshape(T, N, 3), cd=cd, w=w,
                L_def=parts[0], L_iso=parts[1], nn_x=nnx[: T * N].reshape(T, N),
                nn_p=nnp[:MT], g_xhat=gx.reshape(T, N, 3))


def backprop(prob: Problem, grid, mlp, g_xhat, magnitude=False):
    """Parameter gradient of a given dL/dx-hat (T x N x 3): the reverse pass
    through Eq. 7-5, Eq. 4, Eq. 2 and Eq. 1. magnitude=True returns instead
    the sums of the absolute values of the products that make up each
    gradient value (dL/do, weights, activations and inputs taken by absolute
    value): the scale against which rounding errors of the operands are
    bounded."""
    c, N, T = prob.cfg, prob.N, prob.T
    _, px = _d(prob.x)
    _, pn = _d(prob.n)
    g, pg = _d(grid)
    m, pm = _d(mlp)
    gx, pgx = _d(np.asarray(g_xhat).reshape(-1))
    gg, pgg = _out_d(grid_len(c))
    gm, pgm = _out_d(mlp_len(c))
    fn = lib().or_backprop_magnitude if magnitude else lib().or_backprop
    fn(C.byref(c), N, px, pn, T, pg, pm, pgx, pgg, pgm)
    return gg, gm


def precondition(r, F, lam, g, tol=1e-13, max_iter=100000):
    """Sec. 3.5, Eq. 9: (I + lambda L)^-2 g per channel of an r^3 x F block."""
    g, pg = _d(g)
    out, po = _out_d(len(g))
    its = lib().or_precondition(int(r), int(F), float(lam), pg, po, float(tol), int(max_iter))
    return out[: len(g)], int(its)


def adam(p, g, m, v, lr, step, b1=0.9, b2=0.999, eps=1e-8):
    """Adam (bias-corrected), in place on copies; returns (p, m, v)."""
    p = np.array(p, dtype=np.float64)
    m = np.array(m, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    g, pgg = _d(g)
    lib().or_adam(len(p), p.ctypes.data_as(C.POINTER(C.c_double)), pgg,
                  m.ctypes.data_as(C.POINTER(C.c_double)),
                  v.ctypes.data_as(C.POINTER(C.c_double)), float(lr), float(b1), float(b2),
                  float(eps), int(step))
    return p, m, v


class State:
    """Parameters and Adam moments of one run of the oracle."""

    def __init__(self, prob: Problem, grid, mlp):
        self.grid = np.array(grid, dtype=np.float64)
        self.mlp = np.array(mlp, dtype=np.float64)
        self.m_grid = np.zeros_like(self.grid)
        self.v_grid = np.zeros_like(self.grid)
        self.m_mlp = np.zeros_like(self.mlp)
        self.v_mlp = np.zeros_like(self.mlp)
        self.e = 0


def iteration(prob: Problem, st: State, e_max, lr_grid, lr_mlp, lam, b1=0.9, b2=0.999,
              eps=1e-8, decide_f32=False, cg_tol=1e-13):
    """One optimisation iteration (Sec. 3.5): loss, gradient, Eq. 9 on every
    grid level, Adam. Updates ``st`` in place; returns a dict with the loss,
    cd, raw and preconditioned grid gradient and the MLP gradient."""
    c, N, T = prob.cfg, prob.N, prob.T
    _, px = _d(prob.x)
    _, pn = _d(prob.n)
    _, po = _i64(prob.off)
    _, pp = _d(prob.pts)
    _, pe = _i32(prob.edges)
    P = C.POINTER(C.c_double)
    lrg, plrg = _d(lr_grid)
    lm, plm = _d(lam)
    cd, pcd = _out_d(T)
    gg, pgg = _out_d(grid_len(c))
    gp, pgp = _out_d(grid_len(c))
    gm, pgm = _out_d(mlp_len(c))
    L = lib().or_iteration(C.byref(c), N, px, pn, T, po, pp, prob.E, pe, prob.t_key, st.e,
                           int(e_max), st.grid.ctypes.data_as(P), st.mlp.ctypes.data_as(P),
                           st.m_grid.ctypes.data_as(P), st.v_grid.ctypes.data_as(P),
                           st.m_mlp.ctypes.data_as(P), st.v_mlp.ctypes.data_as(P), plrg,
                           float(lr_mlp), plm, float(b1), float(b2), float(eps),
                           int(bool(decide_f32)), float(cg_tol), pcd, pgg, pgp, pgm)
    st.e += 1
    return dict(loss=float(L), cd=cd, g_grid=gg, g_grid_pc=gp, g_mlp=gm)


EVAL_FIELDS = ("cd", "precision", "recall", "fscore", "nc", "corr")


def evaluate(xhat, gt, faces, tau_rel=0.005):
    """Sec. 4 evaluation metrics per frame (reading in npg_oracle.c): T x 6
    {cd, precision, recall, fscore, nc, corr}; xhat and gt are T x N x 3 with
    the reference mesh's connectivity."""
    xhat = np.ascontiguousarray(xhat, dtype=np.float64)
    T, N = xhat.shape[0], xhat.shape[1]
    x, px = _d(xhat)
    g, pg = _d(gt)
    f, pf = _i32(faces)
    out, po = _out_d(6 * T)
    lib().or_evaluate(T, N, px, pg, len(faces), pf, float(tau_rel), po)
    return out[: 6 * T].reshape(T, 6)


def select_keyframe(points, offsets, bias=1.0):
    """Sec. 3.1 keyframe selection (reading in npg_oracle.c): (t_key, extents)
    for concatenated clouds points (off[T] x 3) with frame offsets (T + 1)."""
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    T = len(off) - 1
    p, pp = _d(np.asarray(points, np.float64).reshape(-1, 3))
    o, po = _out_d(T)
    t_key = lib().or_select_keyframe(T, off.ctypes.data_as(C.POINTER(C.c_int64)), pp,
                                     float(bias), po)
    return int(t_key), o[:T].copy()

