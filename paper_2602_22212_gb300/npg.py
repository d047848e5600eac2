"""Thin ctypes binding of libnpg.so (C ABI in include/npg.h).

The functions below carry the C names and only marshal arguments: every step
of the Neu-PiG iteration runs in the library's CUDA kernels. Device pointers
come from torch CUDA tensors, host pointers from numpy arrays or CPU tensors;
streams are torch CUDA streams. If libnpg.so has not been built, importing this
module raises ImportError: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnpg.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`"
        " (or python paper_2602_22212_gb300/build.py)")

_lib = C.CDLL(LIB_PATH)

MAX_LEVELS = 16
MAX_FREQ = 8
TIME_FOURIER, TIME_POLY, TIME_GAUSS, TIME_LEARNED = 0, 1, 2, 3
DELTA_SQRT, DELTA_CONST, DELTA_LINEAR, DELTA_EXP, DELTA_INTERP = 0, 1, 2, 3, 4
OMEGA_CUMULATIVE, OMEGA_CONST, OMEGA_HALF, OMEGA_SINGLE = 0, 1, 2, 3
OK, EINVAL, ENOMEM, ECUDA, ESTATE, ETIMEOUT, ENOTIMPL = 0, -1, -2, -3, -4, -5, -6
ROT_QUAT, ROT_EXPMAP, ROT_CAYLEY = 0, 1, 2
FP32, BF16_MLP = 0, 1
PRECOND_FP32, PRECOND_TC = 0, 1
(BUF_GRID, BUF_MLP, BUF_GRID_GRAD, BUF_GRID_PC, BUF_MLP_GRAD, BUF_XHAT, BUF_NN_X, BUF_NN_P,
 BUF_CD, BUF_WCONF, BUF_ADAM_M_GRID, BUF_ADAM_V_GRID, BUF_ADAM_M_MLP, BUF_ADAM_V_MLP,
 BUF_DIST_X, BUF_DIST_P, BUF_DXHAT, BUF_DISP, BUF_DEVICE_ERROR) = range(19)

_BUF_DTYPE = {BUF_NN_X: np.int32, BUF_NN_P: np.int32, BUF_CD: np.float64, BUF_WCONF: np.float64,
              BUF_DEVICE_ERROR: np.int32}

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class npg_config(C.Structure):
    """Mirror of ``npg_config``."""

    _fields_ = [
        ("L", C.c_int),
        ("res", C.c_int * MAX_LEVELS),
        ("F_p", C.c_int),
        ("F_n", C.c_int),
        ("res_n", C.c_int),
        ("H", C.c_int),
        ("depth", C.c_int),
        ("leaky_slope", C.c_float),
        ("rot_mode", C.c_int),
        ("n_freq", C.c_int),
        ("alpha", C.c_float),
        ("lr_mlp", C.c_float),
        ("lr_grid", C.c_float * (MAX_LEVELS + 1)),
        ("lambda_", C.c_float * (MAX_LEVELS + 1)),
        ("adam_beta1", C.c_float),
        ("adam_beta2", C.c_float),
        ("adam_eps", C.c_float),
        ("w_iso", C.c_float),
        ("e_max", C.c_int),
        ("precision", C.c_int),
        ("nn_cells", C.c_int),
        ("precond_mode", C.c_int),
        ("use_graph", C.c_int),
        ("stream", C.c_void_p),
        ("alloc", ALLOC_FN),
        ("free", FREE_FN),
        ("alloc_user", C.c_void_p),
        ("time_enc", C.c_int),
        ("time_B", C.c_float * MAX_FREQ),
        ("conf_delta", C.c_int),
        ("conf_omega", C.c_int),
        ("time_hidden", C.c_int),
    ]


_vp, _i, _sz = C.c_void_p, C.c_int, C.c_size_t
_cfgp = C.POINTER(npg_config)
_SIG = {
    "npg_config_default": (_i, [_cfgp, _i, _i, _i, _i, _i, _i]),
    "npg_create": (_i, [C.POINTER(_vp), _cfgp, _vp, _vp, _i, _vp, _i, _vp, _vp, _i, _i, _vp, _sz,
                        _i]),
    "npg_forward": (_i, [_vp, _vp]),
    "npg_loss": (_i, [_vp, _vp, _vp]),
    "npg_backward": (_i, [_vp]),
    "npg_step": (_i, [_vp]),
    "npg_backprop": (_i, [_vp, _vp]),
    "npg_iteration": (_i, [_vp, _vp]),
    "npg_set_points": (_i, [_vp, _vp, _vp, _i]),
    "npg_size": (_sz, [_vp, _i]),
    "npg_get": (_i, [_vp, _i, _vp, _sz, _i]),
    "npg_set": (_i, [_vp, _i, _vp, _sz, _i]),
    "npg_get_epoch": (_i, [_vp]),
    "npg_set_epoch": (_i, [_vp, _i]),
    "npg_get_state": (_i, [_vp, _vp, C.POINTER(_sz)]),
    "npg_set_state": (_i, [_vp, _vp, _sz]),
    "npg_destroy": (_i, [_vp]),
    "npg_last_error": (C.c_char_p, [_vp]),
    "npg_nearest": (_i, [_vp, _i, _vp, _i, _vp, _vp, _i, _vp]),
    "npg_select_keyframe": (_i, [_vp, _vp, _i, _i, C.c_double, _vp, C.POINTER(C.c_int), _vp]),
    "npg_precondition": (_i, [_vp, _vp, _i, _i, C.c_float, _vp]),
    "npg_precondition_static": (_i, [_vp, _vp, _i, _i, C.c_float, _vp]),
    "npg_precondition_tc": (_i, [_vp, _vp, _i, _i, C.c_float, _vp]),
    "npg_timing": (_i, [_vp, _i]),
    "npg_timing_read": (_i, [_vp, _i, C.POINTER(C.c_double), C.POINTER(C.c_int)]),
    "npg_launch_count": (C.c_longlong, [_vp]),
    "npg_search_stats": (_i, [_vp, C.POINTER(C.c_longlong)]),
    "npg_evaluate": (_i, [_vp, _vp, _i, C.c_float, _vp]),
    "npg_batch_create": (_i, [C.POINTER(_vp), _i, C.POINTER(_vp), _vp]),
    "npg_batch_iteration": (_i, [_vp, _vp]),
    "npg_batch_destroy": (_i, [_vp]),
    "npg_batch_set_width": (_i, [_vp, _i]),
    "npg_fp32_fma_rate": (_i, [C.POINTER(C.c_double), C.POINTER(C.c_double), _vp]),
    "npg_autotune": (_i, [_vp, _i, C.POINTER(C.c_int)]),
}
for _name, (_res, _args) in _SIG.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_SIG)


class NpgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"npg error {code}: {msg}")
        self.code = code


def _check(rc, ctx=None):
    if rc != OK:
        raise NpgError(rc, _lib.npg_last_error(ctx).decode(errors="replace"))
    return rc


# ----------------------------------------------------------------- marshalling

def _ptr(x):
    """Address of a torch tensor, numpy array, int or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"], "arrays must be C-contiguous"
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous(), "tensors must be contiguous"
        return x.data_ptr()
    raise TypeError(f"cannot take the address of {type(x)}")


def _on_device(x):
    return bool(hasattr(x, "is_cuda") and x.is_cuda)


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ----------------------------------------------------------------- C names

def npg_config_default(L, r_min, r_max, F_p, H, depth) -> npg_config:
    cfg = npg_config()
    _check(_lib.npg_config_default(C.byref(cfg), L, r_min, r_max, F_p, H, depth))
    return cfg


def npg_create(cfg: npg_config, ref_xyz, ref_nrm, faces, points, frame_offsets, t_key, mlp_init):
    """All array inputs on the same side: all torch CUDA tensors, or all host arrays."""
    dev = _on_device(ref_xyz)
    N = int(ref_xyz.shape[0])
    T = int(frame_offsets.shape[0]) - 1
    out = C.c_void_p()
    rc = _lib.npg_create(C.byref(out), C.byref(cfg), _ptr(ref_xyz), _ptr(ref_nrm), N, _ptr(faces),
                         int(faces.shape[0]), _ptr(points), _ptr(frame_offsets), T, int(t_key),
                         _ptr(mlp_init), int(mlp_init.shape[0]), int(dev))
    _check(rc)
    return out.value


def npg_forward(ctx, xhat_out=None):
    _check(_lib.npg_forward(ctx, _ptr(xhat_out)), ctx)


def npg_loss(ctx, loss_out=None, cd_out=None):
    _check(_lib.npg_loss(ctx, _ptr(loss_out), _ptr(cd_out)), ctx)


def npg_backward(ctx):
    _check(_lib.npg_backward(ctx), ctx)


def npg_step(ctx):
    _check(_lib.npg_step(ctx), ctx)


def npg_backprop(ctx, dxhat=None):
    """dxhat: torch CUDA tensor (T x N x 3 FP32) or None."""
    _check(_lib.npg_backprop(ctx, _ptr(dxhat)), ctx)


def npg_iteration(ctx, loss_out=None):
    _check(_lib.npg_iteration(ctx, _ptr(loss_out)), ctx)


EVAL_FIELDS = ("cd", "precision", "recall", "fscore", "nc", "corr")


def npg_evaluate(ctx, gt_xyz, tau_rel=0.005):
    """Sec. 4 metrics of the last forward's x-hat against ground-truth vertices
    (T x N x 3, host array or CUDA tensor): (T + 1) x 6 array, the last row the
    mean over frames; columns EVAL_FIELDS."""
    T = int(gt_xyz.shape[0])
    out = np.zeros((T + 1, 6))
    if not _on_device(gt_xyz):
        gt_xyz = np.ascontiguousarray(gt_xyz, dtype=np.float32)
    _check(_lib.npg_evaluate(ctx, _ptr(gt_xyz), int(_on_device(gt_xyz)), float(tau_rel),
                             out.ctypes.data), ctx)
    return out


def npg_batch_create(ctxs, stream):
    """ctxs: context handles, each created with its own non-default stream."""
    arr = (C.c_void_p * len(ctxs))(*ctxs)
    out = C.c_void_p()
    _check(_lib.npg_batch_create(C.byref(out), len(ctxs), arr, _stream_handle(stream)))
    return out.value


def npg_batch_iteration(batch, loss_out=None):
    """loss_out: host float64 array of S x 3, or None."""
    _check(_lib.npg_batch_iteration(batch, _ptr(loss_out)))


def npg_batch_set_width(batch, width):
    _check(_lib.npg_batch_set_width(batch, int(width)))


def npg_batch_destroy(batch):
    _check(_lib.npg_batch_destroy(batch))


def npg_set_points(ctx, points, frame_offsets):
    _check(_lib.npg_set_points(ctx, _ptr(points), _ptr(frame_offsets), int(_on_device(points))),
           ctx)


def npg_size(ctx, which) -> int:
    return int(_lib.npg_size(ctx, which))


def npg_get(ctx, which, dst):
    nbytes = dst.nbytes if isinstance(dst, np.ndarray) else dst.numel() * dst.element_size()
    _check(_lib.npg_get(ctx, which, _ptr(dst), nbytes, int(_on_device(dst))), ctx)
    return dst


def npg_set(ctx, which, src):
    nbytes = src.nbytes if isinstance(src, np.ndarray) else src.numel() * src.element_size()
    _check(_lib.npg_set(ctx, which, _ptr(src), nbytes, int(_on_device(src))), ctx)


def npg_get_epoch(ctx) -> int:
    return int(_lib.npg_get_epoch(ctx))


def npg_set_epoch(ctx, e):
    _check(_lib.npg_set_epoch(ctx, int(e)), ctx)


def npg_get_state(ctx) -> bytes:
    n = C.c_size_t(0)
    _check(_lib.npg_get_state(ctx, None, C.byref(n)), ctx)
    buf = np.zeros(n.value, dtype=np.uint8)
    _check(_lib.npg_get_state(ctx, buf.ctypes.data, C.byref(n)), ctx)
    return buf.tobytes()


def npg_set_state(ctx, blob: bytes):
    buf = np.frombuffer(blob, dtype=np.uint8).copy()
    _check(_lib.npg_set_state(ctx, buf.ctypes.data, buf.nbytes), ctx)


STAGES = ("encode", "decode", "bucket", "nn_x", "nn_p", "loss", "dxhat", "mlp_bwd", "scatter",
          "precond", "adam")


def npg_timing(ctx, n_iters):
    _check(_lib.npg_timing(ctx, int(n_iters)), ctx)


def npg_timing_read(ctx, stage):
    """(total milliseconds, iterations measured) of one stage."""
    ms, n = C.c_double(0), C.c_int(0)
    _check(_lib.npg_timing_read(ctx, int(stage), C.byref(ms), C.byref(n)), ctx)
    return ms.value, n.value


def npg_search_stats(ctx):
    """(candidates, rows) vertex->point, (candidates, rows) point->vertex."""
    a = (C.c_longlong * 4)()
    _check(_lib.npg_search_stats(ctx, a), ctx)
    return tuple(int(x) for x in a)


def npg_launch_count(ctx) -> int:
    return int(_lib.npg_launch_count(ctx))


def npg_destroy(ctx):
    if ctx:
        _lib.npg_destroy(ctx)


def npg_last_error(ctx=None) -> str:
    return _lib.npg_last_error(ctx).decode(errors="replace")


def npg_nearest(q, cand, idx, dist=None, cells=0, stream=None):
    """Device tensors: q (nq x 3), cand (nc x 3) FP32; idx (nq) int32; dist (nq) FP32."""
    _check(_lib.npg_nearest(_ptr(q), int(q.shape[0]), _ptr(cand), int(cand.shape[0]), _ptr(idx),
                            _ptr(dist), int(cells), _stream_handle(stream)))


def npg_select_keyframe(points, frame_offsets, bias=1.0, stream=None):
    """Keyframe selection (Sec. 3.1): (t_key, per-frame extents). points
    (M_total x 3 FP32) and frame_offsets (T + 1 int64) are both numpy arrays
    (host) or both CUDA tensors (device)."""
    on_device = not isinstance(points, np.ndarray)
    T = int(frame_offsets.shape[0]) - 1
    ext = np.zeros(max(T, 1), np.float64)
    t_key = C.c_int(-1)
    _check(_lib.npg_select_keyframe(_ptr(points), _ptr(frame_offsets), T, int(on_device),
                                    float(bias), ext.ctypes.data, C.byref(t_key),
                                    _stream_handle(stream)))
    return t_key.value, ext[:T]


def npg_precondition(g, out, r, F, lam, stream=None):
    _check(_lib.npg_precondition(_ptr(g), _ptr(out), int(r), int(F), float(lam),
                                 _stream_handle(stream)))


def npg_precondition_tc(g, out, r, F, lam, stream=None):
    """npg_precondition with the DCT passes on the tensor cores (split BF16)."""
    _check(_lib.npg_precondition_tc(_ptr(g), _ptr(out), int(r), int(F), float(lam),
                                    _stream_handle(stream)))


def npg_precondition_static(g, out, r, F, lam, stream=None):
    """Allocation-free npg_precondition (fixed-size scratch; see include/npg.h)."""
    _check(_lib.npg_precondition_static(_ptr(g), _ptr(out), int(r), int(F), float(lam),
                                        _stream_handle(stream)))


def npg_autotune(ctx, reps=3):
    """Tune the context's launch shapes; returns (vertex-side cells, point-side
    cells, decode CTAs per SM, ball rows per thread x -> P, P -> x)."""
    out = (C.c_int * 5)()
    _check(_lib.npg_autotune(ctx, int(reps), out), ctx)
    return tuple(int(v) for v in out)


def npg_fp32_fma_rate(stream=None):
    """(TFLOP/s, ms) of the FP32 FMA probe on the current device."""
    t, ms = C.c_double(0), C.c_double(0)
    _check(_lib.npg_fp32_fma_rate(C.byref(t), C.byref(ms), _stream_handle(stream)))
    return t.value, ms.value


# ----------------------------------------------------------------- convenience

def make_config(L, res, F_p, H, depth, *, F_n=2, res_n=4, slope=0.01, rot_mode=ROT_QUAT,
                precision=FP32, e_max=1000, w_iso=100.0, lr_mlp=1e-3, lr_grid=None,
                lam=None, n_freq=4, alpha=0.1, nn_cells=0, use_graph=False, stream=None,
                precond_mode=PRECOND_FP32, time_enc=TIME_FOURIER, time_B=None,
                conf_delta=DELTA_SQRT, conf_omega=OMEGA_CUMULATIVE, time_hidden=0):
    """npg_config with the paper's defaults (Sec. 3.2-3.5) and explicit resolutions."""
    cfg = npg_config_default(L, 2, 2, F_p, H, depth)
    for k, r in enumerate(res):
        cfg.res[k] = int(r)
    cfg.F_n, cfg.res_n, cfg.leaky_slope, cfg.rot_mode = int(F_n), int(res_n), float(slope), int(
        rot_mode)
    cfg.precision, cfg.e_max, cfg.w_iso, cfg.lr_mlp = int(precision), int(e_max), float(w_iso), \
        float(lr_mlp)
    cfg.n_freq, cfg.alpha, cfg.nn_cells, cfg.use_graph = int(n_freq), float(alpha), int(
        nn_cells), int(bool(use_graph))
    cfg.precond_mode = int(precond_mode)
    cfg.time_enc, cfg.conf_delta, cfg.conf_omega = int(time_enc), int(conf_delta), int(conf_omega)
    cfg.time_hidden = int(time_hidden)
    for j, b in enumerate(time_B if time_B is not None else []):
        cfg.time_B[j] = float(b)
    if lr_grid is not None:
        for k, v in enumerate(lr_grid):
            cfg.lr_grid[k] = float(v)
    if lam is not None:
        for k, v in enumerate(lam):
            cfg.lambda_[k] = float(v)
    cfg.stream = _stream_handle(stream)
    return cfg


def mlp_len(cfg) -> int:
    H, D = cfg.H, cfg.depth
    K = cfg.F_n + cfg.F_p + 2 * cfg.n_freq
    NO = 7 if cfg.rot_mode == ROT_QUAT else 6
    n = H * K + H + (D - 1) * (H * H + H) + NO * H + NO
    if cfg.time_enc == TIME_LEARNED:
        Ht, G2 = cfg.time_hidden, 2 * cfg.n_freq
        n += 2 * Ht + G2 * Ht + G2
    return n


def grid_len(cfg) -> int:
    return sum(cfg.res[l] ** 3 * cfg.F_p for l in range(cfg.L)) + cfg.res_n ** 3 * cfg.F_n


class Context:
    """Owns one npg context; arrays come back as numpy (host) copies."""

    def __init__(self, cfg, seq, mlp_init, device_inputs=False):
        self.cfg = cfg
        self.N, self.T = int(seq.x.shape[0]), int(len(seq.offsets) - 1)
        arrs = [np.ascontiguousarray(seq.x, dtype=np.float32),
                np.ascontiguousarray(seq.n, dtype=np.float32),
                np.ascontiguousarray(seq.faces, dtype=np.int32),
                np.ascontiguousarray(seq.points, dtype=np.float32),
                np.ascontiguousarray(seq.offsets, dtype=np.int64),
                np.ascontiguousarray(mlp_init, dtype=np.float32)]
        if device_inputs:
            import torch
            arrs = [torch.from_numpy(a).cuda() for a in arrs]
        x, n, f, p, o, m = arrs
        self.h = npg_create(cfg, x, n, f, p, o, seq.t_key, m)

    def close(self):
        npg_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            if getattr(self, "h", None):
                self.close()
        except Exception:
            pass

    def get(self, which):
        n = npg_size(self.h, which)
        dt = _BUF_DTYPE.get(which, np.float32)
        out = np.zeros(n // np.dtype(dt).itemsize, dtype=dt)
        return npg_get(self.h, which, out)

    def set(self, which, arr):
        dt = _BUF_DTYPE.get(which, np.float32)
        npg_set(self.h, which, np.ascontiguousarray(arr, dtype=dt))

    def forward(self):
        npg_forward(self.h)

    def loss(self):
        out = np.zeros(3)
        cd = np.zeros(self.T)
        npg_loss(self.h, out, cd)
        return out, cd

    def backward(self):
        npg_backward(self.h)

    def step(self):
        npg_step(self.h)

    def iteration(self):
        out = np.zeros(3)
        npg_iteration(self.h, out)
        return out


def _autograd():
    import torch

    class NpgLossFn(torch.autograd.Function):
        """L(grid, mlp) of one sequence (Eq. 8); backward runs npg_backward, the
        hand-written adjoint (stop-grad on w_conf and keyframe edge lengths)."""

        @staticmethod
        def forward(fctx, grid, mlp, handle):
            npg_set(handle, BUF_GRID, grid.detach().contiguous())
            npg_set(handle, BUF_MLP, mlp.detach().contiguous())
            npg_forward(handle)
            out = np.zeros(3)
            npg_loss(handle, out)
            fctx.handle = handle
            fctx.dev = grid.device
            return torch.tensor(out[0], dtype=torch.float64, device=grid.device)

        @staticmethod
        def backward(fctx, gout):
            h = fctx.handle
            npg_backward(h)
            gg = torch.empty(npg_size(h, BUF_GRID_GRAD) // 4, dtype=torch.float32, device=fctx.dev)
            gm = torch.empty(npg_size(h, BUF_MLP_GRAD) // 4, dtype=torch.float32, device=fctx.dev)
            npg_get(h, BUF_GRID_GRAD, gg)
            npg_get(h, BUF_MLP_GRAD, gm)
            s = gout.to(torch.float32)
            return gg * s, gm * s, None

    return NpgLossFn


def npg_loss_fn():
    """The torch.autograd.Function wrapping npg_forward + npg_loss / npg_backward."""
    return _autograd()
