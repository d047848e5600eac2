"""Host-side checks of the C ABI (no GPU compute): the library loads, exports
every entry point include/npg.h declares, and its host-only logic (defaults,
argument validation, error reporting) behaves as documented."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "npg.h")


def _declared():
    names = []
    with open(HEADER) as f:
        for line in f:
            m = re.match(r"^NPG_API\s+[\w\s\*]+?\b(npg_\w+)\s*\(", line)
            if m:
                names.append(m.group(1))
    return names


@pytest.fixture(scope="module")
def npg():
    from paper_2602_22212_gb300 import build
    build.build()
    from paper_2602_22212_gb300 import npg as mod
    return mod


def test_header_declares_the_boundary():
    names = set(_declared())
    for n in ("npg_create", "npg_forward", "npg_loss", "npg_backward", "npg_step", "npg_destroy",
              "npg_iteration", "npg_get", "npg_set", "npg_get_state", "npg_set_state",
              "npg_nearest", "npg_precondition", "npg_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(npg):
    out = subprocess.run(["nm", "-D", "--defined-only", npg.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (npg_\w+)", out))
    for n in _declared():
        assert n in exported, n
        assert hasattr(npg._lib, n)
    # the binding wraps exactly the declared names
    assert set(npg.EXPORTED) == set(_declared())


def test_config_struct_matches_header_layout(npg):
    # npg_config_default is host-only: it fills the paper's defaults
    cfg = npg.npg_config_default(8, 16, 256, 4, 64, 3)
    assert [cfg.res[l] for l in range(8)] == [16, 50, 85, 119, 153, 187, 222, 256]
    np.testing.assert_allclose([cfg.lr_grid[l] for l in range(8)],
                               [0.005 * 2.5 ** l for l in range(8)], rtol=1e-6)
    np.testing.assert_allclose([cfg.lambda_[l] for l in range(8)],
                               [0.4 * 1.5 ** l for l in range(8)], rtol=1e-6)
    assert cfg.lr_grid[8] == pytest.approx(0.005) and cfg.lambda_[8] == pytest.approx(0.4)
    assert (cfg.F_n, cfg.res_n, cfg.n_freq, cfg.rot_mode) == (2, 4, 4, npg.ROT_QUAT)
    assert cfg.alpha == pytest.approx(0.1) and cfg.w_iso == pytest.approx(100.0)
    assert cfg.lr_mlp == pytest.approx(1e-3) and cfg.leaky_slope == pytest.approx(0.01)
    assert (cfg.adam_beta1, cfg.adam_beta2) == (pytest.approx(0.9), pytest.approx(0.999))
    assert cfg.stream is None and cfg.use_graph == 0


def test_invalid_arguments_are_rejected_before_any_device_work(npg):
    cfg = npg.npg_config_default(2, 4, 8, 2, 64, 2)
    out = C.c_void_p()
    x = np.zeros((3, 3), np.float32)
    f = np.array([[0, 1, 2]], np.int32)
    off = np.array([0, 3], np.int64)
    m = np.zeros(npg.mlp_len(cfg), np.float32)
    # N = 0
    rc = npg._lib.npg_create(C.byref(out), C.byref(cfg), x.ctypes.data, x.ctypes.data, 0,
                             f.ctypes.data, 1, x.ctypes.data, off.ctypes.data, 1, 0,
                             m.ctypes.data, m.size, 0)
    assert rc == npg.EINVAL and out.value is None
    assert "bad sizes" in npg.npg_last_error()
    # t_key out of range
    rc = npg._lib.npg_create(C.byref(out), C.byref(cfg), x.ctypes.data, x.ctypes.data, 3,
                             f.ctypes.data, 1, x.ctypes.data, off.ctypes.data, 1, 5,
                             m.ctypes.data, m.size, 0)
    assert rc == npg.EINVAL
    # bad config
    bad = npg.npg_config_default(2, 4, 8, 2, 64, 2)
    bad.res[0] = 1
    rc = npg._lib.npg_create(C.byref(out), C.byref(bad), x.ctypes.data, x.ctypes.data, 3,
                             f.ctypes.data, 1, x.ctypes.data, off.ctypes.data, 1, 0,
                             m.ctypes.data, m.size, 0)
    assert rc == npg.EINVAL and "res[0]" in npg.npg_last_error()
    # NULL context
    assert npg._lib.npg_forward(None, None) == npg.EINVAL
    assert npg._lib.npg_destroy(None) == npg.OK
    assert npg._lib.npg_size(None, npg.BUF_GRID) == 0
    # standalone ops validate their sizes
    assert npg._lib.npg_nearest(None, -1, None, 0, None, None, 0, None) == npg.EINVAL
    assert npg._lib.npg_precondition(None, None, 1, 1, 0.4, None) == npg.EINVAL
    # keyframe selection validates sizes, bias and host offsets before any device work
    pts = np.zeros((4, 3), np.float32)
    tk = C.c_int(-1)
    sel = lambda off, bias, T: npg._lib.npg_select_keyframe(
        pts.ctypes.data, off.ctypes.data, T, 0, bias, None, C.byref(tk), None)
    assert sel(np.array([0, 2, 4], np.int64), 1.0, 0) == npg.EINVAL
    assert sel(np.array([0, 2, 4], np.int64), 1.5, 2) == npg.EINVAL
    assert sel(np.array([1, 2, 4], np.int64), 1.0, 2) == npg.EINVAL
    assert sel(np.array([0, 2, 2], np.int64), 1.0, 2) == npg.EINVAL
    assert "no points" in npg.npg_last_error()
    assert tk.value == -1


def test_mlp_and_grid_lengths(npg):
    cfg = npg.make_config(4, [8, 27, 45, 64], 2, 64, 2)
    K = 2 + 2 + 8
    assert npg.mlp_len(cfg) == 64 * K + 64 + (64 * 64 + 64) + 7 * 64 + 7
    assert npg.grid_len(cfg) == (8 ** 3 + 27 ** 3 + 45 ** 3 + 64 ** 3) * 2 + 4 ** 3 * 2
