"""npg_precondition_static: the allocation-free preconditioner entry point.

It exists for callers that cannot allocate device memory where they need the
preconditioner (GPU memory owned by another allocator, fixed memory budgets,
code that must not risk the implicit synchronisation of cudaMalloc/cudaFree).
Its output must equal npg_precondition's, call after call, although every call
reuses the same file-scope scratch array whose contents the previous call left.
This file is collected last on purpose.
"""
import ctypes as C
import os

import numpy as np
import pytest


@pytest.fixture(scope="module")
def npg():
    """The binding; builds libnpg.so when nvcc is available, else uses the
    library already built, else skips (the argument checks need no GPU but do
    need the library)."""
    import shutil
    from paper_2602_22212_gb300 import build
    if shutil.which(build.NVCC) is not None:
        build.build()
    elif not os.path.exists(build.LIB):
        pytest.skip("neither nvcc nor a built libnpg.so is available")
    from paper_2602_22212_gb300 import npg as mod
    return mod


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.gpu
def test_static_matches_allocating_entry_point_twice_in_a_row(npg):
    import torch
    s = torch.cuda.current_stream()
    # two different blocks back to back: the second call runs on the scratch
    # contents the first one left behind
    for r, F, lam, seed in ((37, 4, 1.35, 0), (64, 4, 6.8, 1)):
        g = torch.from_numpy(np.random.default_rng(seed).normal(size=r ** 3 * F)
                             .astype(np.float32)).cuda()
        want = torch.empty_like(g)
        got = torch.full_like(g, float("nan"))
        npg.npg_precondition(g, want, r, F, lam, stream=s)
        rc = npg._lib.npg_precondition_static(C.c_void_p(g.data_ptr()),
                                              C.c_void_p(got.data_ptr()), r, F, C.c_float(lam),
                                              C.c_void_p(s.cuda_stream))
        assert rc == npg.OK, npg.npg_last_error()
        torch.cuda.synchronize()
        w, o = want.cpu().numpy().astype(np.float64), got.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(o))
        assert _rel(o, w) <= 2e-6
    # a further call allocates nothing: the device's free memory is unchanged
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    rc = npg._lib.npg_precondition_static(C.c_void_p(g.data_ptr()), C.c_void_p(got.data_ptr()),
                                          r, F, C.c_float(lam), C.c_void_p(s.cuda_stream))
    assert rc == npg.OK, npg.npg_last_error()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_static_rejects_blocks_beyond_its_scratch(npg):
    x = C.c_void_p(16)
    rc = npg._lib.npg_precondition_static(x, x, 65, 4, C.c_float(0.4), None)  # 65^3*4 > 2^20
    assert rc == npg.EINVAL
    assert "static scratch limit" in npg.npg_last_error()
    assert npg._lib.npg_precondition_static(x, x, 600, 1, C.c_float(0.4), None) == npg.EINVAL
    # r = 102 with F = 1 is past the cube root of the limit
    assert npg._lib.npg_precondition_static(x, x, 102, 1, C.c_float(0.4), None) == npg.EINVAL
