"""Failure paths of the context, made on the host (no GPU fault is caused):

  allocation   a caller-supplied allocator (npg_config.alloc) that refuses the
               k-th request: npg_create returns NPG_ENOMEM, leaves *out NULL
               and hands every block it did get back to the caller's free
  device wait  the device error word that a kernel sets when a bounded wait
               gives up, written here from the host: the next synchronising
               call returns NPG_ETIMEOUT and clears it, and the context stays
               usable
"""
import ctypes as C

import numpy as np
import pytest

from paper_2602_22212_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def npg():
    from paper_2602_22212_gb300 import build
    build.build()
    from paper_2602_22212_gb300 import npg as mod
    return mod


def _small(npg, seq):
    return npg.make_config(2, [8, 17], 2, 64, 2, slope=0.0, e_max=10)


class CountingAllocator:
    """Device blocks from torch's caching allocator; refuses request `fail_at`
    (0-based; None = never) and records what is still held."""

    def __init__(self, npg, fail_at):
        import torch
        self.torch = torch
        self.fail_at = fail_at
        self.calls = 0
        self.live = {}
        self.alloc_fn = npg.ALLOC_FN(self._alloc)
        self.free_fn = npg.FREE_FN(self._free)

    def _alloc(self, nbytes, user):
        k = self.calls
        self.calls += 1
        if self.fail_at is not None and k == self.fail_at:
            return None
        p = self.torch.cuda.caching_allocator_alloc(int(nbytes))
        self.live[p] = int(nbytes)
        return p

    def _free(self, ptr, user):
        assert ptr in self.live, "freed a block that was not handed out"
        del self.live[ptr]
        self.torch.cuda.caching_allocator_delete(ptr)

    def attach(self, cfg):
        cfg.alloc = self.alloc_fn
        cfg.free = self.free_fn
        cfg.alloc_user = None


def test_allocation_failure_returns_enomem_and_leaks_nothing(npg):
    seq = I.sphere_blob(subdiv=2, T=3, M=200, seed=0)
    mlp = I.mlp_init(2 + 2 + 8, 64, 2, 7, seed=0)
    # how many blocks a successful create takes
    ok = CountingAllocator(npg, None)
    cfg = _small(npg, seq)
    ok.attach(cfg)
    ctx = npg.Context(cfg, seq, mlp)
    n_blocks = ok.calls
    assert n_blocks > 10 and len(ok.live) == n_blocks
    ctx.close()
    assert not ok.live
    for k in sorted({0, 1, n_blocks // 2, n_blocks - 1}):
        a = CountingAllocator(npg, k)
        cfg = _small(npg, seq)
        a.attach(cfg)
        with pytest.raises(npg.NpgError) as ei:
            npg.Context(cfg, seq, mlp)
        assert ei.value.code == npg.ENOMEM, (k, str(ei.value))
        assert not a.live, (k, len(a.live))
    # a NULL out-pointer contract: *out stays NULL on failure
    a = CountingAllocator(npg, 0)
    cfg = _small(npg, seq)
    a.attach(cfg)
    arrs = [np.ascontiguousarray(v) for v in (seq.x.astype(np.float32),
                                              seq.n.astype(np.float32),
                                              seq.faces.astype(np.int32),
                                              seq.points.astype(np.float32),
                                              seq.offsets.astype(np.int64),
                                              mlp.astype(np.float32))]
    out = C.c_void_p(12345)
    rc = npg._lib.npg_create(C.byref(out), C.byref(cfg), arrs[0].ctypes.data,
                             arrs[1].ctypes.data, seq.N, arrs[2].ctypes.data, len(seq.faces),
                             arrs[3].ctypes.data, arrs[4].ctypes.data, seq.T, seq.t_key,
                             arrs[5].ctypes.data, arrs[5].size, 0)
    assert rc == npg.ENOMEM and not out.value and not a.live


def test_device_error_word_gives_etimeout_then_recovers(npg):
    seq = I.sphere_blob(subdiv=2, T=3, M=200, seed=1)
    mlp = I.mlp_init(2 + 2 + 8, 64, 2, 7, seed=1, zero_last=False)
    ctx = npg.Context(_small(npg, seq), seq, mlp)
    try:
        assert ctx.get(npg.BUF_DEVICE_ERROR)[0] == 0
        ctx.set(npg.BUF_DEVICE_ERROR, np.array([1], np.int32))
        assert ctx.get(npg.BUF_DEVICE_ERROR)[0] == 1  # reading does not clear it
        ctx.forward()
        with pytest.raises(npg.NpgError) as ei:
            ctx.loss()
        assert ei.value.code == npg.ETIMEOUT
        assert ctx.get(npg.BUF_DEVICE_ERROR)[0] == 0  # reported once, then cleared
        ctx.forward()
        loss, _ = ctx.loss()
        assert np.isfinite(loss[0]) and loss[0] > 0
        ctx.backward()
        ctx.step()
    finally:
        ctx.close()
