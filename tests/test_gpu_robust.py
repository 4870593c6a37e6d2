"""Failure and fallback paths of the decimation (needs a GPU; no fault is induced).

  * The context's allocator returns NULL on its N-th request (a host-side
    fault injection, for every N the call makes): the failing call returns
    PD_ENOMEM, and every device block the library took is given back.
  * Rounds the device cannot settle: a danger-pair capacity of a few pairs
    (the PD_PAIR_CAP diagnostic) makes k >= 2 rounds overflow, so the host
    falls back to removing the global maximum; a 1-D lattice of equal costs
    makes the k = 1 fixpoint need more sweeps than the device runs.  Both must
    still give the oracle's retained set.
"""
import ctypes
import os

import numpy as np
import pytest

import oracle
from paper_2311_17604_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pd():
    from paper_2311_17604_gb300 import build
    build.build()
    import paper_2311_17604_gb300.pd as pdm
    return pdm


class FailingAllocator:
    """pd_allocator over torch's caching allocator that fails its N-th call."""

    def __init__(self, pd, fail_at):
        self.calls = 0
        self.live = {}
        self.fail_at = fail_at

        @ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
        def _alloc(user, nbytes, stream):
            self.calls += 1
            if self.calls == self.fail_at:
                return None
            p = torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
            self.live[int(p)] = int(nbytes)
            return p

        @ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
        def _free(user, ptr, stream):
            self.live.pop(int(ptr), None)
            torch.cuda.caching_allocator_delete(int(ptr))

        self._cb = (_alloc, _free)
        self.a = pd.pd_allocator(_alloc, _free, None)
        h = ctypes.c_void_p()
        assert pd.lib().pd_ctx_create(ctypes.byref(self.a), ctypes.byref(h)) == 0
        self.h = h

    def close(self, pd):
        pd.lib().pd_ctx_destroy(self.h)


def _run(pd, ctx_h, xd, n, k, m):
    """build + decimate through the C ABI; returns (status, keep or None)."""
    L = pd.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    g = ctypes.c_void_p()
    rc = L.pd_build_grid(ctx_h, ctypes.c_void_p(xd.data_ptr()), None, n, None, stream,
                         ctypes.byref(g))
    if rc:
        return rc, None
    keep = torch.empty(n, dtype=torch.uint8, device="cuda")
    cp = pd.cost_params(k)
    rc = L.pd_decimate_count(g, ctypes.byref(cp), m, ctypes.c_void_p(keep.data_ptr()), stream)
    L.pd_grid_free(g)
    return rc, keep


@pytest.mark.parametrize("k", [1, 4])
def test_allocator_failure_at_every_request(pd, k):
    s = synth.room_scan(seed=3, n_az=120, n_el=40)
    xd = torch.from_numpy(s.xyz).cuda()
    m = oracle.target_count(s.n, 0.25)
    ref = oracle.decimate(s.xyz, k, m)
    probe = FailingAllocator(pd, fail_at=0)          # count the requests of one clean run
    rc, keep = _run(pd, probe.h, xd, s.n, k, m)
    assert rc == 0 and np.array_equal(keep.cpu().numpy(), ref)
    total = probe.calls
    assert not probe.live
    probe.close(pd)
    assert total > 10
    for fail_at in range(1, total + 1):
        fa = FailingAllocator(pd, fail_at)
        rc, keep = _run(pd, fa.h, xd, s.n, k, m)
        torch.cuda.synchronize()
        assert rc == pd.PD_ENOMEM, (fail_at, rc)
        assert not fa.live, (fail_at, len(fa.live))   # nothing leaked
        fa.close(pd)


def test_overflowing_danger_rounds_settle_on_host(pd, monkeypatch):
    s = synth.room_scan(seed=4, n_az=200, n_el=60)
    m = oracle.target_count(s.n, 0.3)
    ref = oracle.decimate(s.xyz, 4, m)
    monkeypatch.setenv("PD_PAIR_CAP", "8")
    ctx = pd.Context()
    g = pd.Grid(ctx, torch.from_numpy(s.xyz).cuda())
    keep = pd.pd_decimate_count(g, m, k=4).cpu().numpy()
    st = g.stats()
    g.free()
    ctx.close()
    assert np.array_equal(keep, ref)
    assert st["rounds"] > 0


def test_long_tie_chains_settle_on_host(pd):
    x = synth.lattice_line(3000, step=7)          # equal costs: chains of index ties
    ctx = pd.Context()
    for m in (1, 700, 2999):
        g = pd.Grid(ctx, torch.from_numpy(x).cuda())
        keep = pd.pd_decimate_count(g, m, k=1).cpu().numpy()
        g.free()
        assert np.array_equal(keep, oracle.decimate(x, 1, m))
    ctx.close()


@pytest.mark.parametrize("sweeps", ["1", "3"])
def test_k1_rounds_settled_on_host_after_few_sweeps(pd, monkeypatch, sweeps):
    """PD_FIX_SWEEPS caps the device sweeps of the k = 1 fixpoint, so that
    ordinary rounds are settled on the host; the result is the oracle's."""
    s = synth.room_scan(seed=6, n_az=500, n_el=100)
    m = oracle.target_count(s.n, 0.2)
    monkeypatch.setenv("PD_FIX_SWEEPS", sweeps)
    ctx = pd.Context()
    g = pd.Grid(ctx, torch.from_numpy(s.xyz).cuda())
    keep = pd.pd_decimate_count(g, m, k=1).cpu().numpy()
    g.free()
    ctx.close()
    assert np.array_equal(keep, oracle.decimate(s.xyz, 1, m))
