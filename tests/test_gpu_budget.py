"""Clouds beyond a device-memory budget: blocks in pinned host memory (needs a GPU).

With a budget set on the context, large blocks past it (and cold ones) are
allocated in pinned, mapped host memory and the kernels address them in place
(the second memory tier that stands in for the paper's out-of-core voxels,
section "Scaling to massive point clouds").  The placement must not change a
result: the retained sets equal the oracle's and the unbudgeted run's.
"""
import numpy as np
import pytest

import oracle
from paper_2311_17604_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MiB = 1 << 20


@pytest.fixture(scope="module")
def pd():
    from paper_2311_17604_gb300 import build
    build.build()
    import paper_2311_17604_gb300.pd as pdm
    return pdm


def _run(pd, ctx, s, m, **kw):
    g = pd.Grid(ctx, torch.from_numpy(s.xyz).cuda(),
                rgb=torch.from_numpy(s.rgb).cuda() if s.rgb is not None else None)
    keep = pd.pd_decimate_count(g, m, **kw).cpu().numpy()
    g.free()
    torch.cuda.synchronize()
    return keep


def test_no_budget_tracks_nothing(pd):
    ctx = pd.Context()
    mem = ctx.memory()
    assert mem["tracked"] == 0 and mem["host_peak"] == 0 and mem["budget"] == 0
    ctx.close()


@pytest.mark.parametrize("k", [1, 4])
def test_everything_spilled_equals_oracle(pd, k):
    """A 1-byte budget with no size floor beyond the library's 1 MiB puts every
    large block (points, neighbour lists, keys, cell table, sort buffers) in
    host memory."""
    s = synth.room_scan(seed=3, n_az=1000, n_el=200)
    m = oracle.target_count(s.n, 0.25)
    ctx = pd.Context()
    ctx.set_device_budget(1)
    keep = _run(pd, ctx, s, m, k=k)
    mem = ctx.memory()
    ctx.close()
    assert mem["tracked"] == 1 and mem["host_peak"] >= 8 * MiB
    assert mem["host_bytes"] == 0          # every host block was freed
    assert int(keep.sum()) == m
    assert np.array_equal(keep, oracle.decimate(s.xyz, k, m))


def test_partial_budget_weighted_equals_unbudgeted(pd):
    """A budget of half the unbudgeted peak: some blocks on each side; the
    colour-term result is the unbudgeted one bit for bit."""
    s = synth.room_scan(seed=5, n_az=2000, n_el=400, rgb=True)
    m = oracle.target_count(s.n, 0.2)
    kw = dict(k=1, term=pd.PD_TERM_COLOR, weight=0.3)
    ref = _run(pd, pd.Context(), s, m, **kw)          # untracked: all in device memory
    ref_ctx = pd.Context()
    ref_ctx.set_device_budget(1 << 50)    # tracked; only the cold blocks spill
    assert np.array_equal(_run(pd, ref_ctx, s, m, **kw), ref)
    peak = ref_ctx.memory()["device_peak"]
    ref_ctx.close()
    ctx = pd.Context()
    budget = peak // 2
    ctx.set_device_budget(budget)
    keep = _run(pd, ctx, s, m, **kw)
    mem = ctx.memory()
    ctx.close()
    assert mem["host_peak"] > 0
    assert mem["device_peak"] <= budget + 16 * MiB   # blocks under 1 MiB may pass it
    assert np.array_equal(keep, ref)


def test_host_entry_point_with_budget(pd):
    """pd_decimate_host under a budget: its input copies and keep staging are
    cold blocks, placed in host memory."""
    s = synth.room_scan(seed=7, n_az=1000, n_el=200)
    m = oracle.target_count(s.n, 0.3)
    ctx = pd.Context()
    ctx.set_device_budget(1 << 40)        # large: only cold blocks spill
    keep, _ = pd.pd_decimate_host(ctx, s.xyz, m, k=1)
    mem = ctx.memory()
    ctx.close()
    assert mem["host_peak"] >= s.n * 12
    assert np.array_equal(np.asarray(keep), oracle.decimate(s.xyz, 1, m))
