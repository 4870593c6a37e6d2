"""The paper's iterative w_up scheme on the GPU against its oracle (needs a GPU).

pd_decimate_wup restates the removal sweep of section "Sub-sampling
algorithm" as parallel rounds; oracle.decimate_wup runs the same rounds
plainly on the CPU.  Density costs are exact, so the retained sets must be
identical, and so must the number of iterations.
"""
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


def _gpu(pd, ctx, x, k, m, leaf=0):
    g = pd.Grid(ctx, torch.from_numpy(np.ascontiguousarray(x)).cuda(), leaf_max=leaf)
    keep = pd.pd_decimate_wup(g, m, k=k).cpu().numpy()
    st = g.stats()
    g.free()
    return keep, st


@pytest.mark.parametrize("k", [1, 2, 4, 6])
def test_wup_random_clouds_equal_oracle(pd, k):
    ctx = pd.Context()
    for seed in range(3):
        x = synth.random_cloud(seed, 4000, 60)   # many duplicates and ties
        for ratio in (0.0, 0.1, 0.5, 1.0):
            m = oracle.target_count(len(x), ratio)
            keep, st = _gpu(pd, ctx, x, k, m)
            ref, it, _ = oracle.decimate_wup(x, k, m)
            assert int(keep.sum()) == m
            assert np.array_equal(keep, ref), (seed, ratio, int((keep != ref).sum()))
            assert st["iterations"] == it
    ctx.close()


@pytest.mark.parametrize("k,ratio", [(1, 0.25), (4, 0.1), (6, 0.1)])
def test_wup_room_scan_equals_oracle(pd, k, ratio):
    s = synth.room_scan(seed=0, n_az=1000, n_el=200)
    m = oracle.target_count(s.n, ratio)
    ctx = pd.Context()
    ref, it, _ = oracle.decimate_wup(s.xyz, k, m)
    for leaf in (12, 32):   # the cell size never changes the result
        keep, st = _gpu(pd, ctx, s.xyz, k, m, leaf)
        assert np.array_equal(keep, ref), (leaf, int((keep != ref).sum()))
        assert st["iterations"] == it
    ctx.close()


def test_wup_outdoor_sector_equals_oracle(pd):
    s = synth.outdoor_scan(seed=1, n_az=2000, n_el=400)
    m = oracle.target_count(s.n, 0.1)
    ctx = pd.Context()
    keep, _ = _gpu(pd, ctx, s.xyz, 4, m)
    ctx.close()
    assert np.array_equal(keep, oracle.decimate_wup(s.xyz, 4, m)[0])


def test_wup_rejects_unsupported_costs(pd):
    ctx = pd.Context()
    g = pd.Grid(ctx, torch.from_numpy(synth.random_cloud(0, 100, 50)).cuda())
    with pytest.raises(pd.PdError):
        pd.pd_decimate_wup(g, 10, k=7)
    g.free()
    ctx.close()
