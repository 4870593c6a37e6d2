"""The leaf-capacity autotuner (needs a GPU).

pd_autotune times whole decimations of a sample of the caller's cloud at
several octree leaf capacities and stores the fastest in the context.  The
capacity only changes speed: a grid built afterwards with the tuned capacity
must give exactly the result of the default capacity and of the oracle.
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


def test_autotune_picks_a_capacity_and_keeps_results(pd):
    ctx = pd.Context()
    s = synth.room_scan(seed=14, n_az=400, n_el=100)
    xd = torch.from_numpy(s.xyz).cuda()
    m = oracle.target_count(s.n, 0.25)
    leaf = pd.pd_autotune(ctx, xd, 0.25, k=4, sample=20000)
    assert leaf in (12, 16, 24, 32)
    g = pd.Grid(ctx, xd)                      # leaf_max 0: the tuned capacity
    tuned = pd.pd_decimate_count(g, m, k=4).cpu().numpy()
    assert g.stats()["leaf_max"] == leaf
    g.free()
    g = pd.Grid(ctx, xd, leaf_max=32)
    plain = pd.pd_decimate_count(g, m, k=4).cpu().numpy()
    assert g.stats()["leaf_max"] == 32
    g.free()
    assert np.array_equal(tuned, plain)
    assert np.array_equal(tuned, oracle.decimate(s.xyz, 4, m))
    ctx.close()


def test_autotune_rejects_bad_arguments(pd):
    ctx = pd.Context()
    x = torch.from_numpy(synth.random_cloud(0, 100, 50)).cuda()
    with pytest.raises(pd.PdError) as e:
        pd.pd_autotune(ctx, x, 1.5)
    assert e.value.code == pd.PD_EINVAL
    ctx.close()
