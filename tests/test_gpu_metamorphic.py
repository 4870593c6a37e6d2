"""Metamorphic checks of the GPU decimation (needs a GPU).

The retained set may not change under
  * an integer translation of the cloud (distances are unchanged);
  * scaling by 2 (every squared distance x 4: k = 1 orders integers, and for
    k >= 2 every binary64 term 1/d^2 and every partial sum scales by exactly
    1/4, barring subnormals, so the order of the costs is unchanged);
  * the stream the call runs on.
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


@pytest.fixture(scope="module")
def ctx(pd):
    c = pd.Context()
    yield c
    c.close()


def _keep(pd, ctx, xyz, m, k, stream=None):
    g = pd.Grid(ctx, torch.from_numpy(np.ascontiguousarray(xyz)).cuda(), stream=stream)
    keep = pd.pd_decimate_count(g, m, k=k, stream=stream)
    if stream is not None:
        stream.synchronize()
    out = keep.cpu().numpy()
    g.free()
    return out


@pytest.mark.parametrize("k", [1, 4])
def test_translation_scale_and_stream_invariance(pd, ctx, k):
    s = synth.room_scan(seed=9, n_az=400, n_el=100)
    m = oracle.target_count(s.n, 0.2)
    base = _keep(pd, ctx, s.xyz, m, k)
    shifted = s.xyz + np.array([1_000_003, -2_000_011, 3_000_017], dtype=np.int32)
    assert np.array_equal(_keep(pd, ctx, shifted, m, k), base)
    assert np.array_equal(_keep(pd, ctx, s.xyz * 2, m, k), base)
    side = torch.cuda.Stream()
    assert np.array_equal(_keep(pd, ctx, s.xyz, m, k, stream=side), base)
    assert int(base.sum()) == m
