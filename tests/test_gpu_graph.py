"""Rounds replayed from a captured CUDA graph give the same result (needs a GPU).

From the third removal round on, a decimation of a cloud of up to 8M points
captures one round's launches into a CUDA graph (on a private stream) and
replays it while the grid layout stays the same; PD_ROUND_GRAPH forces the
choice.  Replayed and directly launched rounds must give bit-identical
retained sets (and, for the density cost, the oracle's).
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


@pytest.mark.parametrize("k,term", [(1, 0), (4, 0), (1, 1), (4, 1)])
def test_graph_rounds_equal_direct_rounds(pd, monkeypatch, k, term):
    s = synth.room_scan(seed=8, n_az=600, n_el=150, rgb=True)
    m = oracle.target_count(s.n, 0.2)
    kw = dict(k=k, term=term, weight=0.3 if term else 0.0)
    ctx = pd.Context()
    out = {}
    for mode in ("1", "0"):
        monkeypatch.setenv("PD_ROUND_GRAPH", mode)
        g = pd.Grid(ctx, torch.from_numpy(s.xyz).cuda(), rgb=torch.from_numpy(s.rgb).cuda())
        out[mode] = (pd.pd_decimate_count(g, m, **kw).cpu().numpy(), g.stats())
        g.free()
    ctx.close()
    (kg, sg), (kd, sd) = out["1"], out["0"]
    assert sg["graph_rounds"] > 0 and sd["graph_rounds"] == 0
    assert np.array_equal(kg, kd)
    assert int(kg.sum()) == m
    if term == 0:
        assert np.array_equal(kg, oracle.decimate(s.xyz, k, m))
