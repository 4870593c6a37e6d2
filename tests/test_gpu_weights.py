"""Colour and orientation weights on the GPU against hand-worked costs (needs a GPU).

The clouds and their exact costs are the hand-worked cases of
tests/test_oracle_weights.py (section "Additional cost terms", Eq. 11 with the
per-neighbour factor of Eq. 13 and the colour reading).  The kernels compute
each weight and each term in binary64 with the same rounding steps as the
oracle, so the costs must be within a few ulps of the exact values.
"""
import numpy as np
import pytest

import test_oracle_weights as hw

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pd():
    from paper_2311_17604_gb300 import build
    build.build()
    import paper_2311_17604_gb300.pd as pdm
    return pdm


@pytest.mark.parametrize("name", sorted(hw.CASES))
def test_gpu_weighted_cost_hand_worked(pd, name):
    xyz, rgb, nrm, term, a, k, expected = hw.CASES[name]
    ctx = pd.Context()
    xd = torch.from_numpy(xyz).cuda()
    rd = torch.from_numpy(rgb).cuda() if rgb is not None else None
    nd = torch.from_numpy(nrm).cuda() if nrm is not None else None
    for leaf in (4, 32):
        g = pd.Grid(ctx, xd, rgb=rd, leaf_max=leaf)
        cost, knn = pd.pd_knn_cost(g, k=k, term=term, weight=a, normals=nd)
        g.free()
        c = cost.cpu().numpy()
        for p, ex in enumerate(expected(a)):
            assert hw._close(float(c[p]), ex), (name, leaf, p, c[p], ex)
    ctx.close()
