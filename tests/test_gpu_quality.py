"""Quality report on the GPU against the oracle (needs a GPU).

Section "Results and Discussion" (cube experiment): neighbour counts of the
retained points within growing radii, their fractile bands and mean, the
regression of count on area (slope = density estimate, R^2, RMSE) and Eq. 2's
smallest spacing.  Integer results (counts, fractiles, spacing) must equal
the oracle's exactly; the regression and the mean spacing are binary64 values
computed in another order, so they must agree to 1e-9 relative.
"""
import numpy as np
import pytest

import oracle
from oracle import quality
from paper_2311_17604_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pd():
    from paper_2311_17604_gb300 import build
    build.build()
    import paper_2311_17604_gb300.pd as pdm
    return pdm


def _check(got, ref):
    assert got["points"] == ref["points"]
    if ref["points"] == 0:
        return
    assert got["fractile"] == ref["fractile"]
    assert np.allclose(got["mean"], ref["mean"], rtol=1e-12, atol=0)
    assert got["min_spacing2_mm2"] == ref["min_spacing2_mm2"]
    if ref["points"] >= 2:
        assert got["mean_spacing_mm"] == pytest.approx(ref["mean_spacing_mm"], rel=1e-9)
    for key in ("slope_per_m2", "intercept", "r2", "rmse"):
        if np.isnan(ref[key]):
            assert np.isnan(got[key])
        else:
            assert got[key] == pytest.approx(ref[key], rel=1e-9, abs=1e-9), key


@pytest.mark.parametrize("case", ["room_k1", "room_k4", "random_all", "lattice"])
def test_quality_report_equals_oracle(pd, case):
    ctx = pd.Context()
    if case == "lattice":
        i, j = np.meshgrid(np.arange(60), np.arange(60), indexing="ij")
        x = np.zeros((3600, 3), np.int32)
        x[:, 0], x[:, 1] = (10 * i).ravel(), (10 * j).ravel()
        keep = None
        radii = [10, 15, 20, 25, 30]
    elif case == "random_all":
        x = synth.random_cloud(4, 8000, 400)   # duplicates: spacing 0
        keep = None
        radii = [5, 10, 20, 40]
    else:
        s = synth.room_scan(seed=1, n_az=400, n_el=100)
        x = s.xyz
        k = 1 if case == "room_k1" else 4
        m = oracle.target_count(s.n, 0.2)
        g = pd.Grid(ctx, torch.from_numpy(x).cuda())
        keep = pd.pd_decimate_count(g, m, k=k).cpu().numpy()
        g.free()
        radii = [20, 40, 60, 80, 100, 150, 200]
    xd = torch.from_numpy(x).cuda()
    kd = torch.from_numpy(keep).cuda() if keep is not None else None
    got = pd.pd_quality_report(ctx, xd, kd, radii)
    ctx.close()
    ref = quality.report(x, keep, radii)
    _check(got, ref)


def test_quality_report_edge_cases(pd):
    ctx = pd.Context()
    x = torch.from_numpy(synth.random_cloud(1, 50, 100)).cuda()
    none = torch.zeros(50, dtype=torch.uint8, device="cuda")
    assert pd.pd_quality_report(ctx, x, none, [10])["points"] == 0
    one = none.clone()
    one[7] = 1
    r = pd.pd_quality_report(ctx, x, one, [10, 20])
    assert r["points"] == 1 and r["min_spacing2_mm2"] == -1 and r["mean"] == [0.0, 0.0]
    single = pd.pd_quality_report(ctx, x, None, [30])   # one radius: no regression
    assert np.isnan(single["slope_per_m2"])
    with pytest.raises(pd.PdError):
        pd.pd_quality_report(ctx, x, None, [20, 10])     # radii must ascend
    with pytest.raises(pd.PdError):
        pd.pd_quality_report(ctx, x, None, list(range(1, 40)))
    ctx.close()
