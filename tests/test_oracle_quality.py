"""Pins for the oracle's quality report (no GPU).

Section "Results and Discussion" (cube experiment): neighbour counts against
neighbourhood area, their fractile bands, regression slope / R^2 / RMSE, and
Eq. 2's smallest spacing.  Each piece is tied to something other than the
oracle itself:
  * counts on a square lattice equal the Gauss circle counts (lattice points
    (i, j) != 0 with i^2 + j^2 <= (r/h)^2, listed by hand);
  * the regression equals numpy.polyfit on the expanded samples, R^2 the
    squared correlation coefficient, RMSE the root mean squared residual;
  * fractiles equal numpy.quantile with the inverted-CDF rule;
  * the lattice's smallest and mean spacing are its step.
"""
import math

import numpy as np
import pytest

from oracle import quality
from paper_2311_17604_gb300 import synth

# Gauss circle counts without the centre: #{(i,j) != 0 : i^2 + j^2 <= t^2}
GAUSS = {1.0: 4, 1.5: 8, 2.0: 12, 2.5: 20, 3.0: 28}


def _lattice(h=10, side=41):
    i, j = np.meshgrid(np.arange(side), np.arange(side), indexing="ij")
    xyz = np.zeros((side * side, 3), np.int32)
    xyz[:, 0] = (h * i).ravel()
    xyz[:, 1] = (h * j).ravel()
    return xyz, i.ravel(), j.ravel()


def test_lattice_counts_equal_gauss_circle(orc):
    h, side = 10, 41
    xyz, i, j = _lattice(h, side)
    radii = [int(t * h) for t in sorted(GAUSS)]
    counts = orc.radius_counts(xyz, radii)
    interior = (i >= 3) & (i < side - 3) & (j >= 3) & (j < side - 3)
    for col, t in enumerate(sorted(GAUSS)):
        assert np.all(counts[interior, col] == GAUSS[t])
    # the corner point sees a quarter of the disk (plus the two axis rays)
    corner = np.nonzero((i == 0) & (j == 0))[0][0]
    assert counts[corner, radii.index(20)] == 5  # (1,0) (2,0) (0,1) (0,2) (1,1)


def test_lattice_spacing_and_density(orc):
    h = 10
    xyz, _, _ = _lattice(h, 41)
    rep = quality.report(xyz, None, [10, 20, 30, 40])
    assert rep["min_spacing2_mm2"] == h * h
    assert rep["mean_spacing_mm"] == float(h)
    # an even lattice of 1 point per 100 mm^2 = 10^4 points per m^2: the
    # slope of count against area approaches it (boundary points see less)
    assert 0.8e4 < rep["slope_per_m2"] < 1.0e4
    assert rep["r2"] > 0.9


def test_regression_equals_polyfit(orc):
    x = synth.random_cloud(5, 400, 300)
    radii = [15, 30, 45, 60, 90]
    counts = orc.radius_counts(x, radii)
    slope, icpt, r2, rmse = quality.regression(counts, radii)
    X = np.repeat(np.array([[quality.area_m2(r) for r in radii]]), len(x), axis=0).ravel()
    Y = counts.astype(np.float64).ravel()
    b, a = np.polyfit(X, Y, 1)
    assert slope == pytest.approx(b, rel=1e-9) and icpt == pytest.approx(a, rel=1e-9, abs=1e-9)
    assert r2 == pytest.approx(np.corrcoef(X, Y)[0, 1] ** 2, rel=1e-9)
    res = Y - (b * X + a)
    assert rmse == pytest.approx(math.sqrt(np.mean(res * res)), rel=1e-7)


def test_fractiles_equal_inverted_cdf_quantile():
    rng = np.random.default_rng(3)
    for P in (1, 2, 7, 100, 1001):
        v = rng.integers(0, 40, size=P)
        for f in quality.FRACTILES:
            want = int(np.quantile(v, f / 100.0, method="inverted_cdf"))
            assert quality.fractile(v, f) == want, (P, f)


def test_report_of_subset_uses_retained_points_only(orc):
    x = synth.random_cloud(8, 600, 200)
    keep = np.zeros(600, np.uint8)
    keep[::3] = 1
    rep = quality.report(x, keep, [20, 40])
    sub = quality.report(x[keep.astype(bool)], None, [20, 40])
    assert rep["points"] == 200
    for key in ("mean", "fractile", "slope_per_m2", "r2", "min_spacing2_mm2"):
        assert rep[key] == sub[key]
