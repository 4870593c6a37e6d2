"""Quality report of a decimated cloud, plain CPU version (oracle).

TEST INFRASTRUCTURE ONLY: the tests and the benchmark may import it; the
library never does.

Section "Results and Discussion" (the cube experiment) judges a decimated
cloud by the number of retained points within a growing radius of every
retained point.  On an evenly sampled surface the count grows linearly with
the neighbourhood's area pi r^2: the paper plots fractile bands of the counts
(0.01-0.99, 0.1-0.9, 0.25-0.75) and their mean against the area, takes the
least-squares slope as the density estimate, and reads R^2 and RMSE as the
goodness of fit.  Eq. 2's quantity, the smallest nearest-neighbour distance
d_p of the retained set, is reported beside it.

Every step follows the definition directly: brute-force counts (C), the
fractile as the smallest count reaching ceil(f P) points, and the regression
in exact rational arithmetic over the P * J samples (x = pi r_j^2 in m^2 as
a binary64 value, y = N_j(p)).
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

FRACTILES = (1, 10, 25, 50, 75, 90, 99)  # percent


def fractile(values, pct):
    """Smallest v such that at least ceil(pct/100 * P) of the values are <= v."""
    v = np.sort(np.asarray(values, dtype=np.int64))
    P = len(v)
    rank = max(1, -(-pct * P // 100))
    return int(v[rank - 1])


def area_m2(r_mm):
    r = float(r_mm) / 1000.0
    return math.pi * r * r


def regression(counts, radii_mm):
    """Least squares of y = counts[p, j] on x = pi r_j^2 over every (p, j).

    Returns (slope, intercept, r2, rmse) computed exactly (Fractions) from
    the binary64 areas and the integer counts, rounded to binary64 at the end.
    """
    counts = np.asarray(counts, dtype=np.int64)
    P, J = counts.shape
    xs = [Fraction(area_m2(r)) for r in radii_mm]
    N = P * J
    sx = sum(xs) * P
    sxx = sum(x * x for x in xs) * P
    col = [int(c) for c in counts.sum(axis=0)]
    sy = sum(col)
    syy = int((counts * counts).sum())
    sxy = sum(x * c for x, c in zip(xs, col))
    vx = sxx - sx * sx / N
    cv = sxy - sx * sy / N
    vy = Fraction(syy) - Fraction(sy * sy, N)
    if J < 2 or vx == 0:
        return (math.nan,) * 4
    slope = cv / vx
    icpt = Fraction(sy, N) - slope * sx / N
    r2 = cv * cv / (vx * vy) if vy != 0 else Fraction(1)
    ssres = vy - cv * cv / vx
    rmse = math.sqrt(float(ssres / N))
    return float(slope), float(icpt), float(r2), rmse


def report(xyz, keep, radii_mm):
    """The quality report of the retained points (keep None = all points)."""
    import oracle
    x = np.asarray(xyz, dtype=np.int32)
    if keep is not None:
        x = x[np.asarray(keep).astype(bool)]
    P = len(x)
    out = {"points": P, "radius_mm": list(radii_mm)}
    if P == 0:
        return out
    counts = oracle.radius_counts(x, radii_mm)
    out["mean"] = [float(c) / P for c in counts.sum(axis=0)]
    out["fractile"] = [[fractile(counts[:, j], f) for f in FRACTILES]
                       for j in range(len(radii_mm))]
    out["slope_per_m2"], out["intercept"], out["r2"], out["rmse"] = regression(counts, radii_mm)
    if P >= 2:
        d2, _, _ = oracle.knn_cost(x, 1, backend=oracle.KDTREE)
        out["min_spacing2_mm2"] = int(d2[:, 0].min())
        out["mean_spacing_mm"] = math.fsum(math.sqrt(float(v)) for v in d2[:, 0]) / P
    else:
        out["min_spacing2_mm2"] = -1
        out["mean_spacing_mm"] = 0.0
    out["counts"] = counts
    return out
