"""Second, independent CPU oracle: greedy decimation recomputed from scratch.

TEST INFRASTRUCTURE ONLY.  Pure numpy / Python floats, no heap and no
incremental updates: before every removal it recomputes, for every live point,
the full sorted list of squared distances to the other live points and the
cost from it, then removes the point with the largest (cost, index) key.
It is quadratic per step, so it is meant for clouds of a few hundred points.

Definitions followed (arXiv 2311.17604):
  * Eq. 10 / Eq. 11: cost = sum over the k nearest of 1 / d^2, summed in
    ascending-distance order in binary64; k = 1 density-only compares d1^2 as
    integers.
  * Greedy removal of the highest cost (section "Computing per-sample costs"),
    larger index first among equal costs.
  * Optional neighbour weights for the orientation term (Eq. 13, read with an
    absolute value because estimated normals are unoriented) and the colour
    term (no formula printed in the paper; this library's reading).
Also here: an exhaustive enumerator of removal orders for tiny inputs and the
Eq. 2 optimum (largest achievable minimum spacing) by brute force.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

TERM_NONE, TERM_COLOR, TERM_ORIENT = 0, 1, 2


def _weight(term, a, rgb, nrm, p, q):
    if term == TERM_COLOR:
        dr = float(rgb[p, 0]) - float(rgb[q, 0])
        dg = float(rgb[p, 1]) - float(rgb[q, 1])
        db = float(rgb[p, 2]) - float(rgb[q, 2])
        s = dr * dr
        s = s + dg * dg
        s = s + db * db
        return 1.0 - a * (math.sqrt(s) / (255.0 * math.sqrt(3.0)))
    if term == TERM_ORIENT:
        d = float(nrm[p, 0]) * float(nrm[q, 0])
        d = d + float(nrm[p, 1]) * float(nrm[q, 1])
        d = d + float(nrm[p, 2]) * float(nrm[q, 2])
        return 1.0 - a * (1.0 - abs(d))
    return 1.0


def keys_from_scratch(xyz, live, k, term=TERM_NONE, a=0.0, rgb=None, nrm=None):
    """Key of every live point computed from scratch.

    Returns a list of (primary, index) tuples (None for removed points) whose
    Python tuple order is the removal order: the larger key goes first.
    primary is -d1^2 for the k = 1 density cost (an exact integer) and the
    binary64 cost otherwise.
    """
    xyz = np.asarray(xyz, dtype=np.int64)
    ids = np.nonzero(live)[0]
    keys = [None] * len(xyz)
    for p in ids:
        others = ids[ids != p]
        d = xyz[others] - xyz[p]
        d2 = (d * d).sum(axis=1)
        # ascending (d2, index) order; equal distances sort by index
        order = np.lexsort((others, d2))[:k]
        if k == 1 and term == TERM_NONE:
            prim = -int(d2[order[0]]) if len(order) else -(1 << 62)
        else:
            c = 0.0
            for j in order:
                w = _weight(term, a, rgb, nrm, p, int(others[j]))
                dd = float(d2[j])
                c = c + (w / dd if dd != 0.0 else math.inf)
            prim = c
        keys[p] = (prim, int(p))
    return keys


def greedy_from_scratch(xyz, k, m, term=TERM_NONE, a=0.0, rgb=None, nrm=None):
    """Remove the max-key live point until m remain; returns (keep, order)."""
    n = len(xyz)
    live = np.ones(n, dtype=bool)
    order = []
    while live.sum() > m:
        keys = keys_from_scratch(xyz, live, k, term, a, rgb, nrm)
        best = max(kk for kk in keys if kk is not None)
        live[best[1]] = False
        order.append(best[1])
    return live.astype(np.uint8), order


def rounds_from_scratch(xyz, k, m, danger=True, band=None):
    """Parallel removal rounds recomputed from scratch every round (density
    cost), following the rules of the library's rounds:
      R2  the key is among the `need` = live - m largest;
      R1  the key beats the key of every live q != p that shares a
          tie-inclusive k-ball with p: d^2(p, q) <= r_k^2(p) or
          d^2(p, q) <= r_k^2(q), r_k^2 the k-th smallest squared distance to
          the other live points;
      R3  (danger=True) with tau the least key of the R1 and R2 candidates
          and "low" the live points of key below tau, a candidate p is
          rejected when some live q of larger key has d^2(q, p) < lambda(q),
          the k-th smallest squared distance from q to a low point other than
          q (infinite when fewer than k low points exist).
    Every point left after the rules goes at once.  R1 and R2 alone are the
    exactness argument for k = 1; for k >= 2 a removal can pull a point into
    a larger key's k-ball later, which R3 rules out.  band (a fraction of the
    live points, as the library's rounds use): R2 takes the rank-th largest
    key, rank = max(1, min(floor(band * live), need)), in place of the
    need-th, and R3's tau is that key.  Returns (keep, rounds).
    """
    x = np.asarray(xyz, dtype=np.int64)
    live = np.ones(len(x), dtype=bool)
    big = np.iinfo(np.int64).max
    rounds = 0
    while live.sum() > m:
        rounds += 1
        keys = keys_from_scratch(x, live, k)
        ids = np.nonzero(live)[0]
        need = len(ids) - m
        rank = need if band is None else max(1, min(int(band * len(ids)), need))
        kstar = sorted((keys[p] for p in ids), reverse=True)[rank - 1]
        d = x[ids][:, None, :] - x[ids][None, :, :]
        d2 = (d * d).sum(axis=2)
        np.fill_diagonal(d2, big)
        rk = np.sort(d2, axis=1)[:, min(k, len(ids) - 1) - 1]
        cand = []
        for a, p in enumerate(ids):
            if keys[p] < kstar:
                continue
            ok = True
            for b, q in enumerate(ids):
                if a != b and (d2[a, b] <= rk[a] or d2[a, b] <= rk[b]) and not keys[p] > keys[q]:
                    ok = False
                    break
            if ok:
                cand.append(a)
        if danger:
            tau = kstar if band is not None else min(keys[ids[a]] for a in cand)
            low = np.array([keys[q] < tau for q in ids])
            lam = np.full(len(ids), big, dtype=np.int64)
            for b, q in enumerate(ids):
                if keys[q] >= tau:
                    dl = np.sort(d2[b][low & (np.arange(len(ids)) != b)])
                    if len(dl) >= k:
                        lam[b] = dl[k - 1]
            cand = [a for a in cand
                    if not any(b != a and keys[q] > keys[ids[a]] and
                               (lam[b] == big or d2[b, a] < lam[b])
                               for b, q in enumerate(ids))]
        live[ids[cand]] = False  # never empty: the largest key always qualifies
    return live.astype(np.uint8), rounds


def greedy_orders_exhaustive(xyz, k, m):
    """All removal sequences of length n - m whose every step removes the key max.

    Enumerates every ordered sequence of distinct points and keeps those in
    which each removed point holds the largest key among the live points at
    that step.  The greedy's tie-break makes keys distinct, so exactly one
    sequence must qualify.
    """
    n = len(xyz)
    good = []
    for seq in itertools.permutations(range(n), n - m):
        live = np.ones(n, dtype=bool)
        ok = True
        for p in seq:
            keys = keys_from_scratch(xyz, live, k)
            if max(kk for kk in keys if kk is not None)[1] != p:
                ok = False
                break
            live[p] = False
        if ok:
            good.append(list(seq))
    return good


def min_spacing2(xyz, sel=None):
    """Smallest squared distance between two selected points (Eq. 2 objective)."""
    x = np.asarray(xyz, dtype=np.int64)
    if sel is not None:
        x = x[np.asarray(sel, dtype=bool)]
    if len(x) < 2:
        return math.inf
    d = x[:, None, :] - x[None, :, :]
    d2 = (d * d).sum(axis=2)
    np.fill_diagonal(d2, np.iinfo(np.int64).max)
    return int(d2.min())


def best_spacing2(xyz, m):
    """Eq. 2 optimum by brute force: max over |C'| = m of the min squared spacing."""
    n = len(xyz)
    best = -1
    for sub in itertools.combinations(range(n), m):
        sel = np.zeros(n, dtype=bool)
        sel[list(sub)] = True
        best = max(best, min_spacing2(xyz, sel))
    return best


def wup_from_scratch(xyz, k, m, S):
    """The iterative w_up scheme with parallel removal rounds, written out
    plainly (pure Python lists, brute-force neighbours) as a second check of
    the C oracle's orc_decimate_wup.  Returns (keep, iterations)."""
    x = [tuple(int(v) for v in p) for p in np.asarray(xyz)]
    n = len(x)
    live = [True] * n

    def d2(a, b):
        return sum((x[a][t] - x[b][t]) ** 2 for t in range(3))

    def cost_of(p, lst):
        c = 0.0
        for q in lst[:k]:
            dd = d2(p, q)
            c = c + (1.0 / dd if dd else math.inf)
        return c

    iters = 0
    while sum(live) > m:
        iters += 1
        nbr, key, dirty = {}, {}, set()
        for p in range(n):
            if live[p]:
                others = sorted((d2(p, q), q) for q in range(n) if q != p and live[q])
                nbr[p] = [q for _, q in others[:S]]
                key[p] = (cost_of(p, nbr[p]), p)
        order = sorted((key[p] for p in key), reverse=True)
        tau = order[sum(live) - m - 1]
        while True:
            cand = {p for p in key if live[p] and p not in dirty and key[p] >= tau}
            if not cand:
                break
            blocked = set()
            for q in cand:
                for x_ in nbr[q][:k]:
                    if key[q] > key[x_]:
                        blocked.add(x_)
                    elif x_ in cand and key[x_] > key[q]:
                        blocked.add(q)
            picks = cand - blocked
            for p in picks:
                live[p] = False
            for p in list(key):
                if not live[p]:
                    continue
                kept = [q for q in nbr[p] if live[q]]
                if len(kept) != len(nbr[p]):
                    nbr[p] = kept
                    if len(kept) >= k:
                        key[p] = (cost_of(p, kept), p)
                    else:
                        dirty.add(p)
            if sum(live) <= m:
                break
    return np.array(live, dtype=np.uint8), iters
