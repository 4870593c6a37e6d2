"""Pins for the colour and orientation neighbour weights of the oracle (no GPU).

Section "Additional cost terms" weights each of the k nearest neighbours of
p (Eq. 13 for normals; the colour term is described in words, with no
formula).  The library reads both as a per-neighbour factor w(p, q) in the
sum of Eq. 11:

    cost_p = sum over q in N_k(p), nearest first, of w(p, q) / d(p, q)^2
    colour       w = 1 - a * ||rgb_p - rgb_q||_2 / (255 * sqrt 3)
    orientation  w = 1 - a * (1 - |n_p . n_q|)

Each case below is a cloud of 4-5 points with hand-picked integer distances
(no ties) and hand-picked colours or normals whose weights are known in
closed form: identical colours give 1, black against white gives 1 - a, a
pure red difference gives 1 - a / sqrt 3; parallel and antiparallel normals
give 1, orthogonal ones 1 - a, a 60 degree angle 1 - a / 2.  The expected
cost of every point is the whole Eq. 11 / Eq. 13 sum worked out exactly
(rational arithmetic, and 50-digit decimals where a square root appears), so
the check covers the neighbour order, the distances and the weights together.
A wrong normaliser (255 instead of 255 sqrt 3), a missing absolute value or a
flipped sign (1 - a x instead of 1 - a (1 - x)) moves some cost by more than
1 %; the last test plants each of those mistakes in the pure-Python oracle
and checks that the pins catch it.
"""
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest

from oracle import slow

getcontext().prec = 50

TOL = 1e-14  # relative; the oracle rounds each of a few binary64 operations


def _dec(x) -> Decimal:
    f = Fraction(x)
    return Decimal(f.numerator) / Decimal(f.denominator)


def _close(got: float, exact: Decimal) -> bool:
    return abs(_dec(got) - exact) <= Decimal(TOL) * abs(exact)


# ------------------------------------------------------------ colour (k = 2)
# P0 black, P1 white, P2 pure red, P3 black.
COLOUR_XYZ = np.array([[0, 0, 0], [30, 0, 0], [0, 40, 0], [0, 0, -20]], np.int32)
COLOUR_RGB = np.array([[0, 0, 0], [255, 255, 255], [255, 0, 0], [0, 0, 0]], np.uint8)
A_COLOUR = 0.3


def _colour_expected(a):
    """Eq. 11 with the colour factor, k = 2, worked out by hand.

    Squared distances: P0-P3 400, P0-P1 900, P1-P3 1300, P0-P2 1600,
    P2-P3 2000, P1-P2 2500.  Weights: black/black 1, black/white 1 - a,
    red/black 1 - a/sqrt 3 (difference (255, 0, 0): 255 / (255 sqrt 3)).
    """
    A = _dec(a)
    s3 = Decimal(3).sqrt()
    w_same, w_bw, w_red = Decimal(1), 1 - A, 1 - A / s3
    return [
        w_same / 400 + w_bw / 900,      # P0: P3 (400), P1 (900)
        w_bw / 900 + w_bw / 1300,       # P1: P0 (900), P3 (1300)
        w_red / 1600 + w_red / 2000,    # P2: P0 (1600), P3 (2000)
        w_same / 400 + w_bw / 1300,     # P3: P0 (400), P1 (1300)
    ]


# A partial colour difference (100, 50, 20): ||.|| = sqrt(12900), k = 1.
PARTIAL_XYZ = np.array([[0, 0, 0], [7, 0, 0], [0, 0, 500]], np.int32)
PARTIAL_RGB = np.array([[200, 100, 50], [100, 50, 30], [0, 0, 0]], np.uint8)


def _partial_expected(a):
    A = _dec(a)
    w01 = 1 - A * Decimal(12900).sqrt() / (255 * Decimal(3).sqrt())
    # P2 (0,0,500) is nearest to P0: d^2 = 250000; colour (200,100,50) vs 0.
    w20 = 1 - A * Decimal(200 ** 2 + 100 ** 2 + 50 ** 2).sqrt() / (255 * Decimal(3).sqrt())
    return [w01 / 49, w01 / 49, w20 / 250000]


# ------------------------------------------------------------ orientation (k = 4)
S60 = np.float32(np.sqrt(3.0) / 2.0)  # sin 60 deg in float32; (S60, 0, 1/2) . (0, 0, 1) = 1/2
ORIENT_XYZ = np.array([[0, 0, 0], [10, 0, 0], [0, 20, 0], [0, 0, 30], [0, 0, -50]], np.int32)
ORIENT_NRM = np.array([[0, 0, 1], [0, 0, 1], [0, 0, -1], [1, 0, 0], [S60, 0, 0.5]], np.float32)
A_ORIENT = 0.5


def _orient_expected(a):
    """Eq. 13 with |n_p . n_q|, k = 4, worked out by hand (exact rationals).

    Squared distances from P0: P1 100, P2 400, P3 900, P4 2500; P1-P2 500,
    P1-P3 1000, P2-P3 1300, P1-P4 2600, P2-P4 2900, P3-P4 6400.
    """
    A = Fraction(a)
    s = Fraction(float(S60))
    half = Fraction(1, 2)
    par = anti = Fraction(1)           # |+1|, |-1|
    orth = 1 - A                        # |0|
    sixty = 1 - A * (1 - half)          # |1/2|
    w3_4 = 1 - A * (1 - s)              # (1,0,0) . (s,0,1/2) = s
    exact = [
        par / 100 + anti / 400 + orth / 900 + sixty / 2500,                  # P0: P1 P2 P3 P4
        par / 100 + anti / 500 + orth / 1000 + sixty / 2600,                 # P1: P0 P2 P3 P4
        anti / 400 + anti / 500 + orth / 1300 + sixty / 2900,                # P2: P0 P1 P3 P4
        orth / 900 + orth / 1000 + orth / 1300 + w3_4 / 6400,                # P3: P0 P1 P2 P4
        sixty / 2500 + sixty / 2600 + sixty / 2900 + w3_4 / 6400,            # P4: P0 P1 P2 P3
    ]
    return [_dec(e) for e in exact]


CASES = {
    "colour_k2": (COLOUR_XYZ, COLOUR_RGB, None, slow.TERM_COLOR, A_COLOUR, 2, _colour_expected),
    "colour_partial_k1": (PARTIAL_XYZ, PARTIAL_RGB, None, slow.TERM_COLOR, A_COLOUR, 1,
                          _partial_expected),
    "orient_k4": (ORIENT_XYZ, None, ORIENT_NRM, slow.TERM_ORIENT, A_ORIENT, 4, _orient_expected),
}


def _slow_costs(xyz, rgb, nrm, term, a, k):
    keys = slow.keys_from_scratch(xyz, np.ones(len(xyz), bool), k, term=term, a=a, rgb=rgb,
                                  nrm=nrm)
    return [kk[0] for kk in keys]


@pytest.mark.parametrize("name", sorted(CASES))
def test_weighted_cost_hand_worked_c_oracle(orc, name):
    xyz, rgb, nrm, term, a, k, expected = CASES[name]
    for backend in (orc.BRUTE, orc.KDTREE):
        _, _, cost = orc.knn_cost(xyz, k, term=term, a=a, rgb=rgb, nrm=nrm, backend=backend)
        for p, ex in enumerate(expected(a)):
            assert _close(cost[p], ex), (name, p, cost[p], ex)


@pytest.mark.parametrize("name", sorted(CASES))
def test_weighted_cost_hand_worked_slow_oracle(name):
    xyz, rgb, nrm, term, a, k, expected = CASES[name]
    for p, (got, ex) in enumerate(zip(_slow_costs(xyz, rgb, nrm, term, a, k), expected(a))):
        assert _close(got, ex), (name, p, got, ex)


def test_weighted_removal_order_hand_worked(orc):
    """The greedy pops the largest weighted cost first: with the colour case
    the two black points near each other (P0, P3: 1/400 + ...) outrank the
    rest, and of those P0 (its second neighbour is nearer) goes first."""
    ex = _colour_expected(A_COLOUR)
    order_by_hand = sorted(range(4), key=lambda p: (ex[p], p), reverse=True)
    _, order, _ = orc.decimate(COLOUR_XYZ, 2, 1, term=slow.TERM_COLOR, a=A_COLOUR,
                               rgb=COLOUR_RGB, want_order=True)
    # the first pop is fixed by the initial costs alone
    assert int(order[0]) == order_by_hand[0] == 0


def _mutant(kind):
    import math

    def w(term, a, rgb, nrm, p, q):
        if term == slow.TERM_COLOR:
            d = [float(rgb[p, i]) - float(rgb[q, i]) for i in range(3)]
            dist = math.sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2])
            if kind == "normaliser":
                return 1.0 - a * (dist / (255.0 * 3.0))
            if kind == "sign":
                return 1.0 - a * (1.0 - dist / (255.0 * math.sqrt(3.0)))
            return 1.0 - a * (dist / (255.0 * math.sqrt(3.0)))
        if term == slow.TERM_ORIENT:
            d = sum(float(nrm[p, i]) * float(nrm[q, i]) for i in range(3))
            if kind == "abs":
                return 1.0 - a * (1.0 - d)
            if kind == "sign":
                return 1.0 - a * abs(d)
            return 1.0 - a * (1.0 - abs(d))
        return 1.0
    return w


@pytest.mark.parametrize("kind", ["normaliser", "abs", "sign"])
def test_pins_catch_planted_weight_mistakes(monkeypatch, kind):
    """Plant a plausible mistake in the pure-Python oracle's weight and check
    that at least one hand-worked case fails by more than 1 %."""
    monkeypatch.setattr(slow, "_weight", _mutant(kind))
    worst = 0.0
    for name, (xyz, rgb, nrm, term, a, k, expected) in CASES.items():
        for got, ex in zip(_slow_costs(xyz, rgb, nrm, term, a, k), expected(a)):
            worst = max(worst, float(abs(_dec(got) - ex) / abs(ex)))
    assert worst > 0.01, (kind, worst)
