"""Pins for the oracle of the paper's iterative w_up scheme (no GPU).

Section "Sub-sampling algorithm": until lambda |C| points remain, recompute
every cost, take w_up as the cost of the lambda |C|-th cheapest point and
remove points above it while updating their reverse neighbours (an extended
k+b neighbourhood, dirty points wait for the next iteration).  The oracle
restates the removal sweep as parallel rounds (the largest key first among
interacting candidates).  Tied to:
  * the exact count of Eq. 1 (|C'| = m) and at least one removal per
    iteration;
  * closed forms: on well separated pairs with distinct gaps the scheme
    removes the higher index of the r tightest pairs, and on a 1-D lattice of
    equal costs it keeps {0, ..., m - 1}, as the sequential greedy does;
  * a second, plain-Python restatement recomputed from scratch;
  * context: it agrees with the sequential greedy on most points.
"""
import numpy as np
import pytest

from oracle import slow
from paper_2311_17604_gb300 import synth


@pytest.mark.parametrize("k", [1, 2, 4, 6])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_wup_equals_plain_restatement(orc, k, seed):
    x = synth.random_cloud(seed, 70, 25)   # duplicates and ties
    for m in (0, 1, 23, 69, 70):
        keep, it, _ = orc.decimate_wup(x, k, m)
        ref, it2 = slow.wup_from_scratch(x, k, m, orc.wup_width(k))
        assert int(keep.sum()) == m
        assert np.array_equal(keep, ref), (k, seed, m)
        assert it == it2


def test_wup_separated_pairs_closed_form(orc):
    rng = np.random.default_rng(5)
    P = 40
    gaps = rng.permutation(np.arange(3, 3 + P))
    xyz = np.zeros((2 * P, 3), np.int32)
    for i in range(P):
        xyz[2 * i] = (1000 * i, 0, 0)
        xyz[2 * i + 1] = (1000 * i + gaps[i], 0, 0)
    tight = np.argsort(gaps)
    for r in (1, 7, 20, 40):
        keep, _, _ = orc.decimate_wup(xyz, 1, 2 * P - r)
        want = np.ones(2 * P, np.uint8)
        want[2 * tight[:r] + 1] = 0
        assert np.array_equal(keep, want), r


def test_wup_lattice_line_keeps_lowest_indices(orc):
    x = synth.lattice_line(200, step=5)
    for m in (1, 50, 199):
        keep, _, _ = orc.decimate_wup(x, 1, m)
        assert np.array_equal(np.nonzero(keep)[0], np.arange(m))


def test_wup_iterations_and_agreement_with_greedy(orc):
    s = synth.room_scan(seed=2, n_az=300, n_el=80)
    for k in (1, 4, 6):
        m = orc.target_count(s.n, 0.25)
        keep, it, rounds = orc.decimate_wup(s.xyz, k, m)
        assert int(keep.sum()) == m
        assert 1 <= it <= rounds
        greedy = orc.decimate(s.xyz, k, m)
        assert (keep == greedy).mean() > 0.9
