"""Pins of the oracle's canonical mode order (the output contract's ordering).

Modes are reported by density score descending; equal scores are ordered by
their coordinates, lexicographically ascending (first coordinate first).  The
expected orders below were worked out by hand from that rule, and a brute-force
comparison sort over all pairs checks random cases with many exact ties.  A
plausible slip in the oracle (ascending scores, coordinates compared last
first or descending, an unstable tie) fails one of these.
"""
import functools

import numpy as np
import pytest

import oracle as orc
from fms_compare import order_violations


def test_hand_case_score_then_coordinates():
    modes = np.array([[1.0, 2.0],    # 0: score 2
                      [0.0, 5.0],    # 1: score 3
                      [1.0, 1.0],    # 2: score 2, before 0 ([1,1] < [1,2])
                      [0.0, 9.0],    # 3: score 1, before 4 (first coordinate 0 < 1)
                      [1.0, 0.0],    # 4: score 1
                      [-2.0, 7.0]])  # 5: score 3, before 1 (-2 < 0)
    scores = np.array([2.0, 3.0, 2.0, 1.0, 1.0, 3.0])
    assert list(orc.canonical_order(modes, scores)) == [5, 1, 2, 0, 3, 4]


def test_hand_case_first_coordinate_decides_before_later_ones():
    # equal scores; the first coordinates differ, the later ones disagree
    modes = np.array([[2.0, -5.0, 0.0], [1.0, 9.0, 9.0], [1.0, 9.0, -1.0]])
    scores = np.ones(3)
    assert list(orc.canonical_order(modes, scores)) == [2, 1, 0]


def _brute_force_order(modes, scores):
    def before(i, j):
        if scores[i] != scores[j]:
            return -1 if scores[i] > scores[j] else 1
        for a, b in zip(modes[i], modes[j]):
            if a != b:
                return -1 if a < b else 1
        return -1 if i < j else (1 if i > j else 0)
    return sorted(range(len(scores)), key=functools.cmp_to_key(before))


@pytest.mark.parametrize("seed", range(6))
def test_random_cases_with_ties_match_a_pairwise_sort(seed):
    rng = np.random.default_rng(seed)
    M, d = 40, 3
    # few distinct values so that scores and coordinates tie often
    modes = rng.integers(0, 3, (M, d)).astype(np.float64)
    scores = rng.integers(0, 4, M).astype(np.float64)
    assert list(orc.canonical_order(modes, scores)) == _brute_force_order(modes, scores)


def test_order_check_flags_an_inverted_pair_and_allows_near_ties():
    scores = np.array([10.0, 5.0, 5.0000001, 1.0])
    # identity: no violations
    assert order_violations(np.array([0, 1, 2, 3]), scores) == 0
    # a near-tie (relative gap 2e-8) may come in either order
    assert order_violations(np.array([0, 2, 1, 3]), scores) == 0
    # a real inversion is counted (scores 10 and 5, and 10 and 1)
    assert order_violations(np.array([1, 0, 2, 3]), scores) == 1
    assert order_violations(np.array([3, 1, 2, 0]), scores) == 5
