"""Pins of Seed Selection, Eq. 12 and Early Stopping in the oracle (no GPU).

* SplitMix64 outputs match published reference values (tests/golden).
* The keyed Feistel permutation is a bijection of [0, n) (brute force).
* Eq. 12 (Sec. II-C) equals the fraction of compositions with no empty
  cluster (enumerated), and the uniform-draw coverage probability matches
  Monte Carlo; the two differ (N = M = 2: 1/3 vs 1/2).
* Early Stopping picks the ceil(gamma*N)-th convergence iteration.
"""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import fms_inputs as fi
import oracle as orc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_reference_values():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt"))
            if l.strip() and not l.startswith("#")]
    for i, v in rows:
        assert orc.splitmix64(0, int(i)) == int(v, 16)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 16, 17, 63, 64, 65, 1000, 4097])
@pytest.mark.parametrize("key", [0, 1, 0xDEADBEEFCAFEF00D])
def test_feistel_permutation_is_bijection(n, key):
    p = orc.seed_permutation(n, key, 0, n)
    assert sorted(p.tolist()) == list(range(n))


def test_feistel_prefix_is_prefix():
    n = 5000
    full = orc.seed_permutation(n, 42, 0, 600)
    assert np.array_equal(full[:128], orc.seed_permutation(n, 42, 0, 128))
    assert np.array_equal(full[128:256], orc.seed_permutation(n, 42, 128, 256))


def test_feistel_first_entry_roughly_uniform():
    n, keys = 10, 4000
    counts = np.bincount([orc.seed_permutation(n, k, 0, 1)[0] for k in range(keys)], minlength=n)
    exp = keys / n
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    assert chi2 < 30.0      # 9 dof: p ~ 4e-4


def _compositions(N, M):
    for cut in itertools.combinations(range(N + M - 1), M - 1):
        prev, parts = -1, []
        for c in cut + (N + M - 1,):
            parts.append(c - prev - 1)
            prev = c
        yield parts


@pytest.mark.parametrize("N,M", [(2, 2), (3, 2), (5, 3), (7, 4), (9, 3), (10, 5)])
def test_eq12_equals_fraction_of_nonempty_compositions(N, M):
    comps = list(_compositions(N, M))
    assert len(comps) == math.comb(N + M - 1, M - 1)
    good = sum(1 for c in comps if min(c) >= 1)
    assert abs(orc.eq12_coverage(N, M) - good / len(comps)) <= 1e-15
    # the factorial form printed beside Eq. 12
    fact = Fraction(math.factorial(N - 1) * math.factorial(N),
                    math.factorial(N - M) * math.factorial(N + M - 1))
    assert abs(orc.eq12_coverage(N, M) - float(fact)) <= 1e-15


@pytest.mark.parametrize("N,M", [(2, 2), (6, 3), (20, 5), (40, 10)])
def test_uniform_draw_coverage_monte_carlo(N, M):
    rng = np.random.default_rng(N * 100 + M)
    trials = 20000
    draws = rng.integers(0, M, size=(trials, N))
    hit = np.array([len(np.unique(r)) == M for r in draws])
    p = orc.coverage_uniform_draws(N, M)
    assert abs(hit.mean() - p) <= 4 * math.sqrt(p * (1 - p) / trials) + 1e-12


def test_eq12_is_not_the_uniform_draw_probability():
    assert abs(orc.eq12_coverage(2, 2) - 1 / 3) < 1e-15
    assert abs(orc.coverage_uniform_draws(2, 2) - 1 / 2) < 1e-15


def test_early_stop_rule():
    conv = np.array([3, 1, -1, 2, 5, 2, 4, -1, 6, 2], dtype=np.int32)
    # gamma 0.5 -> 5th smallest of {1,2,2,2,3,4,5,6,inf,inf} = 3
    t, kept = orc.early_stop(conv, 0.5, 100)
    assert t == 3 and kept.tolist() == [c != -1 and c <= 3 for c in conv.tolist()]
    # gamma 0.9 -> 9th smallest is inf -> max_iter; all converged kept
    t, kept = orc.early_stop(conv, 0.9, 50)
    assert t == 50 and kept.sum() == 8
    # gamma 1 keeps every seed
    t, kept = orc.early_stop(conv, 1.0, 50)
    assert t == 50 and kept.all()
    t, kept = orc.early_stop(np.array([1, 4, 2], np.int32), 1.0, 50)
    assert t == 4 and kept.all()


def test_doubling_rule_reaches_L_times_M():
    w = fi.separated_blobs(seed=4, k=30, d=2, per=150, sigma=0.5, h=0.8)
    res = orc.cluster(w.X, w.h, w.tol, w.max_iter, gamma=0.95, n_initial=16, L=8.0, rng_seed=9)
    M = res.modes.shape[0]
    assert res.n_history[0] == 16
    assert all(b == min(2 * a, w.X.shape[0]) for a, b in zip(res.n_history, res.n_history[1:]))
    assert res.n_seeds >= 8 * M or res.n_seeds == w.X.shape[0]
    # the seeds are the permutation prefix of the final N
    assert np.array_equal(res.seeds, orc.seed_permutation(w.X.shape[0], 9, 0, res.n_seeds))
