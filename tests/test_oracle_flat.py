"""Pins of the oracle's flat-kernel variant (Eq. 12-15).

* closed forms: two points closer than h move to their midpoint in one update;
  two points farther apart than h stay put; a window count is exact;
* the whole flat mean-shift clustering against scikit-learn's MeanShift (a
  flat-kernel implementation: each seed iterates the mean of the points within
  the bandwidth until the move is at most 1e-3 * bandwidth, duplicates within
  the bandwidth are removed in order of window count), on the same seeds.
"""
import numpy as np
import pytest
from scipy.optimize import linear_sum_assignment

import oracle as orc


def test_flat_two_points():
    h = 1.0
    X = np.array([[0.0], [0.8]])
    out = orc.step(X, X, h, kernel="flat")
    assert np.allclose(out, 0.4)
    X2 = np.array([[0.0], [1.2]])
    assert np.allclose(orc.step(X2, X2, h, kernel="flat"), X2)
    # inclusive boundary: distance exactly h is inside the window
    X3 = np.array([[0.0], [1.0]])
    assert np.allclose(orc.step(X3, X3[:1], h, kernel="flat"), 0.5)


def test_flat_density_is_window_count():
    rng = np.random.default_rng(3)
    X = rng.uniform(-3, 3, (500, 2))
    Y = rng.uniform(-3, 3, (40, 2))
    cnt = orc.kde(X, Y, 1.3, kernel="flat")
    want = [(np.sqrt(((X - y) ** 2).sum(1)) <= 1.3).sum() for y in Y]
    assert np.array_equal(cnt, want)


def test_flat_empty_window_fails_seed():
    X = np.array([[0.0, 0.0], [10.0, 0.0]])
    Y, conv, _ = orc.trajectories(X, np.array([[5.0, 0.0]]), 1.0, 1e-3, 10, kernel="flat")
    assert conv[0] == -2


@pytest.mark.parametrize("seed", [0, 1])
def test_flat_cluster_matches_sklearn(seed):
    sk = pytest.importorskip("sklearn.cluster")
    rng = np.random.default_rng(seed)
    centers = rng.uniform(0, 40, (5, 2))
    X = np.concatenate([c + rng.standard_normal((120, 2)) * 1.2 for c in centers])
    X = X.astype(np.float32)
    h = 3.0
    ms = sk.MeanShift(bandwidth=h, seeds=X.astype(np.float64), bin_seeding=False,
                      cluster_all=True, max_iter=300).fit(X.astype(np.float64))
    ref = orc.cluster(X, h, 1e-3 * h, 300, all_seeds=True, refine=False, kernel="flat")
    A, B = np.asarray(ms.cluster_centers_), ref.modes
    assert A.shape == B.shape, (A.shape, B.shape)
    D = np.sqrt(((A[:, None] - B[None]) ** 2).sum(-1))
    r, c = linear_sum_assignment(D)
    assert D[r, c].max() < 1e-9 * h
    perm = np.empty(len(c), dtype=np.int64)
    perm[r] = c
    assert np.array_equal(perm[ms.labels_], ref.labels)
