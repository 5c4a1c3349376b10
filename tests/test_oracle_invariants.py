"""Pins of the FP64 oracle by invariants (no GPU).

* The density never decreases along a Gaussian mean-shift trajectory
  (convex, decreasing profile; the convergence proof the paper cites [b5]).
* Every returned mode is a fixed point of the update within tol.
* Results are equivariant under translation, uniform scaling (X*c, h*c,
  tol*c) and permutation of the points (with the same explicit seeds).
* Well-separated blobs give exactly the planted number of modes, each near
  its planted centre.
"""
import numpy as np
import pytest

import fms_inputs as fi
import oracle as orc


@pytest.mark.parametrize("seed", range(3))
def test_monotone_density_ascent(seed):
    rng = np.random.default_rng(seed)
    X = np.concatenate([rng.standard_normal((150, 2)) * 1.5,
                        rng.standard_normal((100, 2)) + 6.0,
                        rng.uniform(-4, 10, (50, 2))])
    h = 1.0
    Y = X[rng.choice(X.shape[0], 20, replace=False)].copy()
    f_prev = orc.kde(X, Y, h)
    for _ in range(40):
        Y = orc.step(X, Y, h)
        f = orc.kde(X, Y, h)
        assert np.all(f >= f_prev * (1 - 1e-14))
        f_prev = f


def test_modes_are_fixed_points():
    w = fi.plain_2d()
    res = orc.cluster(w.X, w.h, w.tol, w.max_iter, all_seeds=True)
    X = w.X.astype(np.float64)
    moved = np.linalg.norm(orc.step(X, res.modes, w.h) - res.modes, axis=1)
    assert np.all(moved <= 1e-5 * w.h)       # refined to 1e-5*h
    res2 = orc.cluster(w.X, w.h, w.tol, w.max_iter, all_seeds=True, refine=False)
    moved2 = np.linalg.norm(orc.step(X, res2.modes, w.h) - res2.modes, axis=1)
    assert np.all(moved2 <= w.tol * 1.0001)


def _small_problem():
    return fi.separated_blobs(seed=11, k=4, d=3, per=60, sigma=0.7, h=1.0)


def test_translation_and_scale_equivariance():
    w = _small_problem()
    seeds = np.arange(0, w.X.shape[0], 5, dtype=np.int64)
    base = orc.cluster(w.X, w.h, w.tol, w.max_iter, seed_indices=seeds)
    shift = np.array([123.5, -40.25, 7.0], dtype=np.float32)
    t = orc.cluster(w.X + shift, w.h, w.tol, w.max_iter, seed_indices=seeds)
    assert t.modes.shape == base.modes.shape
    assert np.max(np.abs(t.modes - shift - base.modes)) <= 1e-3 * w.h
    assert np.array_equal(t.labels, base.labels)
    c = 4.0   # a power of two keeps float32 inputs exact
    s = orc.cluster(w.X * np.float32(c), w.h * c, w.tol * c, w.max_iter, seed_indices=seeds)
    assert np.max(np.abs(s.modes / c - base.modes)) <= 1e-9 * w.h
    assert np.array_equal(s.labels, base.labels)


def test_permutation_equivariance():
    w = _small_problem()
    n = w.X.shape[0]
    seeds = np.arange(0, n, 7, dtype=np.int64)
    base = orc.cluster(w.X, w.h, w.tol, w.max_iter, seed_indices=seeds)
    p = np.random.default_rng(1).permutation(n)
    inv = np.argsort(p)
    perm = orc.cluster(w.X[p], w.h, w.tol, w.max_iter, seed_indices=inv[seeds])
    assert np.max(np.abs(perm.modes - base.modes)) <= 1e-9 * w.h
    assert np.array_equal(perm.labels[inv], base.labels)


@pytest.mark.parametrize("seed,k,d", [(1, 5, 2), (2, 8, 3), (3, 12, 4)])
def test_separated_blobs_give_planted_count(seed, k, d):
    w = fi.separated_blobs(seed=seed, k=k, d=d, per=200, sigma=1.0, h=1.5)
    res = orc.cluster(w.X, w.h, w.tol, w.max_iter, gamma=0.95, rng_seed=seed)
    assert res.modes.shape[0] == k
    for c in w.centers:
        assert np.min(np.linalg.norm(res.modes - c, axis=1)) <= 0.5
    # the labelling reproduces the planted partition up to renaming
    pairs = set(zip(w.planted.tolist(), res.labels.tolist()))
    assert len(pairs) == k


def test_plain_2d_planted_count():
    w = fi.plain_2d()
    res = orc.cluster(w.X, w.h, w.tol, w.max_iter, all_seeds=True)
    assert res.modes.shape[0] == 5


def test_frame_seed_count_rule():
    """Sec. II-D: N > H*M reduces the next frame's seed count by M."""
    assert orc.next_frame_seed_count(512, 12, 32.0) == 500     # 512 > 384
    assert orc.next_frame_seed_count(384, 12, 32.0) == 384     # not strictly larger
    assert orc.next_frame_seed_count(128, 2, 32.0) == 126
    assert orc.next_frame_seed_count(256, 20, 32.0) == 256


def test_frames_equal_single_calls_with_carried_counts():
    """Each frame's result is exactly cluster() started from the carried count."""
    import fms_inputs as fi
    frames = fi.drifting_frames(seed=3, frames=4, n=3000, k=3)
    res, starts = orc.cluster_frames(frames, 5.0, 5e-3, 300, n_initial=256, H=32.0)
    assert starts[0] == 256
    for f, X in enumerate(frames):
        one = orc.cluster(X, 5.0, 5e-3, 300, n_initial=starts[f])
        assert np.array_equal(one.modes, res[f].modes)
        assert np.array_equal(one.labels, res[f].labels)
        if f + 1 < len(frames):
            M = res[f].modes.shape[0]
            N = res[f].n_seeds
            assert starts[f + 1] == (N - M if N > 32.0 * M else N)
    # few modes, many seeds: the count shrinks from frame to frame
    assert starts[-1] < starts[0]
