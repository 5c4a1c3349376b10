"""Pins of the FP64 oracle by brute force on tiny inputs (no GPU).

* Local maxima of the Gaussian density for n <= 8 points in 1-D and 2-D are
  found by a dense grid scan plus Newton polishing, written here in plain
  Python with an analytic gradient and Hessian; every oracle mode must be one
  of them.
* Nearest-mode labels are checked against an exhaustive Python argmin.
* The density sum is checked against a Python loop.
"""
import itertools
import math

import numpy as np
import pytest

import oracle as orc


def _f_grad_hess(X, y, h):
    d = len(y)
    f = 0.0
    g = [0.0] * d
    H = [[0.0] * d for _ in range(d)]
    for x in X:
        u = [x[k] - y[k] for k in range(d)]
        w = math.exp(-sum(t * t for t in u) / (2 * h * h))
        f += w
        for a in range(d):
            g[a] += w * u[a] / (h * h)
            for b in range(d):
                H[a][b] += w * (u[a] * u[b] / h ** 4 - (1.0 if a == b else 0.0) / (h * h))
    return f, np.array(g), np.array(H)


def _brute_force_maxima(X, h, grid=161):
    X = [list(map(float, x)) for x in X]
    d = len(X[0])
    lo = [min(x[k] for x in X) - 2 * h for k in range(d)]
    hi = [max(x[k] for x in X) + 2 * h for k in range(d)]
    axes = [np.linspace(lo[k], hi[k], grid if d == 1 else 81) for k in range(d)]
    pts = list(itertools.product(*axes))
    vals = {p: _f_grad_hess(X, p, h)[0] for p in pts}
    shape = [len(a) for a in axes]
    idx = list(itertools.product(*[range(s) for s in shape]))
    cands = []
    for ii in idx:
        p = tuple(axes[k][ii[k]] for k in range(d))
        v = vals[p]
        is_max = True
        for off in itertools.product(*([(-1, 0, 1)] * d)):
            if all(o == 0 for o in off):
                continue
            jj = [ii[k] + off[k] for k in range(d)]
            if any(j < 0 or j >= shape[k] for k, j in enumerate(jj)):
                continue
            q = tuple(axes[k][jj[k]] for k in range(d))
            if vals[q] > v:
                is_max = False
                break
        if is_max:
            cands.append(np.array(p))
    maxima = []
    for y in cands:
        for _ in range(100):
            f, g, H = _f_grad_hess(X, y, h)
            step = np.linalg.solve(H, -g)
            y = y + step
            if np.max(np.abs(step)) < 1e-14 * (1 + np.max(np.abs(y))):
                break
        f, g, H = _f_grad_hess(X, y, h)
        if np.all(np.linalg.eigvalsh(H) < 0) and np.max(np.abs(g)) < 1e-9:
            if not any(np.max(np.abs(y - m)) < 1e-7 * h for m in maxima):
                maxima.append(y)
    return maxima


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("d", [1, 2])
def test_oracle_modes_are_brute_force_maxima(seed, d):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(3, 9))
    X = rng.uniform(0.0, 6.0, size=(n, d))
    h = float(rng.uniform(0.4, 1.2))
    maxima = _brute_force_maxima(X, h)
    assert len(maxima) >= 1
    # every trajectory ends at a brute-force maximum
    Y, conv, _ = orc.trajectories(X, X, h, 1e-13 * h, 200000)
    for y in Y:
        dist = min(np.max(np.abs(y - m)) for m in maxima)
        assert dist <= 1e-6 * h
    # and so does every refined mode of the full clustering
    res = orc.cluster(X.astype(np.float32), h, 1e-6 * h, 10000, all_seeds=True,
                      merge_radius=1e-3 * h, refine_tol=1e-12, refine_max_iter=100000)
    X32 = X.astype(np.float32).astype(np.float64)
    maxima32 = _brute_force_maxima(X32, h)
    for m in res.modes:
        dist = min(np.max(np.abs(m - q)) for q in maxima32)
        assert dist <= 1e-6 * h


@pytest.mark.parametrize("seed", range(4))
def test_labels_exhaustive(seed):
    rng = np.random.default_rng(seed)
    n, d, M = 300, 3, 7
    X = rng.standard_normal((n, d))
    modes = rng.standard_normal((M, d))
    modes[3] = modes[1]            # an exact tie: the lower index must win
    X[:5] = modes[1]               # points sitting on the tied modes
    lab, mar = orc.label(X, modes)
    for j in range(n):
        ds = [math.sqrt(sum((X[j][k] - modes[m][k]) ** 2 for k in range(d))) for m in range(M)]
        best = min(range(M), key=lambda m: (ds[m], m))
        assert lab[j] == best
        rest = sorted(ds)
        assert abs(mar[j] - (rest[1] - rest[0])) <= 1e-12


def test_label_single_mode_margin_is_inf():
    X = np.arange(12.0).reshape(6, 2)
    lab, mar = orc.label(X, X[:1])
    assert np.all(lab == 0) and np.all(np.isinf(mar))


def test_kde_matches_python_loop():
    rng = np.random.default_rng(5)
    X = rng.standard_normal((50, 4))
    Y = rng.standard_normal((6, 4))
    h = 0.9
    got = orc.kde(X, Y, h)
    for i in range(6):
        s = 0.0
        for j in range(50):
            s += math.exp(-sum((Y[i][k] - X[j][k]) ** 2 for k in range(4)) / (2 * h * h))
        assert abs(got[i] - s) <= 1e-13 * s


def test_merge_hand_case():
    """Greedy prune: highest score first, suppress within r, ties by rank."""
    # three points close together (one cluster) and one far away
    X = np.array([[0.0, 0.0], [0.1, 0.0], [0.0, 0.1], [10.0, 10.0]])
    Y = np.array([[0.05, 0.05], [0.04, 0.05], [10.0, 10.0], [0.05, 0.04]])
    acc, score = orc.merge(X, Y, np.arange(4), 1.0, 1.0)
    assert len(acc) == 2
    assert int(np.argmax(score[:2])) in (0, 1)
    # the accepted representative of the tight cluster is its best-scoring row
    tight = [0, 1, 3]
    best = max(tight, key=lambda i: (score[i], -i))
    assert best in acc and 2 in acc
    # equal scores: the lower rank wins
    Y2 = np.array([[5.0, 5.0], [5.0, 5.0]])
    acc2, _ = orc.merge(X, Y2, np.array([7, 3]), 1.0, 1.0)
    assert list(acc2) == [1]
