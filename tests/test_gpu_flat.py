"""N2: the flat (uniform) kernel of Eq. 12-15 through fms_cluster, against the
FP64 oracle's flat variant (itself pinned to scikit-learn's MeanShift).

The flat update is discontinuous in the points that sit on a window boundary,
so FP32 and FP64 can take different windows for a point within rounding of
||x - y|| = h.  The inputs keep every window away from such points: blobs whose
radius is well inside h and whose centres are far apart, so each window is a
whole blob and the fixed point is the blob mean.  With those inputs modes,
labels and the Early-Stopping bookkeeping must match the oracle exactly as for
the Gaussian kernel.
"""
import numpy as np
import pytest
import torch

import fms_inputs as fi
import oracle as orc
from fms_compare import compare_clustering

pytestmark = pytest.mark.gpu

fms = pytest.importorskip("paper_2112_13891_gb300")


def _blobs(seed, k, d, per, sigma, h):
    rng = np.random.default_rng(seed)
    centers = []
    while len(centers) < k:
        c = rng.uniform(0, 30 * h, d)
        if all(np.linalg.norm(c - e) > 4 * h for e in centers):
            centers.append(c)
    # points within 0.35 h of their centre (truncated normal), so a window of
    # radius h around any point of a blob holds the whole blob and nothing else
    X = []
    for c in centers:
        z = rng.standard_normal((per * 3, d)) * sigma
        z = z[np.linalg.norm(z, axis=1) < 0.35 * h][:per]
        X.append(c + z)
    return np.concatenate(X).astype(np.float32)


@pytest.mark.parametrize("d,k", [(2, 6), (3, 8), (5, 5), (16, 7)])
def test_flat_faster_matches_oracle(d, k):
    h = 2.0
    X = _blobs(10 + d, k, d, 400, 0.3, h)
    tol = 1e-3 * h
    res = fms.cluster(torch.from_numpy(X).cuda(), h, tol, 300, kernel="flat", gamma=0.95,
                      rng_seed=1)
    ref = orc.cluster(X, h, tol, 300, kernel="flat", gamma=0.95, rng_seed=1)
    cmp = compare_clustering(res.modes.cpu().numpy(), res.labels.cpu().numpy(), ref, h)
    assert cmp["mode_ok"] and cmp["label_mismatch"] == 0, cmp
    assert res.stats["n_modes"] == k
    assert res.stats["rounds"] == len(ref.n_history)
    assert res.stats["t_star_last"] == ref.t_star[-1]
    assert res.stats["n_kept"] == int(ref.kept.sum())
    assert res.stats["coarse_launches"] == 0


def test_flat_all_seeds_matches_oracle():
    h = 2.0
    X = _blobs(5, 6, 3, 300, 0.3, h)
    res = fms.cluster(torch.from_numpy(X).cuda(), h, 1e-3 * h, 300, kernel="flat",
                      all_seeds=True)
    ref = orc.cluster(X, h, 1e-3 * h, 300, kernel="flat", all_seeds=True)
    cmp = compare_clustering(res.modes.cpu().numpy(), res.labels.cpu().numpy(), ref, h)
    assert cmp["mode_ok"] and cmp["label_mismatch"] == 0, cmp


def test_flat_modes_are_window_means():
    """The flat fixed point is exactly the mean of its window (here: its blob)."""
    h = 2.0
    X = _blobs(7, 4, 2, 500, 0.3, h)
    res = fms.cluster(torch.from_numpy(X).cuda(), h, 1e-3 * h, 300, kernel="flat")
    modes = res.modes.cpu().numpy().astype(np.float64)
    lab = res.labels.cpu().numpy()
    for k in range(modes.shape[0]):
        want = X[lab == k].astype(np.float64).mean(axis=0)
        assert np.abs(modes[k] - want).max() <= 1e-5 * h


def test_flat_rejected_by_batched_and_validated():
    X = torch.zeros((64, 3), device="cuda")
    with pytest.raises(fms.FmsError):
        fms.cluster_batched([X, X], 1.0, kernel="flat")
    with pytest.raises(fms.FmsError):
        fms.cluster(X, 1.0, kernel=2)
