"""GPU parity of the batched clustering (A8) through fms_cluster_batched.

Every set of a batch must match the FP64 oracle run on that set alone with the
same options (modes within 1e-3*h, labels equal away from ties, the seed count
history and the stop update equal), whatever the other sets in the batch are.
"""
import numpy as np
import pytest
import torch

import fms_inputs as fi
import oracle as orc
from fms_compare import compare_clustering

pytestmark = pytest.mark.gpu

fms = pytest.importorskip("paper_2112_13891_gb300")


def _mixed_sets(seed, B, d, lo, hi, h):
    rng = np.random.default_rng(seed)
    sets = []
    for b in range(B):
        n = int(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        k = int(rng.integers(3, 12))
        w = fi.separated_blobs(seed=seed * 1000 + b, k=k, d=d, per=max(n // k, 20), sigma=1.0, h=h)
        sets.append(w)
    return sets


def _check_set(w, modes, labels, margins_ok=True):
    ref = orc.cluster(w.X, w.h, w.tol, w.max_iter, gamma=0.95, rng_seed=0)
    cmp = compare_clustering(modes.cpu().numpy(), labels.cpu().numpy(), ref, w.h)
    assert cmp["mode_ok"], cmp
    assert cmp["label_mismatch"] == 0, cmp
    return ref


@pytest.mark.parametrize("d,h", [(3, 1.5), (16, 3.0)])
def test_batched_matches_oracle_per_set(d, h):
    sets = _mixed_sets(7 + d, 10, d, 300, 4000, h)
    X = [torch.from_numpy(w.X).cuda() for w in sets]
    res = fms.cluster_batched(X, h, 1e-3 * h, 300, gamma=0.95, rng_seed=0, max_modes=512)
    assert res.status == fms.FMS_OK
    torch.cuda.synchronize()
    off = np.concatenate([[0], np.cumsum([w.X.shape[0] for w in sets])])
    for b, w in enumerate(sets):
        _check_set(w, res.modes[b], res.labels[off[b]:off[b + 1]])


def test_batched_equals_single_set_calls():
    h = 1.5
    sets = _mixed_sets(3, 6, 3, 500, 3000, h)
    X = [torch.from_numpy(w.X).cuda() for w in sets]
    res = fms.cluster_batched(X, h, 1e-3 * h, 300, max_modes=64)
    off = np.concatenate([[0], np.cumsum([w.X.shape[0] for w in sets])])
    for b, w in enumerate(sets):
        one = fms.cluster(X[b], h, 1e-3 * h, 300)
        assert one.modes.shape == res.modes[b].shape
        assert torch.allclose(one.modes, res.modes[b], atol=1e-3 * h, rtol=0)
        lab_b = res.labels[off[b]:off[b + 1]]
        assert (one.labels == lab_b).float().mean().item() > 0.999


def test_batched_full_configuration_sampled():
    sets = fi.batched_16d()                       # 256 sets, 1K..50K points, d = 16
    X = [torch.from_numpy(w.X).cuda() for w in sets]
    res = fms.cluster_batched(X, 2.5, 2.5e-3, 300, gamma=0.95, rng_seed=0, max_modes=128)
    torch.cuda.synchronize()
    sizes = [w.X.shape[0] for w in sets]
    off = np.concatenate([[0], np.cumsum(sizes)])
    pick = {int(np.argmin(sizes)), int(np.argmax(sizes)), 17, 131}
    for b in sorted(pick):
        _check_set(sets[b], res.modes[b], res.labels[off[b]:off[b + 1]])
    assert res.stats["kernel_launches"] > 0
