"""GPU parity of the cosine-metric variant (metric="cosine") with the FP64 oracle.

The points are normalised on the device, every update is projected back onto
the sphere (cluster rounds for d <= 7, the global step and update kernels for
larger d, and both refinements), and labels compare the points' directions
with the unit modes.  Acceptance is the cluster parity bar: modes within
1e-3*h (chord distance) matched one-to-one with the oracle's, identical labels.
"""
import numpy as np
import pytest
import torch

import fms_inputs as fi
import oracle as orc
from fms_compare import compare_clustering

pytestmark = pytest.mark.gpu

fms = pytest.importorskip("paper_2112_13891_gb300")


def _check(w, **kw):
    X = torch.from_numpy(w.X).cuda()
    res = fms.cluster(X, w.h, w.tol, w.max_iter, metric="cosine", **kw)
    torch.cuda.synchronize()
    ref = orc.cluster(w.X, w.h, w.tol, w.max_iter, metric="cosine", **kw)
    cmp = compare_clustering(res.modes.cpu().numpy(), res.labels.cpu().numpy(), ref, w.h)
    print(w.name, cmp, res.stats)
    assert cmp["mode_ok"], cmp
    assert cmp["label_mismatch"] == 0, cmp
    m = res.modes.cpu().numpy().astype(np.float64)
    assert np.allclose(np.linalg.norm(m, axis=1), 1.0, atol=1e-5)
    return res, ref


@pytest.mark.parametrize("d,k", [(3, 6), (5, 8), (7, 8), (16, 12), (32, 16)])
def test_cosine_parity(d, k):
    w = fi.directional_blobs(seed=d * 10 + k, k=k, d=d, per=300, spread=0.05, h=0.15)
    res, ref = _check(w, gamma=0.95, rng_seed=1)
    assert res.stats["n_modes"] == k


def test_cosine_flat_kernel():
    w = fi.directional_blobs(seed=77, k=5, d=3, per=400, spread=0.04, h=0.2)
    _check(w, gamma=0.95, rng_seed=2, kernel="flat")


def test_cosine_ignores_the_points_norms():
    w = fi.directional_blobs(seed=5, k=6, d=4, per=300, spread=0.05, h=0.15)
    X = torch.from_numpy(w.X).cuda()
    a = fms.cluster(X, w.h, w.tol, w.max_iter, metric="cosine", rng_seed=3)
    b = fms.cluster(X * 7.5, w.h, w.tol, w.max_iter, metric="cosine", rng_seed=3)
    assert torch.equal(a.labels, b.labels)
    assert torch.allclose(a.modes, b.modes, atol=1e-5)


def test_cosine_graph_form_matches_host_path():
    w = fi.directional_blobs(seed=9, k=6, d=3, per=400, spread=0.05, h=0.15)
    X = torch.from_numpy(w.X).cuda()
    n, d = X.shape
    ws = fms.Workspace(fms.workspace_size(n, d, metric="cosine"), X.device)
    modes = torch.empty((n, d), device="cuda")
    labels = torch.empty(n, dtype=torch.int32, device="cuda")
    margins = torch.empty(n, device="cuda")
    outs = []
    for _ in range(3):
        r = fms.cluster(X, w.h, w.tol, w.max_iter, metric="cosine", rng_seed=4, workspace=ws,
                        out=(modes, labels, margins))
        torch.cuda.synchronize()
        outs.append((r.modes.clone(), labels.clone(), margins.clone(), r.stats["graph"]))
    assert [o[3] for o in outs] == [0, 1, 1]
    for o in outs[1:]:
        assert torch.equal(o[0], outs[0][0]) and torch.equal(o[1], outs[0][1])
        assert torch.equal(o[2], outs[0][2])


def test_cosine_rejects_zero_points_and_batched():
    X = torch.ones((100, 3), device="cuda")
    X[7] = 0.0
    with pytest.raises(fms.FmsError):
        fms.cluster(X, 0.2, metric="cosine")
    Y = torch.randn((200, 3), device="cuda")
    with pytest.raises(fms.FmsError):
        fms.cluster_batched([Y, Y], 0.2, metric="cosine")


@pytest.mark.parametrize("d,k,spread,h,ang", [(3, 20, 0.04, 0.12, 0.5), (16, 32, 0.04, 0.25, 0.9)])
def test_cosine_at_the_200k_size(d, k, spread, h, ang):
    # the configurations the cosine line of bench.py times: every label and
    # mode against the oracle at full size
    w = fi.directional_blobs(seed=100 + d, k=k, d=d, per=200_000 // k, spread=spread, h=h,
                             min_angle=ang)
    res, ref = _check(w)
    assert res.stats["n_modes"] == k
