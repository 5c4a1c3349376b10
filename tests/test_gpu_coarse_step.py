"""GPU parity of the coarse tensor-core update (fms_mean_shift_step_coarse) and
of clustering with the tensor-core step on (FMS_PRECISION_TENSOR).

The coarse update computes the same weighted mean as Eq. 6 with each weight
perturbed by a bounded relative error eps (BF16 rounding of the weight, 2^-9,
plus the error of the split-BF16 cross term, at most about 6 * 2^-18 * |u_y| *
|u_x| in the exponent of 2, u the scaled coordinates).  If every weight is
w_j (1 + delta_j) with |delta_j| <= eps then

    |m_hat - m| <= eps / (1 - eps) * sum_j w_j |x_j - m| / sum_j w_j,
    |W_hat - W| <= eps * W,

which is the bound the tests check, per seed, with eps computed from the
inputs and a factor 1.5 for the FP32 accumulation and the x hi/lo split
(relative 2^-17 of |x|).  Clustering with the coarse step must give the same
modes as the FP64 oracle within 1e-3*h and the same labels, as the FP32 path.
"""
import math

import numpy as np
import pytest
import torch

import fms_inputs as fi
import oracle as orc
from fms_compare import compare_clustering

pytestmark = pytest.mark.gpu

fms = pytest.importorskip("paper_2112_13891_gb300")

LOG2E = 1.4426950408889634


def _cloud(rng, n, d, box=30.0, k=5, sigma=2.0):
    c = rng.uniform(0, box, (k, d))
    lab = rng.integers(0, k, n)
    return (c[lab] + rng.standard_normal((n, d)) * sigma).astype(np.float32)


def _bound(X, Y, h, ref):
    """Per-seed bounds on |m_hat - m| (max over coordinates) and |W_hat/W - 1|."""
    s = math.sqrt(LOG2E / (2.0 * h * h))
    Xd = X.astype(np.float64)
    Yd = Y.astype(np.float64)
    ux = np.linalg.norm(Xd, axis=1).max() * s
    uy = np.linalg.norm(Yd, axis=1) * s
    eps = 2.0 ** -9 + math.log(2.0) * (6 * 2.0 ** -18 * uy * ux + 2.0 ** -20 * (uy ** 2 + ux ** 2))
    eps = eps + 2.0 ** -20
    d2 = ((Yd[:, None, :] - Xd[None, :, :]) ** 2).sum(-1)
    w = np.exp(-d2 / (2.0 * h * h))
    W = w.sum(1)
    spread = (w * np.linalg.norm(Xd[None, :, :] - ref[:, None, :], axis=-1)).sum(1) / W
    return 1.5 * eps / (1.0 - eps) * spread + 2.0 ** -17 * np.abs(Xd).max(), eps


@pytest.mark.parametrize("d", [1, 3, 8, 9, 16, 17, 24, 32])
@pytest.mark.parametrize("n,m", [(1, 1), (127, 5), (1000, 129), (4097, 300)])
def test_coarse_step_within_bf16_bound(d, n, m):
    rng = np.random.default_rng(31 * d + n + m)
    X = _cloud(rng, n, d)
    h = 3.0
    Y = (X[rng.integers(0, n, m)] + rng.standard_normal((m, d)).astype(np.float32)).astype(np.float32)
    out, W = fms.mean_shift_step_coarse(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), h,
                                        with_wsum=True)
    out = out.cpu().numpy().astype(np.float64)
    W = W.cpu().numpy().astype(np.float64)
    ref = orc.step(X, Y, h)
    refW = orc.kde(X, Y, h)
    bnd, eps = _bound(X, Y, h, ref)
    err = np.abs(out - ref).max(axis=1)
    assert np.all(err <= bnd), (err.max(), bnd[np.argmax(err - bnd)])
    assert np.all(np.abs(W - refW) <= 1.5 * eps * refW), np.abs(W / refW - 1).max()


def test_coarse_step_far_from_origin():
    """Large coordinates: the cancellation in |u_y|^2 + |u_x|^2 - 2 u_y.u_x."""
    rng = np.random.default_rng(77)
    d = 32
    X = _cloud(rng, 3000, d, box=6.0) + 40.0
    h = 2.0
    Y = X[rng.integers(0, 3000, 200)] + 0.5 * rng.standard_normal((200, d)).astype(np.float32)
    Y = Y.astype(np.float32)
    out = fms.mean_shift_step_coarse(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), h)
    out = out.cpu().numpy().astype(np.float64)
    ref = orc.step(X, Y, h)
    bnd, _ = _bound(X, Y, h, ref)
    err = np.abs(out - ref).max(axis=1)
    assert np.all(err <= bnd), (err.max(), bnd.min())


def test_coarse_step_rejects_wide_dimension():
    X = torch.zeros((10, 33), device="cuda")
    with pytest.raises(fms.FmsError):
        fms.mean_shift_step_coarse(X, X[:2], 1.0)


def _cluster_check(w, precision, **kw):
    X = torch.from_numpy(w.X).cuda()
    res = fms.cluster(X, w.h, w.tol, w.max_iter, precision=precision, profile=True, **kw)
    torch.cuda.synchronize()
    ref = orc.cluster(w.X, w.h, w.tol, w.max_iter, **kw)
    cmp = compare_clustering(res.modes.cpu().numpy(), res.labels.cpu().numpy(), ref, w.h)
    print(w.name, precision, cmp, res.stats)
    assert cmp["mode_ok"], cmp
    assert cmp["label_mismatch"] == 0, cmp
    return res, ref


@pytest.mark.parametrize("precision", ["fp32", "tensor"])
def test_embedding_32d_both_precisions(precision):
    w = fi.embedding_32d()
    res, ref = _cluster_check(w, precision, gamma=0.95, rng_seed=0)
    if precision == "tensor":
        assert res.stats["coarse_launches"] > 0 and res.stats["coarse_evals"] > 0
    else:
        assert res.stats["coarse_launches"] == 0


@pytest.mark.parametrize("k,d,sigma", [(9, 8, 1.0), (9, 16, 1.0), (7, 24, 1.0), (5, 32, 0.5)])
def test_separated_blobs_tensor(k, d, sigma):
    # sigma * sqrt(d) <= ~5 h: wider blobs at d = 32 leave every point its own mode
    w = fi.separated_blobs(seed=k + d + 100, k=k, d=d, per=400, sigma=sigma, h=1.5)
    res, ref = _cluster_check(w, "tensor", gamma=0.95, rng_seed=3)
    assert res.stats["n_modes"] == ref.modes.shape[0]
    assert res.stats["coarse_launches"] > 0


def test_tensor_all_seeds_d16():
    w = fi.separated_blobs(seed=5, k=6, d=16, per=500, sigma=1.0, h=1.5)
    res, ref = _cluster_check(w, "tensor", all_seeds=True)
    assert res.stats["n_modes"] == ref.modes.shape[0]


def test_tensor_ragged_sizes():
    """n not a multiple of the 128-point tile, tiny sets, single point."""
    for n_per, k in ((1, 1), (3, 2), (129, 3), (333, 4)):
        w = fi.separated_blobs(seed=n_per, k=k, d=20, per=n_per, sigma=0.7, h=1.5)
        _cluster_check(w, "tensor", gamma=0.95, rng_seed=1)


def test_precision_option_validated():
    X = torch.zeros((10, 16), device="cuda")
    with pytest.raises(fms.FmsError):
        fms.cluster(X, 1.0, precision=3)
