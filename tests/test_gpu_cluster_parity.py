"""GPU parity of the full clustering (fms_cluster through the C ABI).

Acceptance (the project's stated bar): modes matched one-to-one with the FP64
oracle within 1e-3*h; labels identical after mapping GPU mode indices to the
oracle's, except points whose oracle margin is below 1e-2*h (their count is
reported).  The Early-Stopping bookkeeping (N history, stop update, kept
count) must match the oracle exactly on these inputs.
"""
import numpy as np
import pytest
import torch

import fms_inputs as fi
import oracle as orc
from fms_compare import compare_clustering

pytestmark = pytest.mark.gpu

fms = pytest.importorskip("paper_2112_13891_gb300")


def _run(w, **kw):
    X = torch.from_numpy(w.X).cuda()
    res = fms.cluster(X, w.h, w.tol, w.max_iter, **kw)
    torch.cuda.synchronize()
    return res


def _check(w, res, ref, report=None):
    cmp = compare_clustering(res.modes.cpu().numpy(), res.labels.cpu().numpy(), ref, w.h)
    if report is not None:
        report.update(cmp)
    print(w.name, cmp, res.stats)
    assert cmp["mode_ok"], cmp
    assert cmp["label_mismatch"] == 0, cmp
    return cmp


def test_plain_2d_all_seeds():
    w = fi.plain_2d()
    res = _run(w, all_seeds=True)
    ref = orc.cluster(w.X, w.h, w.tol, w.max_iter, all_seeds=True)
    _check(w, res, ref)
    assert res.stats["n_modes"] == 5


@pytest.mark.parametrize("n", [20_011, 200_000])
def test_paper_3d_faster(n):
    w = fi.paper_3d(n=n)
    res = _run(w, gamma=0.95, rng_seed=0)
    ref = orc.cluster(w.X, w.h, w.tol, w.max_iter, gamma=0.95, rng_seed=0)
    _check(w, res, ref)
    assert res.stats["n_seeds_final"] == ref.n_seeds
    assert res.stats["rounds"] == len(ref.n_history)
    assert res.stats["t_star_last"] == ref.t_star[-1]
    assert res.stats["n_kept"] == int(ref.kept.sum())


def test_paper_3d_all_seeds_small():
    w = fi.paper_3d(n=6000)
    res = _run(w, all_seeds=True)
    ref = orc.cluster(w.X, w.h, w.tol, w.max_iter, all_seeds=True)
    _check(w, res, ref)


def test_paper_3d_all_seeds_30k():
    # 30,000 seeds: more candidates than the sorted prune's keys can hold in
    # shared memory, so the one-block global greedy runs; checked whole
    # against the oracle
    w = fi.paper_3d(n=30_000)
    res = _run(w, all_seeds=True)
    ref = orc.cluster(w.X, w.h, w.tol, w.max_iter, all_seeds=True)
    _check(w, res, ref)
    assert res.stats["n_kept"] == 30_000


def test_paper_3d_all_seeds_full_size_sampled():
    # Alg. 1 at the 200K size the all-seeds bench line runs: every point is a
    # seed, too many for the oracle to cluster whole.  Trajectories are
    # independent, so sampled seeds' FP64 trajectories are exact references:
    # each one's end point was a prune candidate, so a first-prune mode lies
    # within r_merge = h of it and moves by a few tol in the refinement; the
    # second prune can drop that mode for one within h of it (rare), hence the
    # 2h bound for every sample.  The sampled points' labels are the FP64
    # nearest modes away from ties.
    w = fi.paper_3d()
    res = _run(w, all_seeds=True)
    modes = res.modes.cpu().numpy().astype(np.float64)
    labels = res.labels.cpu().numpy()
    assert res.stats["n_seeds_final"] == w.X.shape[0]
    rng = np.random.default_rng(11)
    sample = rng.choice(w.X.shape[0], 48, replace=False)
    y_end, conv, _ = orc.trajectories(w.X, w.X[sample], w.h, w.tol, w.max_iter)
    assert np.all(conv > 0)
    dist = np.linalg.norm(y_end[:, None, :] - modes[None, :, :], axis=2).min(axis=1)
    assert np.mean(dist < 1.01 * w.h) >= 0.95, np.sort(dist)[-4:]
    assert np.all(dist < 2.02 * w.h), dist.max()
    lab, marg = orc.label(w.X[sample], modes)
    clear = marg > 1e-2 * w.h
    assert np.array_equal(lab[clear], labels[sample][clear])


@pytest.mark.parametrize("k,d", [(6, 2), (10, 5), (12, 8), (9, 16)])
def test_separated_blobs(k, d):
    w = fi.separated_blobs(seed=k + d, k=k, d=d, per=300, sigma=1.0, h=1.5)
    res = _run(w, gamma=0.95, rng_seed=3)
    ref = orc.cluster(w.X, w.h, w.tol, w.max_iter, gamma=0.95, rng_seed=3)
    _check(w, res, ref)
    assert res.stats["n_modes"] == k


@pytest.mark.parametrize("d", [1, 4, 6, 7])
def test_every_low_dimension(d):
    # the cluster rounds, the prune's register visit and the labels are
    # compiled per dimension for d <= 8; the other values run elsewhere
    w = fi.separated_blobs(seed=40 + d, k=5, d=d, per=300, sigma=0.8, h=1.2)
    res = _run(w, gamma=0.95, rng_seed=6)
    ref = orc.cluster(w.X, w.h, w.tol, w.max_iter, gamma=0.95, rng_seed=6)
    _check(w, res, ref)
    assert res.stats["n_modes"] == 5
    assert res.stats["t_star_last"] == ref.t_star[-1]


@pytest.mark.parametrize("k,d", [(300, 2), (200, 3)])
def test_many_modes(k, d):
    # hundreds of modes: the first prunes accept most candidates (the one-warp
    # visit with a long accepted list), later rounds exceed 512 candidates
    # (the block-wide visit); the seed count doubles several times
    w = fi.separated_blobs(seed=k + d, k=k, d=d, per=15, sigma=0.3, h=1.0)
    res = _run(w, gamma=0.95, rng_seed=5)
    ref = orc.cluster(w.X, w.h, w.tol, w.max_iter, gamma=0.95, rng_seed=5)
    _check(w, res, ref)
    assert res.stats["n_modes"] == k
    assert res.stats["n_seeds_final"] == ref.n_seeds
    assert res.stats["rounds"] == len(ref.n_history)


def test_embedding_32d_faster():
    w = fi.embedding_32d()
    res = _run(w, gamma=0.95, rng_seed=0)
    ref = orc.cluster(w.X, w.h, w.tol, w.max_iter, gamma=0.95, rng_seed=0)
    _check(w, res, ref)


def test_toy_distributions():
    for make in (fi.toy_blobs, fi.toy_large_variance, fi.toy_varied_variance,
                 fi.toy_uniform_square, fi.toy_anisotropic):
        w = make()
        Xd = w.X.astype(np.float64)
        h = float(np.median(np.linalg.norm(Xd[:300, None] - Xd[None, :300], axis=-1))) * 0.3
        w = fi.Workload(dict(w, h=h, tol=1e-3 * h, max_iter=300))
        res = _run(w, all_seeds=True)
        ref = orc.cluster(w.X, w.h, w.tol, w.max_iter, all_seeds=True)
        _check(w, res, ref)


def test_explicit_seeds_and_no_refine():
    w = fi.separated_blobs(seed=21, k=5, d=3, per=200, sigma=0.8, h=1.2)
    seeds = np.arange(0, w.X.shape[0], 9, dtype=np.int64)
    res = _run(w, seed_indices=torch.from_numpy(seeds.astype(np.int32)), skip_refine=True)
    ref = orc.cluster(w.X, w.h, w.tol, w.max_iter, seed_indices=seeds, refine=False)
    _check(w, res, ref)


def test_deterministic():
    w = fi.paper_3d(n=30_000)
    a = _run(w)
    b = _run(w)
    assert torch.equal(a.modes, b.modes)
    assert torch.equal(a.labels, b.labels)
    assert torch.equal(a.margins, b.margins)


@pytest.mark.parametrize("n", [1, 2, 3, 100])
def test_tiny_inputs(n):
    # points far apart relative to h (no pair near the a = h bifurcation,
    # where both sides converge only algebraically and stop short of the mode)
    rng = np.random.default_rng(n)
    if n <= 3:
        X = (np.array([[0.0, 0.0], [9.0, 1.0], [3.0, 8.0]])[:n]).astype(np.float32)
        w = fi.Workload(name=f"tiny{n}", X=X, h=1.0, tol=1e-3, max_iter=300)
    else:
        w = fi.separated_blobs(seed=n, k=4, d=2, per=n // 4, sigma=0.5, h=1.0)
    res = _run(w)
    ref = orc.cluster(w.X, w.h, w.tol, w.max_iter)
    _check(w, res, ref)


def test_maximum_dimension():
    # d = FMS_MAX_DIM = 64: the wide FP32 step, the block-wide prune and the
    # generic label kernel
    w = fi.separated_blobs(seed=64, k=6, d=64, per=250, sigma=0.7, h=2.0)
    res = _run(w, gamma=0.95, rng_seed=7, precision="fp32")
    ref = orc.cluster(w.X, w.h, w.tol, w.max_iter, gamma=0.95, rng_seed=7)
    _check(w, res, ref)
    assert res.stats["n_modes"] == 6


@pytest.mark.parametrize("d", [3, 16])
def test_one_update_only(d):
    # max_iter = 1: every seed makes one update; with gamma = 1 the seeds
    # that do not converge in it are kept where the update left them
    w = fi.separated_blobs(seed=90 + d, k=4, d=d, per=200, sigma=0.6, h=1.5)
    w1 = fi.Workload(name=w.name, X=w.X, h=w.h, tol=w.tol, max_iter=1)
    res = _run(w1, gamma=1.0, rng_seed=8, precision="fp32")
    ref = orc.cluster(w.X, w.h, w.tol, 1, gamma=1.0, rng_seed=8)
    _check(w1, res, ref)
    assert res.stats["iterations"] <= 1


def test_gamma_one_keeps_exhausted_seeds_on_the_host_path():
    # d = 16 runs the host-driven path; gamma = 1 with a small max_iter keeps
    # seeds that did not converge, whose prune densities come from a density
    # pass at their positions (not from their last update)
    w = fi.separated_blobs(seed=33, k=5, d=16, per=300, sigma=0.8, h=2.0)
    w6 = fi.Workload(name=w.name, X=w.X, h=w.h, tol=w.tol, max_iter=4)
    res = _run(w6, gamma=1.0, rng_seed=9, precision="fp32")
    ref = orc.cluster(w.X, w.h, w.tol, 4, gamma=1.0, rng_seed=9)
    _check(w6, res, ref)
    assert res.stats["n_kept"] == res.stats["n_seeds_final"]


def test_identical_points():
    X = np.full((500, 3), 2.5, dtype=np.float32)
    w = fi.Workload(name="same", X=X, h=1.0, tol=1e-3, max_iter=300)
    res = _run(w)
    assert res.stats["n_modes"] == 1
    assert np.allclose(res.modes.cpu().numpy(), 2.5)
    assert np.all(res.labels.cpu().numpy() == 0)


def test_errors():
    X = torch.zeros((10, 3), device="cuda")
    X[3, 1] = float("nan")
    with pytest.raises(fms.FmsError) as e:
        fms.cluster(X, 1.0)
    assert e.value.code == fms.FMS_ERR_NONFINITE
    with pytest.raises(fms.FmsError) as e:
        fms.cluster(torch.zeros((10, 3), device="cuda"), -1.0)
    assert e.value.code == fms.FMS_ERR_INVALID_ARG
    with pytest.raises(fms.FmsError) as e:
        fms.cluster(torch.zeros((10, 65), device="cuda"), 1.0)
    assert e.value.code == fms.FMS_ERR_INVALID_ARG
    w = fi.separated_blobs(seed=2, k=4, d=2, per=100, sigma=0.5, h=1.0)
    res = fms.cluster(torch.from_numpy(w.X).cuda(), w.h, max_modes=2)
    assert res.status == fms.FMS_ERR_CAPACITY and res.stats["n_modes"] == 4
    assert res.modes.shape[0] == 2


# The grid round's list handling at other list sizes than the default 128
# seeds: single short lists from the start (8 seeds: one seed per warp on the
# first warps), lists that merge into one (24, 40), several seed groups per
# warp (600 seeds: lists of 300, 18-19 seeds per warp), and other stop
# fractions (a t_stop that changes mid-round takes the serial compaction).
@pytest.mark.parametrize("n_initial,gamma", [(8, 0.95), (24, 0.9), (40, 0.99), (600, 0.95),
                                             (600, 0.8)])
def test_grid_round_list_sizes(n_initial, gamma):
    w = fi.paper_3d(n=40_000)
    res = _run(w, gamma=gamma, rng_seed=11, n_initial=n_initial)
    ref = orc.cluster(w.X, w.h, w.tol, w.max_iter, gamma=gamma, rng_seed=11, n_initial=n_initial)
    _check(w, res, ref)
    assert res.stats["n_seeds_final"] == ref.n_seeds
    assert res.stats["rounds"] == len(ref.n_history)
    assert res.stats["t_star_last"] == ref.t_star[-1]
    assert res.stats["n_kept"] == int(ref.kept.sum())
