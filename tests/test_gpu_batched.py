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


def _check_set_all_seeds(w, modes, labels):
    ref = orc.cluster(w.X, w.h, w.tol, w.max_iter, all_seeds=True)
    cmp = compare_clustering(modes.cpu().numpy(), labels.cpu().numpy(), ref, w.h)
    assert cmp["mode_ok"], cmp
    assert cmp["label_mismatch"] == 0, cmp


def test_batched_all_seeds_sets_above_the_on_chip_prune():
    # every point a seed (Alg. 1 per set).  Set 0 (20,000 points, d = 3) has
    # more prune candidates than the sorted visit's keys can hold in shared
    # memory, so its prune takes the global-memory greedy; set 1 (2,500
    # points) sorts on chip; set 2 is small.
    h = 1.5
    sets = [fi.separated_blobs(seed=41, k=5, d=3, per=4000, sigma=1.0, h=h),
            fi.separated_blobs(seed=42, k=5, d=3, per=500, sigma=1.0, h=h),
            fi.separated_blobs(seed=43, k=3, d=3, per=100, sigma=1.0, h=h)]
    X = [torch.from_numpy(w.X).cuda() for w in sets]
    res = fms.cluster_batched(X, h, 1e-3 * h, 300, all_seeds=True, max_modes=64)
    assert res.status == fms.FMS_OK
    assert res.stats["graph"] == 1
    assert res.stats["n_kept"] > 16384 + 2000
    off = np.concatenate([[0], np.cumsum([w.X.shape[0] for w in sets])])
    for b, w in enumerate(sets):
        _check_set_all_seeds(w, res.modes[b], res.labels[off[b]:off[b + 1]])


def test_batched_all_seeds_wide_set_reads_modes_from_global_memory():
    # d = 16, 2,500 candidates: the sort keys fit in shared memory but the
    # accepted modes' coordinates do not, so the visit reads them back from
    # global memory
    h = 3.0
    sets = [fi.separated_blobs(seed=44, k=5, d=16, per=500, sigma=1.0, h=h),
            fi.separated_blobs(seed=45, k=4, d=16, per=150, sigma=1.0, h=h)]
    X = [torch.from_numpy(w.X).cuda() for w in sets]
    res = fms.cluster_batched(X, h, 1e-3 * h, 300, all_seeds=True, max_modes=64)
    assert res.status == fms.FMS_OK
    off = np.concatenate([[0], np.cumsum([w.X.shape[0] for w in sets])])
    for b, w in enumerate(sets):
        _check_set_all_seeds(w, res.modes[b], res.labels[off[b]:off[b + 1]])


def test_batched_call_is_one_graph_with_counted_launches():
    # the second call with the same arguments reuses the cached graph; both
    # report the same work and a launch count that follows the loop counts
    h = 1.5
    sets = _mixed_sets(5, 8, 3, 400, 3000, h)
    X = [torch.from_numpy(w.X).cuda() for w in sets]
    Xc = torch.cat(X)
    offs = np.concatenate([[0], np.cumsum([x.shape[0] for x in X])]).astype(np.int64)
    r1 = fms.cluster_batched(Xc, h, 1e-3 * h, 300, offsets=offs, max_modes=64)
    r2 = fms.cluster_batched(Xc, h, 1e-3 * h, 300, offsets=offs, max_modes=64)
    for r in (r1, r2):
        assert r.status == fms.FMS_OK and r.stats["graph"] == 1
    s1, s2 = r1.stats, r2.stats
    for k in ("rounds", "evals", "n_modes", "n_seeds_final", "refine_iterations",
              "kernel_launches"):
        assert s1[k] == s2[k], k
    assert s1["rounds"] >= 1
    # launches: 2 before the rounds, 7 per round plus 3 per update, 2 + 3 per
    # refinement update, 4 for the density pass and 3 after
    upd = (s1["kernel_launches"] - 2 - 7 * s1["rounds"] - 2 - 3 * s1["refine_iterations"] - 7)
    assert upd > 0 and upd % 3 == 0
    for b in range(len(sets)):
        assert torch.equal(r1.modes[b], r2.modes[b])
    assert torch.equal(r1.labels, r2.labels)


def test_batched_sets_of_other_sizes_reuse_nothing_stale():
    # same B, total and largest size with a different split: the control
    # blocks are copied in before every launch, so the cached graph gives
    # the per-set results of the new split
    h = 1.5
    base = [fi.separated_blobs(seed=51, k=5, d=3, per=300, sigma=1.0, h=h),
            fi.separated_blobs(seed=52, k=4, d=3, per=200, sigma=1.0, h=h),
            fi.separated_blobs(seed=53, k=3, d=3, per=300, sigma=1.0, h=h),
            fi.separated_blobs(seed=54, k=5, d=3, per=400, sigma=1.0, h=h)]
    X = torch.cat([torch.from_numpy(w.X) for w in base]).cuda()
    offs_a = np.array([0, 1500, 2300, 3200, 5200], dtype=np.int64)
    offs_b = np.array([0, 1500, 2200, 3200, 5200], dtype=np.int64)   # 100 points move to set 2
    for offs in (offs_a, offs_b, offs_a):
        res = fms.cluster_batched(X, h, 1e-3 * h, 300, offsets=offs, max_modes=64)
        assert res.status == fms.FMS_OK
        for b in range(4):
            one = fms.cluster(X[offs[b]:offs[b + 1]].contiguous(), h, 1e-3 * h, 300)
            assert one.modes.shape == res.modes[b].shape
            assert torch.allclose(one.modes, res.modes[b], atol=1e-3 * h, rtol=0)


def test_batched_nonfinite_point_ends_the_graph_with_an_error():
    # a NaN point: the packing kernel flags it, every conditional node's
    # condition goes false, the graph runs to its end and the call reports
    # FMS_ERR_NONFINITE (it neither hangs nor returns OK); a clean call with
    # the same shapes afterwards still succeeds
    h = 1.5
    sets = _mixed_sets(21, 3, 3, 300, 900, h)
    X = torch.cat([torch.from_numpy(w.X) for w in sets]).cuda()
    offs = np.concatenate([[0], np.cumsum([w.X.shape[0] for w in sets])]).astype(np.int64)
    bad = X.clone()
    bad[int(offs[1]) + 5, 1] = float("nan")
    with pytest.raises(fms.FmsError) as e:
        fms.cluster_batched(bad, h, 1e-3 * h, 300, offsets=offs, max_modes=64)
    assert e.value.code == fms.FMS_ERR_NONFINITE
    ok = fms.cluster_batched(X, h, 1e-3 * h, 300, offsets=offs, max_modes=64)
    assert ok.status == fms.FMS_OK


@pytest.mark.parametrize("d", [2, 64])
def test_batched_degenerate_and_wide_sets(d):
    # one-point and two-point sets next to ordinary ones (d = 2), and d = 64
    # (the widest staged step); every set against the oracle run alone
    h = 2.0 if d == 2 else 6.0
    rng = np.random.default_rng(70 + d)
    sets = [rng.normal(0, 1, (1, d)).astype(np.float32),
            (rng.normal(0, 1, (2, d)) * 0.1).astype(np.float32),
            fi.separated_blobs(seed=71 + d, k=3, d=d, per=80, sigma=1.0, h=h).X]
    X = [torch.from_numpy(x).cuda() for x in sets]
    res = fms.cluster_batched(X, h, 1e-3 * h, 300, max_modes=32)
    assert res.status == fms.FMS_OK
    off = np.concatenate([[0], np.cumsum([x.shape[0] for x in sets])])
    for b, x in enumerate(sets):
        ref = orc.cluster(x, h, 1e-3 * h, 300, gamma=0.95, rng_seed=0)
        cmp = compare_clustering(res.modes[b].cpu().numpy(), res.labels[off[b]:off[b + 1]].cpu().numpy(), ref, h)
        assert cmp["mode_ok"] and cmp["label_mismatch"] == 0, (b, cmp)


def test_batched_single_set_equals_single_call():
    h = 1.5
    w = fi.separated_blobs(seed=80, k=4, d=3, per=300, sigma=1.0, h=h)
    X = torch.from_numpy(w.X).cuda()
    res = fms.cluster_batched([X], h, 1e-3 * h, 300, max_modes=32)
    one = fms.cluster(X, h, 1e-3 * h, 300)
    assert one.modes.shape == res.modes[0].shape
    assert torch.allclose(one.modes, res.modes[0], atol=1e-3 * h, rtol=0)
    assert torch.equal(one.labels, res.labels)
