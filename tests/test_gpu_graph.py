"""The CUDA-graph form of fms_cluster.

A call seen for the second time with the same arguments (pointers, sizes,
scalars, options) runs as one cached CUDA graph: a conditional WHILE node
repeats the round (the persistent grid round, stop bookkeeping with the
density scores, prune, seed-count decision) while the device asks for another round, and an
IF node runs the refinement, second prune, ordering and labels; the host
synchronises once.  The graph launches the same kernels with the same
arguments as the host-driven path, so results must be bit-identical to it;
when a round or the refinement would not fit the cluster kernels, the graph
hands the state back to the host path (tested by forcing both cases).
"""
import numpy as np
import pytest
import torch

import fms_inputs as fi
import oracle as orc
from fms_compare import compare_clustering

pytestmark = pytest.mark.gpu

fms = pytest.importorskip("paper_2112_13891_gb300")


def _three_calls(X, h, tol, max_iter, **kw):
    """Host path, then the graph built on the second call, then the cached
    graph; all three into the same buffers (cloned after each call)."""
    n, d = X.shape
    ws = fms.Workspace(fms.workspace_size(n, d, **{k: v for k, v in kw.items()
                                                   if k in ("gamma", "L", "n_initial")}), X.device)
    modes = torch.empty((n, d), dtype=torch.float32, device=X.device)
    labels = torch.empty(n, dtype=torch.int32, device=X.device)
    margins = torch.empty(n, dtype=torch.float32, device=X.device)
    out = []
    for _ in range(3):
        modes.fill_(float("nan"))
        labels.fill_(-7)
        margins.fill_(float("nan"))
        r = fms.cluster(X, h, tol, max_iter, workspace=ws, out=(modes, labels, margins), **kw)
        torch.cuda.synchronize()
        out.append((r.modes.clone(), labels.clone(), margins.clone(), dict(r.stats)))
    return out


def _identical(out):
    for m, l, g, st in out[1:]:
        assert torch.equal(m, out[0][0])
        assert torch.equal(l, out[0][1])
        assert torch.equal(g, out[0][2])
        for k in ("n_modes", "rounds", "n_seeds_final", "n_kept", "t_star_last", "iterations",
                  "refine_iterations", "n_converged"):
            assert st[k] == out[0][3][k], (k, st[k], out[0][3][k])


def test_graph_matches_host_path_paper_3d():
    w = fi.paper_3d(n=60_000)
    X = torch.from_numpy(w.X).cuda()
    out = _three_calls(X, w.h, w.tol, w.max_iter, gamma=0.95, rng_seed=0)
    _identical(out)
    st = out[1][3]
    # the graph: packing, seed init, round start; 4 launches per round (grid
    # round, stop bookkeeping, prune, seed-count decision); 4 after
    assert st["kernel_launches"] == 3 + 4 * st["rounds"] + 4
    assert out[0][3]["graph"] == 0 and out[1][3]["graph"] == 1 and out[2][3]["graph"] == 1
    ref = orc.cluster(w.X, w.h, w.tol, w.max_iter, gamma=0.95, rng_seed=0)
    cmp = compare_clustering(out[2][0].cpu().numpy(), out[2][1].cpu().numpy(), ref, w.h)
    assert cmp["mode_ok"] and cmp["label_mismatch"] == 0, cmp


@pytest.mark.parametrize("kernel", ["gaussian", "flat"])
def test_graph_matches_host_path_blobs(kernel):
    w = fi.separated_blobs(seed=11, k=12, d=3, per=500, sigma=0.6, h=1.5)
    X = torch.from_numpy(w.X).cuda()
    out = _three_calls(X, w.h, w.tol, w.max_iter, gamma=0.95, rng_seed=4, kernel=kernel)
    _identical(out)
    assert out[2][3]["graph"] == 1


def test_graph_hands_back_a_round_too_large_for_the_clusters():
    """~300 separated blobs: N doubles past what the cluster kernels take
    (15 clusters x 64 seeds), so the graph stops and the host path runs the
    next round; the result must match the host path and the oracle."""
    rng = np.random.default_rng(5)
    k, per = 300, 20
    C = rng.uniform(0, 2000.0, (k, 2))
    X = (np.repeat(C, per, axis=0) + 0.3 * rng.standard_normal((k * per, 2))).astype(np.float32)
    h = 1.0
    Xd = torch.from_numpy(X).cuda()
    out = _three_calls(Xd, h, 1e-3 * h, 300, gamma=0.95, rng_seed=2)
    _identical(out)
    assert out[0][3]["n_seeds_final"] > 960
    assert out[2][3]["graph"] == 1
    ref = orc.cluster(X, h, 1e-3 * h, 300, gamma=0.95, rng_seed=2)
    cmp = compare_clustering(out[2][0].cpu().numpy(), out[2][1].cpu().numpy(), ref, h)
    assert cmp["mode_ok"] and cmp["label_mismatch"] == 0, cmp


def test_graph_hands_back_a_refinement_too_large_for_the_clusters():
    """More than 15 x 32 merged modes: the refinement runs on the host path."""
    rng = np.random.default_rng(6)
    k, per = 900, 6   # 960 seeds hit ~590 of the 900 blobs
    C = rng.uniform(0, 4000.0, (k, 2))
    X = (np.repeat(C, per, axis=0) + 0.2 * rng.standard_normal((k * per, 2))).astype(np.float32)
    h = 1.0
    Xd = torch.from_numpy(X).cuda()
    out = _three_calls(Xd, h, 1e-3 * h, 300, gamma=0.95, rng_seed=3, n_initial=960, L=1.0)
    _identical(out)
    assert out[0][3]["n_modes"] > 480
    assert out[2][3]["graph"] == 1


def test_concurrent_host_threads():
    # the graph cache, the pinned readback buffer and the capture streams are
    # per host thread: two threads clustering repeatedly on their own streams
    # and workspaces get the serial call's bits (graph form from the second
    # call on)
    import threading
    w = fi.separated_blobs(seed=21, k=6, d=3, per=500, sigma=0.6, h=1.5)
    X = torch.from_numpy(w.X).cuda()
    n, d = X.shape
    ref = fms.cluster(X, w.h, w.tol, w.max_iter, gamma=0.95, rng_seed=5)
    torch.cuda.synchronize()
    results, errors = {}, []

    def worker(tid):
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                ws = fms.Workspace(fms.workspace_size(n, d), X.device)
                modes = torch.empty((n, d), device="cuda")
                labels = torch.empty(n, dtype=torch.int32, device="cuda")
                margins = torch.empty(n, device="cuda")
                out = []
                for _ in range(4):
                    r = fms.cluster(X, w.h, w.tol, w.max_iter, gamma=0.95, rng_seed=5,
                                    workspace=ws, out=(modes, labels, margins))
                    out.append((r.modes.clone(), labels.clone(), r.stats["graph"]))
                s.synchronize()
            results[tid] = out
        except Exception as e:   # reported below
            errors.append(e)

    threads = [threading.Thread(target=worker, args=(t,)) for t in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for tid in range(2):
        assert [o[2] for o in results[tid]] == [0, 1, 1, 1]
        for m, lab, _ in results[tid]:
            assert torch.equal(m, ref.modes) and torch.equal(lab, ref.labels)
