"""N1: the image-pixel workload (512x512x3 and 1024x1024x3 RGB-like values)
through the d = 3 path, against the FP64 oracle on the same seeded pixels.

Acceptance as for every clustering: modes matched one-to-one within 1e-3*h,
labels identical away from oracle margins below 1e-2*h, and the Early-Stopping
bookkeeping (seed history, stop update, kept count) equal to the oracle's.
"""
import numpy as np
import pytest
import torch

import fms_inputs as fi
import oracle as orc
from fms_compare import compare_clustering

pytestmark = pytest.mark.gpu

fms = pytest.importorskip("paper_2112_13891_gb300")


@pytest.mark.parametrize("side", [512, 1024])
def test_pixels_match_oracle(side):
    w = fi.pixels_rgb(seed=side, height=side, width=side)
    X = torch.from_numpy(w.X).cuda()
    res = fms.cluster(X, w.h, w.tol, w.max_iter, gamma=0.95, rng_seed=0)
    torch.cuda.synchronize()
    ref = orc.cluster(w.X, w.h, w.tol, w.max_iter, gamma=0.95, rng_seed=0)
    cmp = compare_clustering(res.modes.cpu().numpy(), res.labels.cpu().numpy(), ref, w.h)
    print(w.name, cmp, res.stats)
    assert cmp["mode_ok"], cmp
    assert cmp["label_mismatch"] == 0, cmp
    assert res.stats["rounds"] == len(ref.n_history)
    assert res.stats["t_star_last"] == ref.t_star[-1]
    assert res.stats["n_kept"] == int(ref.kept.sum())
    # every pixel labelled with a valid mode
    lab = res.labels.cpu().numpy()
    assert lab.min() >= 0 and lab.max() < res.modes.shape[0]
