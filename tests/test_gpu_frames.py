"""N3: the frame-sequence API (fms_cluster_frames) against the oracle's
cluster_frames: per frame the modes and labels, and the seed count each frame
starts with (Sec. II-D: N is carried over and reduced by M when N > H*M)."""
import numpy as np
import pytest
import torch

import fms_inputs as fi
import oracle as orc
from fms_compare import compare_clustering

pytestmark = pytest.mark.gpu

fms = pytest.importorskip("paper_2112_13891_gb300")


@pytest.mark.parametrize("n_initial,H", [(512, 32.0), (128, 32.0), (400, 4.0)])
def test_frames_match_oracle(n_initial, H):
    frames = fi.drifting_frames(seed=n_initial, frames=5, n=20_000, k=8)
    h, tol = 5.0, 5e-3
    res = fms.cluster_frames(torch.from_numpy(np.stack(frames)).cuda(), h, tol, 300, H=H,
                             n_initial=n_initial, gamma=0.95, rng_seed=2)
    torch.cuda.synchronize()
    ref, starts = orc.cluster_frames(frames, h, tol, 300, n_initial=n_initial, H=H,
                                     gamma=0.95, rng_seed=2)
    assert res.seed_counts == starts
    for f, X in enumerate(frames):
        cmp = compare_clustering(res.modes[f].cpu().numpy(), res.labels[f].cpu().numpy(),
                                 ref[f], h)
        assert cmp["mode_ok"] and cmp["label_mismatch"] == 0, (f, cmp)


def test_frames_reject_fixed_seed_counts():
    X = torch.zeros((2, 100, 3), device="cuda")
    o = fms.make_options(all_seeds=True)
    code = fms._lib.fms_cluster_frames(X.data_ptr(), 2, 100, 3, 1.0, 0.0, 10, fms.ctypes.byref(o),
                                       32.0, None, 0, (fms._I32 * 2)(), X.data_ptr(), None, None,
                                       None, 0, None, None)
    assert code == fms.FMS_ERR_INVALID_ARG
