"""GPU parity of the individual steps through the C ABI (needs a GB300).

* Seed Selection: bit-exact against the oracle's keyed permutation.
* One mean-shift update (ms_step + update): within the FP32 error budget of
  the update, |gpu - oracle| <= 2e-4*h + 2^-20*|y| per coordinate.  The
  budget: the points are scaled by s = sqrt(log2(e)/(2h^2)) in FP32 (relative
  rounding 2^-24 of each coordinate), so each weight carries a relative error
  of about 2*|y-x|*s^2*|x|*2^-24*ln2 (< 1e-5 for the sizes below), which moves
  the weighted mean by at most that fraction of the kernel's spread (a few h);
  the FP32 position itself rounds at 2^-24*|y|.
* Nearest-mode labels: identical wherever the oracle margin exceeds 1e-4 of
  the point-mode distance scale; margins within 1e-4 relative.
"""
import numpy as np
import pytest
import torch

import oracle as orc

pytestmark = pytest.mark.gpu

fms = pytest.importorskip("paper_2112_13891_gb300")


@pytest.mark.parametrize("n", [1, 2, 5, 127, 128, 1000, 65536, 200_000, 262_145])
@pytest.mark.parametrize("key", [0, 7, 0xFEEDFACE12345678])
def test_select_seeds_bit_exact(n, key):
    count = min(n, 700)
    got = fms.select_seeds(n, key, 0, count).cpu().numpy()
    want = orc.seed_permutation(n, key, 0, count)
    assert np.array_equal(got, want)
    if n > 300:
        got2 = fms.select_seeds(n, key, 256, 44).cpu().numpy()
        assert np.array_equal(got2, want[256:300])


def _cloud(rng, n, d, box=50.0):
    k = 5
    c = rng.uniform(0, box, (k, d))
    lab = rng.integers(0, k, n)
    return (c[lab] + rng.standard_normal((n, d)) * 2.0).astype(np.float32)


@pytest.mark.parametrize("d", [1, 2, 3, 4, 5, 7, 8, 12, 16, 32, 64])
@pytest.mark.parametrize("n,m", [(1, 1), (33, 5), (4097, 37), (20011, 301)])
def test_mean_shift_step_parity(d, n, m):
    rng = np.random.default_rng(1000 * d + n + m)
    X = _cloud(rng, n, d)
    h = 3.0
    Y = (X[rng.integers(0, n, m)] + rng.standard_normal((m, d)).astype(np.float32)).astype(np.float32)
    out, W = fms.mean_shift_step(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), h,
                                 with_wsum=True)
    out = out.cpu().numpy().astype(np.float64)
    W = W.cpu().numpy().astype(np.float64)
    ref = orc.step(X, Y, h)
    tol = 2e-4 * h + 2.0 ** -20 * np.abs(ref).max()
    err = np.abs(out - ref).max()
    assert err <= tol, (err, tol)
    refW = orc.kde(X, Y, h)
    assert np.all(np.abs(W - refW) <= 1e-4 * refW + 1e-30), np.abs(W / refW - 1).max()


def test_mean_shift_step_large_seed_count():
    """All-seeds shaped launch: many seed groups, few chunks."""
    rng = np.random.default_rng(5)
    X = _cloud(rng, 30000, 3, box=200.0)
    h = 5.0
    Y = X[::3].copy()
    out = fms.mean_shift_step(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), h).cpu().numpy()
    sample = rng.choice(Y.shape[0], 400, replace=False)
    ref = orc.step(X, Y[sample], h)
    tol = 2e-4 * h + 2.0 ** -20 * np.abs(ref).max()
    assert np.abs(out[sample] - ref).max() <= tol


@pytest.mark.parametrize("d", [1, 2, 3, 16, 64])
@pytest.mark.parametrize("n,M", [(1, 1), (1000, 1), (5000, 7), (70001, 300), (3000, 9000)])
def test_label_parity(d, n, M):
    rng = np.random.default_rng(d * 7 + M)
    X = rng.uniform(-20, 20, (n, d)).astype(np.float32)
    modes = rng.uniform(-20, 20, (M, d)).astype(np.float32)
    if M > 3:
        modes[2] = modes[1]            # exact tie: lowest index wins on both sides
    lab, mar = fms.label_points(torch.from_numpy(X).cuda(), torch.from_numpy(modes).cuda())
    lab = lab.cpu().numpy()
    mar = mar.cpu().numpy().astype(np.float64)
    rlab, rmar = orc.label(X, modes)
    if M == 1:
        assert np.all(lab == 0) and np.all(np.isinf(mar))
        return
    scale = np.sqrt(d) * 20.0
    ok = rmar > 1e-4 * scale
    assert np.array_equal(lab[ok], rlab[ok])
    assert np.all(np.abs(mar - rmar) <= 1e-4 * scale)
