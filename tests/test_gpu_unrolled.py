"""GPU parity of the differentiable unrolled steps and their adjoint (A9).

Forward and adjoint are compared with the FP64 oracle (whose adjoint is
pinned by finite differences and autograd) on sets small enough for its dense
numpy code; FP32 budget: relative 2e-4 of each quantity's scale (weights carry
~1e-6 relative error, sums over <= 512 terms).  At the full configuration
(8 sets x 16,384 points, d = 16, T = 20, k = 5) the forward is checked on
sampled seeds (trajectories are independent of each other) and the backward
for finiteness and for the identity dL/dh = -(1/h) [dL/dX . X + dL/dY0 . Y0]
(the map is invariant to scaling X, Y0 and h together, so its derivative
along (X, Y0, h) vanishes).
"""
import numpy as np
import pytest
import torch

import fms_inputs as fi
import oracle as orc

pytestmark = pytest.mark.gpu

fms = pytest.importorskip("paper_2112_13891_gb300")


def _sets(seed, B, n, d, k=4):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(B):
        c = rng.uniform(0, 12, (k, d))
        X = c[rng.integers(0, k, n)] + rng.standard_normal((n, d))
        out.append(X)
    return np.stack(out).astype(np.float32)


@pytest.mark.parametrize("d,n,T,k", [(2, 200, 3, 2), (4, 257, 4, 3), (16, 300, 5, 2), (7, 130, 2, 5)])
def test_forward_and_adjoint_match_oracle(d, n, T, k):
    B, h = 2, 2.0
    X = _sets(d * 100 + n, B, n, d)
    rng = np.random.default_rng(7)
    Y0 = (X + 0.3 * rng.standard_normal(X.shape)).astype(np.float32)
    G = rng.standard_normal(X.shape).astype(np.float32)
    Xt, Yt = torch.from_numpy(X).cuda(), torch.from_numpy(Y0).cuda()
    YT, ck = fms.unrolled_forward(Xt, Yt, h, T, k)
    dX, dY, dh = fms.unrolled_backward(Xt, ck, n, h, T, k, torch.from_numpy(G).cuda())
    torch.cuda.synchronize()
    for b in range(B):
        ref = orc.unrolled_forward(X[b], Y0[b], h, T)[-1]
        assert np.abs(YT[b].cpu().numpy() - ref).max() <= 2e-4 * (1 + np.abs(ref).max())
        rdX, rdY, rdh = orc.unrolled_backward(X[b], Y0[b], h, T, G[b])
        for got, want in ((dX[b], rdX), (dY[b], rdY)):
            got = got.cpu().numpy().astype(np.float64)
            assert np.abs(got - want).max() <= 2e-4 * (1 + np.abs(want).max()), np.abs(got - want).max()
        assert abs(dh[b].item() - rdh) <= 2e-4 * (1 + abs(rdh))


def test_autograd_function():
    B, n, d, h, T, k = 1, 150, 4, 1.5, 3, 2
    X = _sets(3, B, n, d)
    Xt = torch.from_numpy(X).cuda().requires_grad_(True)
    Yt = (torch.from_numpy(X).cuda() + 0.1).requires_grad_(True)
    ht = torch.tensor(h, device="cuda", requires_grad=True)
    out = fms.unrolled_mean_shift(Xt, Yt, ht, T, k)
    G = torch.randn_like(out)
    (out * G).sum().backward()
    rdX, rdY, rdh = orc.unrolled_backward(X[0], (X[0] + 0.1).astype(np.float32), h, T,
                                          G[0].cpu().numpy())
    assert np.abs(Xt.grad[0].cpu().numpy() - rdX).max() <= 2e-4 * (1 + np.abs(rdX).max())
    assert np.abs(Yt.grad[0].cpu().numpy() - rdY).max() <= 2e-4 * (1 + np.abs(rdY).max())
    assert abs(ht.grad.item() - rdh) <= 2e-4 * (1 + abs(rdh))


def test_full_configuration_sampled():
    w = fi.unrolled_16d()
    X = w.X                                        # [8, 16384, 16]
    B, n, d = X.shape
    h, T, k = w.h, w.T, w.k_ckpt
    Xt = torch.from_numpy(X).cuda()
    YT, ck = fms.unrolled_forward(Xt, Xt, h, T, k)
    G = torch.randn_like(YT)
    dX, dY, dh = fms.unrolled_backward(Xt, ck, n, h, T, k, G)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    for b in (0, B - 1):
        idx = rng.choice(n, 8, replace=False)
        ref = orc.unrolled_forward(X[b], X[b][idx], h, T)[-1]
        assert np.abs(YT[b].cpu().numpy()[idx] - ref).max() <= 1e-3 * (1 + np.abs(ref).max())
    assert torch.isfinite(dX).all() and torch.isfinite(dY).all() and torch.isfinite(dh).all()
    # scale invariance: Y_T(cX, cY0, ch) = c Y_T(X, Y0, h)  =>  h dL/dh = -(X.dX + Y0.dY) + Y_T.G
    lhs = h * dh.cpu().numpy()
    rhs = (-(Xt * dX).sum(dim=(1, 2)) - (Xt * dY).sum(dim=(1, 2)) + (YT * G).sum(dim=(1, 2)))
    rhs = rhs.double().cpu().numpy()
    scale = ((Xt * dX).abs().sum(dim=(1, 2)) + (YT * G).abs().sum(dim=(1, 2))).double().cpu().numpy()
    assert np.all(np.abs(lhs - rhs) <= 1e-3 * scale), (lhs, rhs)
