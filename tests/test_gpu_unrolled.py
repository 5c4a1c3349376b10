"""GPU parity of the differentiable unrolled steps and their adjoint (A9).

Forward and adjoint are compared with the FP64 oracle (whose adjoint is
pinned by finite differences and autograd) on sets small enough for its dense
numpy code; FP32 budget: relative 2e-4 of each quantity's scale (weights carry
~1e-6 relative error, sums over <= 512 terms).  At the full configuration
(8 sets x 16,384 points, d = 16, T = 20, k = 5) the forward is checked on
sampled seeds (trajectories are independent of each other) and the backward
for finiteness and for the scaling identity
    h dL/dh = Y_T . G - X . dL/dX - Y0 . dL/dY0
(Y_T(cX, cY0, ch) = c Y_T(X, Y0, h), so differentiating L = G . Y_T along
(X, Y0, h) at c = 1 gives it).  A seed farther than 13 h from every point,
whose Gaussian weights all underflow in FP32, must come out as the oracle's
(which weighs relative to the nearest point), with finite gradients.
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


@pytest.mark.parametrize("d,n,T,k", [(2, 200, 3, 2), (4, 257, 4, 3), (16, 300, 5, 2), (7, 130, 2, 5),
                                     (1, 150, 3, 2), (32, 140, 3, 2)])
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


def test_far_seed_matches_oracle():
    # seed 0 starts 20 h away from every point: exp(-D^2 / 2h^2) < 1e-86, so
    # every unshifted FP32 weight is 0; the library recomputes such seeds with
    # weights relative to the nearest point, as the oracle does
    B, n, d, h, T, k = 1, 180, 3, 1.0, 3, 2
    X = _sets(44, B, n, d)
    rng = np.random.default_rng(9)
    Y0 = (X + 0.2 * rng.standard_normal(X.shape)).astype(np.float32)
    far = X[0].max(axis=0) + 20.0 * h
    Y0[0, 0] = far.astype(np.float32)
    D = np.sqrt(((X[0].astype(np.float64) - Y0[0, 0]) ** 2).sum(-1))
    assert D.min() > 15.0 * h
    G = rng.standard_normal(Y0.shape).astype(np.float32)
    Xt, Yt = torch.from_numpy(X).cuda(), torch.from_numpy(Y0).cuda()
    YT, ck = fms.unrolled_forward(Xt, Yt, h, T, k)
    dX, dY, dh = fms.unrolled_backward(Xt, ck, n, h, T, k, torch.from_numpy(G).cuda())
    torch.cuda.synchronize()
    ref = orc.unrolled_forward(X[0], Y0[0], h, T)[-1]
    got = YT[0].cpu().numpy()
    assert np.all(np.isfinite(got))
    assert np.abs(got - ref).max() <= 2e-4 * (1 + np.abs(ref).max())
    rdX, rdY, rdh = orc.unrolled_backward(X[0], Y0[0], h, T, G[0])
    for g_, want in ((dX[0], rdX), (dY[0], rdY)):
        g_ = g_.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(g_))
        assert np.abs(g_ - want).max() <= 2e-4 * (1 + np.abs(want).max())
    assert abs(dh[0].item() - rdh) <= 2e-4 * (1 + abs(rdh))


def test_fp64_kernels_match_oracle_tightly():
    # the FP64 entry points run the same kernels in double precision: forward
    # and adjoint agree with the FP64 oracle to ~1e-10 (rounding order only)
    B, n, d, h, T, k = 2, 120, 4, 1.5, 4, 3
    X = _sets(61, B, n, d).astype(np.float64)
    rng = np.random.default_rng(3)
    Y0 = X + 0.25 * rng.standard_normal(X.shape)
    G = rng.standard_normal(X.shape)
    Xt, Yt = torch.from_numpy(X).cuda(), torch.from_numpy(Y0).cuda()
    YT, ck = fms.unrolled_forward(Xt, Yt, h, T, k)
    assert YT.dtype == torch.float64
    dX, dY, dh = fms.unrolled_backward(Xt, ck, n, h, T, k, torch.from_numpy(G).cuda())
    torch.cuda.synchronize()
    for b in range(B):
        ref = orc.unrolled_forward(X[b], Y0[b], h, T)[-1]
        assert np.abs(YT[b].cpu().numpy() - ref).max() <= 1e-10 * (1 + np.abs(ref).max())
        rdX, rdY, rdh = orc.unrolled_backward(X[b], Y0[b], h, T, G[b])
        for got, want in ((dX[b], rdX), (dY[b], rdY)):
            got = got.cpu().numpy()
            assert np.abs(got - want).max() <= 1e-9 * (1 + np.abs(want).max())
        assert abs(dh[b].item() - rdh) <= 1e-9 * (1 + abs(rdh))


def test_gradcheck_fp64_on_gpu():
    # torch.autograd.gradcheck of the library's adjoint (FP64 kernels on the
    # GPU) against central finite differences of its own forward, n = 64, d = 4
    B, n, d, T, k = 1, 64, 4, 3, 2
    X = torch.from_numpy(_sets(62, B, n, d).astype(np.float64)).cuda().requires_grad_(True)
    g = torch.Generator(device="cuda").manual_seed(5)
    Y0 = (X.detach() + 0.2 * torch.randn(X.shape, generator=g, device="cuda",
                                          dtype=torch.float64)).requires_grad_(True)
    h = torch.tensor(1.7, dtype=torch.float64, device="cuda", requires_grad=True)
    fn = lambda X_, Y_, h_: fms.unrolled_mean_shift(X_, Y_, h_, T, k)
    assert torch.autograd.gradcheck(fn, (X, Y0, h), eps=1e-6, atol=1e-7, rtol=1e-5)
