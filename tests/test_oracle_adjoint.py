"""Pins of the oracle's unrolled-step adjoint (no GPU).

The adjoint of T Gaussian mean-shift updates is checked in float64 against
(a) central finite differences of the forward and (b) torch autograd through
a dense torch float64 forward written independently here.
"""
import numpy as np
import pytest
import torch

import oracle as orc


def _problem(seed=0, n=64, d=4, m=None):
    rng = np.random.default_rng(seed)
    X = np.concatenate([rng.standard_normal((n // 2, d)), rng.standard_normal((n - n // 2, d)) + 2.5])
    Y0 = X[: (m or n)] + 0.1 * rng.standard_normal(((m or n), d))
    G = rng.standard_normal(((m or n), d))
    return X, Y0, G


def _loss(X, Y0, h, T, G):
    return float((orc.unrolled_forward(X, Y0, h, T)[-1] * G).sum())


@pytest.mark.parametrize("T", [1, 3])
def test_adjoint_vs_finite_differences(T):
    X, Y0, G = _problem(n=24, d=3)
    h = 1.3
    dX, dY, dh = orc.unrolled_backward(X, Y0, h, T, G)
    rng = np.random.default_rng(1)
    e = 1e-6
    for _ in range(6):
        i, k = rng.integers(0, X.shape[0]), rng.integers(0, X.shape[1])
        Xp, Xm = X.copy(), X.copy()
        Xp[i, k] += e
        Xm[i, k] -= e
        fd = (_loss(Xp, Y0, h, T, G) - _loss(Xm, Y0, h, T, G)) / (2 * e)
        assert abs(fd - dX[i, k]) <= 1e-6 * (1 + abs(fd))
        Yp, Ym = Y0.copy(), Y0.copy()
        Yp[i, k] += e
        Ym[i, k] -= e
        fd = (_loss(X, Yp, h, T, G) - _loss(X, Ym, h, T, G)) / (2 * e)
        assert abs(fd - dY[i, k]) <= 1e-6 * (1 + abs(fd))
    fd = (_loss(X, Y0, h + e, T, G) - _loss(X, Y0, h - e, T, G)) / (2 * e)
    assert abs(fd - dh) <= 1e-6 * (1 + abs(fd))


def test_adjoint_vs_torch_autograd():
    X, Y0, G = _problem(n=64, d=4)
    h, T = 2.0, 5
    Xt = torch.tensor(X, dtype=torch.float64, requires_grad=True)
    Yt = torch.tensor(Y0, dtype=torch.float64, requires_grad=True)
    ht = torch.tensor(h, dtype=torch.float64, requires_grad=True)
    Y = Yt
    for _ in range(T):
        D = torch.cdist(Y, Xt) ** 2
        P = torch.softmax(-D / (2 * ht * ht), dim=1)
        Y = P @ Xt
    (Y * torch.tensor(G)).sum().backward()
    dX, dY, dh = orc.unrolled_backward(X, Y0, h, T, G)
    assert np.max(np.abs(dX - Xt.grad.numpy())) <= 1e-9 * (1 + np.max(np.abs(dX)))
    assert np.max(np.abs(dY - Yt.grad.numpy())) <= 1e-9 * (1 + np.max(np.abs(dY)))
    assert abs(dh - ht.grad.item()) <= 1e-9 * (1 + abs(dh))
