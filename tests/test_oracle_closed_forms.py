"""Pins of the FP64 oracle against closed forms (no GPU).

Each case has an answer fixed by mathematics, not by the oracle's own formula:
  * two points at +-a in 1-D: one Gaussian mean-shift update maps y to
    a*tanh(a*y/h^2); the modes are 0 (a <= h) or +-m with m = a*tanh(a*m/h^2);
  * a regular k-gon of radius r: its centre is a fixed point by symmetry and a
    local maximum of the density iff r < sqrt(2)*h;
  * the Gaussian mean-shift vector equals h^2 * grad f / f (Sec. II-A Eq. 6
    with the Gaussian profile), checked with finite differences of the density.
"""
import math

import numpy as np
import pytest
from scipy.optimize import brentq

import oracle as orc


@pytest.mark.parametrize("a,h", [(1.0, 1.5), (2.0, 1.0), (0.3, 0.2), (5.0, 4.0)])
@pytest.mark.parametrize("y", [-0.7, 0.0, 0.25, 1.3, 3.0])
def test_two_point_single_update_is_tanh(a, h, y):
    X = np.array([[a], [-a]])
    got = orc.step(X, np.array([[y]]), h)[0, 0]
    want = a * math.tanh(a * y / (h * h))
    assert abs(got - want) <= 1e-13 * max(1.0, abs(want))


@pytest.mark.parametrize("a,h", [(0.5, 1.0), (1.0, 1.0), (1.5, 1.0), (3.0, 1.0), (2.2, 1.7)])
def test_two_point_modes(a, h):
    X = np.array([[a], [-a]])
    # at a == h the update is y <- h*tanh(y/h) ~ y - y^3/(3h^2): the step falls
    # below tol once |y| ~ (3 tol h^2)^(1/3), so only that bound holds there
    tol = 1e-9 * h if a == h else 1e-12 * h
    Y, conv, _ = orc.trajectories(X, np.array([[a], [-a]]), h, tol, 1000000)
    assert np.all(conv > 0)
    if a <= h:
        bound = 1.01 * (3 * tol * h * h) ** (1 / 3) if a == h else 1e-9 * h
        assert np.all(np.abs(Y[:, 0]) <= bound)
    else:
        m = brentq(lambda t: t - a * math.tanh(a * t / (h * h)), 1e-9, a + 1.0)
        assert abs(Y[0, 0] - m) <= 1e-9 * h
        assert abs(Y[1, 0] + m) <= 1e-9 * h


def test_two_points_in_d_dims_reduce_to_1d():
    rng = np.random.default_rng(7)
    for d in (2, 3, 5, 16):
        u = rng.standard_normal(d)
        u /= np.linalg.norm(u)
        c = rng.uniform(-3, 3, d)
        a, h = 1.7, 1.1
        X = np.stack([c + a * u, c - a * u])
        for y1 in (-0.4, 0.9, 2.5):
            y = c + y1 * u
            got = orc.step(X, y[None], h)[0]
            want = c + a * math.tanh(a * y1 / (h * h)) * u
            assert np.max(np.abs(got - want)) <= 1e-12 * (1 + np.max(np.abs(want)))


def _polygon(k, r, c=(0.0, 0.0), phase=0.3):
    t = phase + 2 * np.pi * np.arange(k) / k
    return np.c_[c[0] + r * np.cos(t), c[1] + r * np.sin(t)]


@pytest.mark.parametrize("k", [3, 4, 6, 9])
@pytest.mark.parametrize("r_over_h", [0.3, 0.5, 1.2, 1.6, 2.5])
def test_polygon_centre_fixed_point_and_stability(k, r_over_h):
    h = 0.8
    c = (3.0, -1.0)
    X = _polygon(k, r_over_h * h, c)
    centre = np.array([c])
    got = orc.step(X, centre, h)[0]
    assert np.max(np.abs(got - centre[0])) <= 1e-12
    # local maximum iff r < sqrt(2) h: compare the density at the centre with
    # the density on a small circle around it
    eps = 1e-3 * h
    ring = centre + eps * np.c_[np.cos(np.linspace(0, 2 * np.pi, 17)),
                                np.sin(np.linspace(0, 2 * np.pi, 17))]
    f0 = orc.kde(X, centre, h)[0]
    fr = orc.kde(X, ring, h)
    if r_over_h < math.sqrt(2.0) - 0.05:
        assert np.all(fr < f0)
    elif r_over_h > math.sqrt(2.0) + 0.05:
        assert np.any(fr > f0)


@pytest.mark.parametrize("k", [3, 5, 8])
def test_polygon_vertices_converge_to_centre_when_small(k):
    h = 2.0
    c = (-4.0, 7.5)
    X = _polygon(k, 0.5 * h, c)
    Y, conv, _ = orc.trajectories(X, X, h, 1e-10 * h, 10000)
    assert np.all(conv > 0)
    assert np.max(np.abs(Y - np.array(c))) <= 1e-8 * h


def test_kde_single_point_closed_form():
    h = 1.3
    X = np.array([[0.5, -1.0, 2.0]])
    for dist in (0.0, 0.1, 1.0, 2.5, 7.0):
        y = X[0] + dist * np.array([0.6, 0.0, 0.8])
        got = orc.kde(X, y[None], h)[0]
        assert abs(got - math.exp(-dist * dist / (2 * h * h))) <= 1e-15


def test_mean_shift_vector_is_scaled_log_gradient():
    """m(y) - y = h^2 grad f(y) / f(y) for the Gaussian kernel (Eq. 6)."""
    rng = np.random.default_rng(3)
    X = rng.standard_normal((40, 3)) * 2.0
    h = 1.4
    for _ in range(5):
        y = rng.standard_normal(3)
        ms = orc.step(X, y[None], h)[0] - y
        g = np.zeros(3)
        e = 1e-5
        for k in range(3):
            dp = y.copy(); dp[k] += e
            dm = y.copy(); dm[k] -= e
            g[k] = (orc.kde(X, dp[None], h)[0] - orc.kde(X, dm[None], h)[0]) / (2 * e)
        want = h * h * g / orc.kde(X, y[None], h)[0]
        assert np.max(np.abs(ms - want)) <= 1e-7 * (1 + np.max(np.abs(want)))
