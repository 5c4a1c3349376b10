"""Pins of the oracle's cosine-metric variant (metric="cosine").

The cosine variant normalises the points to the unit sphere, weighs point x
for seed y by exp((x.y - 1)/h^2) (the Gaussian kernel of the chord distance
between unit vectors) and projects every update back onto the sphere.  The
pins below come from outside the oracle's own code path: the circular closed
form on the unit circle (computed with angles), a fixed point forced by
symmetry, and the invariances the metric implies (the points' norms do not
matter; rotations commute with the whole method).
"""
import math

import numpy as np
import pytest

import oracle as orc


def _circle_step(theta, phi, h):
    # update angle on the unit circle: the direction of sum_j w_j (cos, sin)
    # with w_j = exp((cos(theta_j - phi) - 1) / h^2)
    w = np.exp((np.cos(theta - phi) - 1.0) / (h * h))
    return math.atan2(float((w * np.sin(theta)).sum()), float((w * np.cos(theta)).sum()))


@pytest.mark.parametrize("h", [0.3, 0.7, 1.5])
def test_one_update_on_the_circle_matches_the_angle_form(h):
    rng = np.random.default_rng(3)
    theta = np.concatenate([rng.normal(0.4, 0.2, 60), rng.normal(2.5, 0.3, 40)])
    X = np.stack([np.cos(theta), np.sin(theta)], axis=1)
    for phi in (0.1, 1.3, 2.9, -2.0):
        y0 = np.array([[math.cos(phi), math.sin(phi)]])
        y1, _, it = orc.trajectories(X, y0, h, 0.0, 1, sphere=True)
        assert it[0] == 1
        ang = _circle_step(theta, phi, h)
        assert np.allclose(y1[0], [math.cos(ang), math.sin(ang)], atol=1e-12)
        assert abs(np.linalg.norm(y1[0]) - 1.0) < 1e-14


def test_symmetric_ring_fixes_the_pole():
    # a ring of points at equal polar angle around the north pole, plus the
    # pole itself: by symmetry the pole is a fixed point of the update
    k, alpha = 12, 0.6
    az = 2 * np.pi * np.arange(k) / k
    ring = np.stack([np.sin(alpha) * np.cos(az), np.sin(alpha) * np.sin(az),
                     np.full(k, np.cos(alpha))], axis=1)
    X = np.vstack([ring, [[0.0, 0.0, 1.0]]])
    y, conv, _ = orc.trajectories(X, np.array([[0.0, 0.0, 1.0]]), 0.5, 1e-12, 5, sphere=True)
    assert conv[0] == 1
    assert np.allclose(y[0], [0.0, 0.0, 1.0], atol=1e-14)


def _directional_blobs(seed, k=4, per=150, d=3, kappa_sigma=0.08):
    rng = np.random.default_rng(seed)
    C = rng.standard_normal((k, d))
    C /= np.linalg.norm(C, axis=1, keepdims=True)
    P = np.repeat(C, per, axis=0) + kappa_sigma * rng.standard_normal((k * per, d))
    P /= np.linalg.norm(P, axis=1, keepdims=True)
    return P[rng.permutation(k * per)], C


def test_modes_are_the_cluster_directions():
    X, C = _directional_blobs(5)
    r = orc.cluster(X, 0.25, 1e-3 * 0.25, 300, metric="cosine", gamma=0.95, rng_seed=1)
    assert r.modes.shape[0] == C.shape[0]
    assert np.allclose(np.linalg.norm(r.modes, axis=1), 1.0, atol=1e-12)
    # each true direction has a mode within a few spreads / sqrt(per)
    for c in C:
        assert np.min(np.linalg.norm(r.modes - c, axis=1)) < 0.03


def test_invariant_to_the_points_norms():
    X, _ = _directional_blobs(6)
    rng = np.random.default_rng(7)
    Xs = X * rng.uniform(0.1, 50.0, (X.shape[0], 1))
    a = orc.cluster(X, 0.3, 3e-4, 300, metric="cosine", rng_seed=2)
    b = orc.cluster(Xs, 0.3, 3e-4, 300, metric="cosine", rng_seed=2)
    assert np.array_equal(a.labels, b.labels)
    assert np.allclose(a.modes, b.modes, atol=1e-9)


def test_rotation_equivariant():
    X, _ = _directional_blobs(8, d=4)
    rng = np.random.default_rng(9)
    Q, _ = np.linalg.qr(rng.standard_normal((4, 4)))
    a = orc.cluster(X, 0.3, 3e-4, 300, metric="cosine", rng_seed=4)
    b = orc.cluster(X @ Q, 0.3, 3e-4, 300, metric="cosine", rng_seed=4)
    assert np.array_equal(a.labels, b.labels)
    assert np.allclose(a.modes @ Q, b.modes, atol=1e-9)


def test_cosine_differs_from_euclidean_on_unnormalised_data():
    # two clusters along the same direction at different radii: one direction
    # for the cosine metric, two locations for the Euclidean one
    rng = np.random.default_rng(10)
    u = np.array([1.0, 2.0, 2.0]) / 3.0
    X = np.vstack([u * 1.0 + 0.01 * rng.standard_normal((100, 3)),
                   u * 10.0 + 0.01 * rng.standard_normal((100, 3))])
    e = orc.cluster(X, 0.2, 2e-4, 300, rng_seed=0)
    c = orc.cluster(X, 0.2, 2e-4, 300, metric="cosine", rng_seed=0)
    assert e.modes.shape[0] == 2
    assert c.modes.shape[0] == 1
    assert np.allclose(c.modes[0], u, atol=2e-3)


def test_zero_norm_point_rejected():
    X = np.array([[1.0, 0.0], [0.0, 0.0]])
    with pytest.raises(ValueError):
        orc.cluster(X, 0.5, 1e-3, 10, metric="cosine")
