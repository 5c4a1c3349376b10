"""Seeded synthetic point sets for Gaussian mean-shift clustering.

This module only draws inputs.  It holds none of the clustering arithmetic, so
both the FP64 oracle and the CUDA path can take their inputs from here without
sharing any of the method's code.

All draws use numpy's PCG64 (`numpy.random.default_rng(seed)`).  Points are
returned as C-contiguous float32 arrays of shape [n, d] (the library's input
type); the oracle widens them to float64 itself.

Workloads (the paper's data come from sklearn's blob generator, which is
stood in for by the recipes below; Sec. III-B, Table I):

* ``plain_2d``      -- n=2,000, d=2, 5 equal blobs, centres U[0,100]^2, sigma=2,
                        h=4, every point a seed, tol=1e-3*h, 300 iterations.
* ``paper_3d``      -- n=200,000, d=3, 20 blobs (centres U[0,200]^3,
                        sigma ~ U[1,3], sizes Dirichlet(2,...,2) proportions)
                        plus 2% uniform background noise, h=5.  This is the
                        scaled stand-in for Table I's 200K-point case.
* ``embedding_32d`` -- n=65,536, d=32, 64 blobs of 1,024 points with centres
                        10*u (u uniform on the unit sphere), sigma=0.5, h=1.
* ``batched_16d``   -- 256 sets, sizes log-uniform in [1K, 50K], d=16, 4..40
                        blobs each, centres U[0,50]^16, sigma=1, h=2.5.
* ``unrolled_16d``  -- 8 sets of 16,384 points, d=16, 32 blobs, h=2.
* ``toy_*``         -- the six 1,500-point toy distributions of Fig. 3
                        (Sec. III-B), written from their one-line descriptions.
* ``pixels_rgb``    -- synthetic RGB pixel values (the Fig. 1 image workload).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "Workload", "blobs", "plain_2d", "paper_3d", "embedding_32d", "batched_16d",
    "unrolled_16d", "toy_blobs", "toy_large_variance", "toy_varied_variance",
    "toy_uniform_square", "toy_noisy_circles", "toy_anisotropic", "pixels_rgb",
    "separated_blobs", "WORKLOADS",
]


class Workload(dict):
    """A dict with attribute access: X, h, tol, max_iter, all_seeds, ... ."""

    __getattr__ = dict.__getitem__


def _as_points(a: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


def blobs(rng: np.random.Generator, centers: np.ndarray, sigmas, sizes,
          shuffle: bool = True):
    """Isotropic Gaussian blobs; returns (points float64, planted label)."""
    centers = np.asarray(centers, dtype=np.float64)
    k, d = centers.shape
    sigmas = np.broadcast_to(np.asarray(sigmas, dtype=np.float64), (k,))
    parts, labels = [], []
    for i in range(k):
        parts.append(centers[i] + sigmas[i] * rng.standard_normal((int(sizes[i]), d)))
        labels.append(np.full(int(sizes[i]), i, dtype=np.int32))
    X = np.concatenate(parts, axis=0)
    lab = np.concatenate(labels)
    if shuffle:
        p = rng.permutation(X.shape[0])
        X, lab = X[p], lab[p]
    return X, lab


def plain_2d(seed: int = 0, n: int = 2000) -> Workload:
    """n points in 2-D from 5 equal blobs; plain (all-seeds) mean shift."""
    rng = np.random.default_rng(seed)
    k = 5
    centers = rng.uniform(0.0, 100.0, size=(k, 2))
    sizes = [n // k + (1 if i < n % k else 0) for i in range(k)]
    X, lab = blobs(rng, centers, 2.0, sizes)
    h = 4.0
    return Workload(name="plain_2d", X=_as_points(X), planted=lab, centers=centers,
                    h=h, tol=1e-3 * h, max_iter=300, all_seeds=True, gamma=1.0)


def paper_3d(seed: int = 0, n: int = 200_000, noise_frac: float = 0.02) -> Workload:
    """Paper-scale 3-D problem: 20 Dirichlet-sized blobs plus uniform noise."""
    rng = np.random.default_rng(seed)
    k, d, box = 20, 3, 200.0
    n_noise = int(round(noise_frac * n))
    n_blob = n - n_noise
    centers = rng.uniform(0.0, box, size=(k, d))
    sigmas = rng.uniform(1.0, 3.0, size=k)
    prop = rng.dirichlet(np.full(k, 2.0))
    sizes = np.floor(prop * n_blob).astype(np.int64)
    sizes[int(np.argmax(sizes))] += n_blob - int(sizes.sum())
    Xb, lab = blobs(rng, centers, sigmas, sizes, shuffle=False)
    Xn = rng.uniform(0.0, box, size=(n_noise, d))
    X = np.concatenate([Xb, Xn], axis=0)
    lab = np.concatenate([lab, np.full(n_noise, -1, dtype=np.int32)])
    p = rng.permutation(n)
    h = 5.0
    return Workload(name="paper_3d", X=_as_points(X[p]), planted=lab[p], centers=centers,
                    sigmas=sigmas, h=h, tol=1e-3 * h, max_iter=300, all_seeds=False,
                    gamma=0.95)


def embedding_32d(seed: int = 0, per_cluster: int = 1024, k: int = 64, d: int = 32) -> Workload:
    """Embedding-style clusters: centres 10*u with u uniform on S^{d-1}."""
    rng = np.random.default_rng(seed)
    u = rng.standard_normal((k, d))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    centers = 10.0 * u
    X, lab = blobs(rng, centers, 0.5, [per_cluster] * k)
    h = 1.0
    return Workload(name="embedding_32d", X=_as_points(X), planted=lab, centers=centers,
                    h=h, tol=1e-3 * h, max_iter=300, all_seeds=False, gamma=0.95)


def batched_16d(seed: int = 0, n_sets: int = 256, lo: int = 1000, hi: int = 50_000,
                d: int = 16):
    """Many independent point sets of uneven size (one Workload per set)."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(n_sets):
        n_b = int(math.floor(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        k_b = int(rng.integers(4, 41))
        centers = rng.uniform(0.0, 50.0, size=(k_b, d))
        sizes = np.full(k_b, n_b // k_b, dtype=np.int64)
        sizes[: n_b % k_b] += 1
        X, lab = blobs(rng, centers, 1.0, sizes)
        out.append(Workload(name=f"batched_16d[{b}]", X=_as_points(X), planted=lab,
                            centers=centers, h=2.5, tol=2.5e-3, max_iter=300,
                            all_seeds=False, gamma=0.95))
    return out


def unrolled_16d(seed: int = 0, n_sets: int = 8, n: int = 16_384, d: int = 16, k: int = 32):
    """Sets for the differentiable unrolled steps (all points are seeds)."""
    rng = np.random.default_rng(seed)
    Xs = []
    for _ in range(n_sets):
        centers = rng.uniform(0.0, 50.0, size=(k, d))
        sizes = np.full(k, n // k, dtype=np.int64)
        sizes[: n % k] += 1
        X, _ = blobs(rng, centers, 1.0, sizes)
        Xs.append(X)
    return Workload(name="unrolled_16d", X=_as_points(np.stack(Xs)), h=2.0, T=20, k_ckpt=5)


def separated_blobs(seed: int, k: int, d: int, per: int, sigma: float, h: float,
                    box: float = None) -> Workload:
    """Blobs whose centres are rejection-sampled at least 6*sqrt(sigma^2+h^2) apart."""
    rng = np.random.default_rng(seed)
    sep = 6.0 * math.sqrt(sigma * sigma + h * h)
    if box is None:
        box = sep * 2.0 * max(2.0, k ** (1.0 / d))
    centers = []
    tries = 0
    while len(centers) < k:
        c = rng.uniform(0.0, box, size=d)
        tries += 1
        if tries > 100000:
            raise RuntimeError("could not place separated centres")
        if all(np.linalg.norm(c - e) >= sep for e in centers):
            centers.append(c)
    centers = np.array(centers)
    X, lab = blobs(rng, centers, sigma, [per] * k)
    return Workload(name=f"separated_{k}x{d}", X=_as_points(X), planted=lab, centers=centers,
                    h=h, tol=1e-3 * h, max_iter=300, all_seeds=False, gamma=0.95)


# --- Fig. 3 toy distributions (1,500 points each), from their descriptions ---

def toy_blobs(seed: int = 0, n: int = 1500) -> Workload:
    rng = np.random.default_rng(seed)
    centers = rng.uniform(-10.0, 10.0, size=(3, 2))
    X, lab = blobs(rng, centers, 1.0, [n // 3] * 3)
    return Workload(name="toy_blobs", X=_as_points(X), planted=lab, centers=centers)


def toy_large_variance(seed: int = 1, n: int = 1500) -> Workload:
    rng = np.random.default_rng(seed)
    centers = rng.uniform(-10.0, 10.0, size=(3, 2))
    X, lab = blobs(rng, centers, 2.5, [n // 3] * 3)
    return Workload(name="toy_large_variance", X=_as_points(X), planted=lab, centers=centers)


def toy_varied_variance(seed: int = 2, n: int = 1500) -> Workload:
    rng = np.random.default_rng(seed)
    centers = rng.uniform(-10.0, 10.0, size=(3, 2))
    X, lab = blobs(rng, centers, [1.0, 2.5, 0.5], [n // 3] * 3)
    return Workload(name="toy_varied_variance", X=_as_points(X), planted=lab, centers=centers)


def toy_uniform_square(seed: int = 3, n: int = 1500) -> Workload:
    rng = np.random.default_rng(seed)
    X = rng.uniform(0.0, 1.0, size=(n, 2))
    return Workload(name="toy_uniform_square", X=_as_points(X), planted=np.zeros(n, np.int32))


def toy_noisy_circles(seed: int = 4, n: int = 1500, factor: float = 0.5,
                      noise: float = 0.05) -> Workload:
    rng = np.random.default_rng(seed)
    n_out = n // 2
    n_in = n - n_out
    t_out = rng.uniform(0.0, 2 * np.pi, n_out)
    t_in = rng.uniform(0.0, 2 * np.pi, n_in)
    X = np.concatenate([np.c_[np.cos(t_out), np.sin(t_out)],
                        factor * np.c_[np.cos(t_in), np.sin(t_in)]])
    X += noise * rng.standard_normal(X.shape)
    lab = np.r_[np.zeros(n_out, np.int32), np.ones(n_in, np.int32)]
    return Workload(name="toy_noisy_circles", X=_as_points(X), planted=lab)


def toy_anisotropic(seed: int = 5, n: int = 1500) -> Workload:
    rng = np.random.default_rng(seed)
    centers = rng.uniform(-10.0, 10.0, size=(3, 2))
    X, lab = blobs(rng, centers, 1.0, [n // 3] * 3)
    A = np.array([[0.6, -0.6], [-0.4, 0.8]])
    return Workload(name="toy_anisotropic", X=_as_points(X @ A), planted=lab,
                    centers=centers @ A)


def pixels_rgb(seed: int = 0, height: int = 512, width: int = 512, k: int = 12,
               sigma: float = 6.0) -> Workload:
    """Synthetic RGB pixel values in [0, 255]^3 drawn around k palette colours."""
    rng = np.random.default_rng(seed)
    palette = rng.uniform(20.0, 235.0, size=(k, 3))
    n = height * width
    prop = rng.dirichlet(np.full(k, 2.0))
    sizes = np.floor(prop * n).astype(np.int64)
    sizes[int(np.argmax(sizes))] += n - int(sizes.sum())
    X, lab = blobs(rng, palette, sigma, sizes)
    X = np.clip(X, 0.0, 255.0)
    return Workload(name=f"pixels_rgb_{height}x{width}", X=_as_points(X), planted=lab,
                    centers=palette, h=12.0, tol=12e-3, max_iter=300, all_seeds=False,
                    gamma=0.95)


def drifting_frames(seed: int = 0, frames: int = 8, n: int = 65_536, k: int = 10, d: int = 3,
                    sigma: float = 2.0, box: float = 200.0, drift: float = 0.5):
    """A synthetic frame sequence: k Gaussian blobs whose centres move by a
    small random step (|step| ~ drift) from frame to frame; each frame draws n
    fresh points (equal blob proportions).  Stands in for the paper's video
    tracking use, for which it gives no data."""
    rng = np.random.default_rng(seed)
    centers = rng.uniform(0.0, box, size=(k, d))
    out = []
    sizes = np.full(k, n // k, dtype=np.int64)
    sizes[: n % k] += 1
    for _ in range(frames):
        X, lab = blobs(rng, centers, sigma, sizes)
        out.append(_as_points(X))
        centers = centers + rng.standard_normal((k, d)) * drift
    return out


WORKLOADS = {
    "plain_2d": plain_2d,
    "paper_3d": paper_3d,
    "embedding_32d": embedding_32d,
}


def directional_blobs(seed: int, k: int, d: int, per: int, spread: float, h: float,
                      min_angle: float = 0.9, radius=(0.5, 20.0)) -> Workload:
    """Unit directions (pairwise angles >= min_angle radians, rejection-sampled)
    with Gaussian spread `spread` around each, then every point scaled by a
    random positive length in `radius` (the cosine metric ignores it): the
    embedding-style workload of the cosine-metric variant."""
    rng = np.random.default_rng(seed)
    dirs = []
    tries = 0
    while len(dirs) < k:
        u = rng.standard_normal(d)
        u /= np.linalg.norm(u)
        tries += 1
        if tries > 100000:
            raise RuntimeError("could not place separated directions")
        if all(math.acos(max(-1.0, min(1.0, float(u @ e)))) >= min_angle for e in dirs):
            dirs.append(u)
    dirs = np.array(dirs)
    lab = np.repeat(np.arange(k), per)
    P = dirs[lab] + spread * rng.standard_normal((k * per, d))
    P /= np.linalg.norm(P, axis=1, keepdims=True)
    P *= rng.uniform(radius[0], radius[1], (k * per, 1))
    perm = rng.permutation(k * per)
    return Workload(name=f"directional_{k}x{d}", X=_as_points(P[perm]), planted=lab[perm],
                    centers=dirs, h=h, tol=1e-3 * h, max_iter=300, all_seeds=False, gamma=0.95)
