"""FP64 oracle for Faster Mean-shift with the Euclidean metric.

TEST INFRASTRUCTURE ONLY: only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this module.  It shares no code with
the CUDA library (``paper_2112_13891_gb300``) and never imports it.

Paper: "GPU-accelerated Faster Mean Shift with euclidean distance metrics",
arXiv 2112.13891.  Everything runs in float64 on the host; the O(n) loops are
the plain C of ``ms_core.c`` (OpenMP only spreads independent seeds over
cores), the rest is numpy in the order the paper states the steps.

Readings of the paper used here (where it is silent or garbled):
  * the kernel is the Gaussian exp(-||y-x||^2/(2h^2)); its shadow is itself,
    so the update is the Gaussian-weighted mean over all points (Sec. II-B,
    the update of Alg. 2, the prose after Eq. 11; Eq. 11 itself is garbled).  The
    flat (uniform) kernel of Eq. 12-15 is the alternative (kernel="flat"): the
    update is the mean of the window ||x_i - y|| <= h and the density is the
    window count;
  * convergence: ||y_{t+1} - y_t|| <= tol (Alg. 1 and 2 name no test);
  * Seed Selection (Alg. 2, Sec. II-D): the seeds are the first N
    entries of a keyed pseudo-random permutation of [0, n) (a 6-round Feistel
    network over SplitMix64 round functions with cycle walking); N starts at
    128 and doubles while N < L*M, L = 8 (Sec. II-D);
  * Early Stopping (Sec. II-C): iteration stops once at least ceil(gamma*N)
    seeds have converged; seeds not converged by then are discarded.  With
    gamma = 1 (plain mean shift, Alg. 1) unconverged seeds are kept at their
    last position;
  * the prune of Alg. 1 and Alg. 2 is a greedy suppression in
    order of KDE score (descending, seed rank ascending): a seed is accepted
    unless an accepted mode lies closer than r_merge (default h);
  * each merged mode is then refined (more updates until the step is at most
    1e-5*h, at most 50 updates) and merged again with the same rule; modes are
    reported in canonical order (score descending, ties by coordinates);
  * every point is labelled by its nearest mode (the labelling of Alg. 2), ties to
    the lowest mode index; the margin is the gap to the second-nearest mode;
  * the cosine metric (the sibling method the paper cites, whose formulation
    it does not print; metric="cosine"): points are normalised to the unit
    sphere, the weight is exp((x.y - 1)/h^2) = exp(-||x - y||^2/(2h^2)) for
    unit x, y (the Gaussian kernel of the chord distance), and every update
    is projected back onto the sphere, y <- m(y)/||m(y)||; prune radius,
    tolerances and margins are chord distances; modes are unit vectors.

Parity status of each function is stated in its docstring ("pinned by ...").
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libms_oracle.so")
_lock = threading.Lock()
_lib = None

MASK64 = (1 << 64) - 1
GOLDEN_GAMMA = 0x9E3779B97F4A7C15
FEISTEL_ROUNDS = 6


# ----------------------------------------------------------------------------
# C core loader
# ----------------------------------------------------------------------------

def build(force: bool = False) -> str:
    """Compile ms_core.c with gcc (IEEE float64, no FMA contraction)."""
    src = os.path.join(_HERE, "ms_core.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-shared",
           "-fPIC", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _core():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            P = ctypes.c_void_p
            I64, I32, F64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
            lib.orc_kde.argtypes = [P, I64, I32, P, I64, F64, P]
            lib.orc_kde_flat.argtypes = [P, I64, I32, P, I64, F64, P]
            lib.orc_step.argtypes = [P, I64, I32, F64, P, I64, P]
            lib.orc_step_k.argtypes = [P, I64, I32, F64, P, I64, P, I32]
            lib.orc_trajectories.argtypes = [P, I64, I32, F64, F64, I32, P, I64, P, P]
            lib.orc_trajectories_k.argtypes = [P, I64, I32, F64, F64, I32, P, I64, P, P, I32]
            lib.orc_trajectories_m.argtypes = [P, I64, I32, F64, F64, I32, P, I64, P, P, I32,
                                               I32]
            lib.orc_label.argtypes = [P, I64, I32, P, I64, P, P]
            for f in (lib.orc_kde, lib.orc_kde_flat, lib.orc_step, lib.orc_step_k,
                      lib.orc_trajectories, lib.orc_trajectories_k, lib.orc_trajectories_m,
                      lib.orc_label):
                f.restype = None
            _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


# ----------------------------------------------------------------------------
# Eq. 1, Eq. 6 / 9 / 10: density and one mean-shift update
# ----------------------------------------------------------------------------

KERNELS = {"gaussian": 0, "flat": 1}


def kde(X, Y, h, kernel="gaussian"):
    """Density at each row y of Y (Eq. 1 without 1/(n h^d)).

    gaussian: sum_j exp(-||y - x_j||^2 / (2h^2)); flat (Eq. 12-13): the window
    count #{j : ||y - x_j|| <= h}.
    Pinned by: brute-force Python sums on tiny inputs; closed forms; the flat
    count against sklearn's window intensities.
    """
    X, Y = _f64(X), _f64(np.atleast_2d(Y))
    out = np.empty(Y.shape[0])
    fn = _core().orc_kde_flat if KERNELS[kernel] == 1 else _core().orc_kde
    fn(_ptr(X), X.shape[0], X.shape[1], _ptr(Y), Y.shape[0], float(h), _ptr(out))
    return out


def step(X, Y, h, kernel="gaussian"):
    """One mean-shift update for each row of Y.

    gaussian (Eq. 6, 9-10 with the Gaussian weight): m(y) = sum w x / sum w;
    flat (Eq. 14-15): the mean of the window S_h(y) (NaN when it is empty).
    Pinned by: the two-point closed form, symmetric-polygon fixed points,
    monotone KDE ascent, a gradient-of-KDE identity; the flat update against
    sklearn's flat mean shift and two-point closed forms.
    """
    X, Y = _f64(X), _f64(np.atleast_2d(Y))
    out = np.empty_like(Y)
    _core().orc_step_k(_ptr(X), X.shape[0], X.shape[1], float(h), _ptr(Y), Y.shape[0],
                       _ptr(out), KERNELS[kernel])
    return out


def trajectories(X, Y0, h, tol, max_iter, kernel="gaussian", sphere=False):
    """Independent trajectories y <- m(y) until ||step|| <= tol (the iteration loop of Alg. 1 and Alg. 2).

    Returns (Y_end, conv_iter, iters): conv_iter[i] is the 1-based update at
    which ||y_t - y_{t-1}|| <= tol first held, -1 if never within max_iter,
    -2 if an update was undefined (flat kernel, empty window; on the sphere,
    a mean at the origin).  sphere=True (cosine metric; X and Y0 on the unit
    sphere): every update is projected back, y <- m(y)/||m(y)||.
    Pinned by: closed forms (two points, polygons) and brute-force maxima; on
    the sphere, the circular closed form (update angle = atan2(sum w sin,
    sum w cos) with w = exp((cos(theta - phi) - 1)/h^2)), rotation
    equivariance and invariance to the points' norms.
    """
    X = _f64(X)
    Y = _f64(np.atleast_2d(Y0)).copy()
    m, d = Y.shape
    if d > 64:
        raise ValueError("oracle supports d <= 64")
    conv = np.empty(m, dtype=np.int32)
    iters = np.empty(m, dtype=np.int32)
    _core().orc_trajectories_m(_ptr(X), X.shape[0], d, float(h), float(tol), int(max_iter),
                               _ptr(Y), m, _ptr(conv), _ptr(iters), KERNELS[kernel],
                               1 if sphere else 0)
    return Y, conv, iters


METRICS = ("euclidean", "cosine")


def normalize_rows(X):
    """Rows scaled to unit length (the cosine metric's points); a zero row is
    an error (it has no direction)."""
    X = _f64(X)
    nrm = np.sqrt((X * X).sum(axis=1))
    if np.any(nrm == 0.0):
        raise ValueError("cosine metric: a point has zero norm")
    return X / nrm[:, None]


def label(X, modes, return_margins=True):
    """Nearest-mode labels and margins (the labelling of Alg. 2); ties to the lowest index.

    Pinned by: exhaustive argmin in Python on small inputs.
    """
    X, modes = _f64(X), _f64(np.atleast_2d(modes))
    n = X.shape[0]
    lab = np.empty(n, dtype=np.int32)
    mar = np.empty(n, dtype=np.float64)
    _core().orc_label(_ptr(X), n, X.shape[1], _ptr(modes), modes.shape[0], _ptr(lab), _ptr(mar))
    return (lab, mar) if return_margins else lab


# ----------------------------------------------------------------------------
# Seed Selection (Alg. 2): keyed permutation of [0, n)
# ----------------------------------------------------------------------------

def mix64(z: int) -> int:
    """SplitMix64 output function (Steele, Lea & Flood, OOPSLA 2014)."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def splitmix64(seed: int, i: int) -> int:
    """i-th output (0-based) of the SplitMix64 stream started at `seed`."""
    return mix64((seed + (i + 1) * GOLDEN_GAMMA) & MASK64)


def feistel_half_bits(n: int) -> int:
    """Half-width hb of the Feistel domain [0, 4^hb), the smallest with 4^hb >= n (hb >= 1)."""
    hb = 1
    while (1 << (2 * hb)) < n:
        hb += 1
    return hb


def feistel_encrypt(x: int, keys, hb: int) -> int:
    """Balanced Feistel network on 2*hb bits; round function mix64(k_r ^ R) truncated to hb bits."""
    mask = (1 << hb) - 1
    L, R = x >> hb, x & mask
    for k in keys:
        L, R = R, L ^ (mix64(k ^ R) & mask)
    return (L << hb) | R


def seed_permutation(n: int, rng_seed: int, start: int, stop: int):
    """Entries [start, stop) of the keyed permutation pi of [0, n).

    pi(i) cycle-walks the Feistel bijection of [0, 4^hb) until it lands in
    [0, n) (Black & Rogaway, "Ciphers with arbitrary finite domains", 2002),
    so pi is a bijection of [0, n).  Round keys are SplitMix64 outputs 0..5
    of the stream seeded with rng_seed.  Pinned by: brute-force bijection checks.
    """
    hb = feistel_half_bits(n)
    keys = [splitmix64(rng_seed & MASK64, r) for r in range(FEISTEL_ROUNDS)]
    out = np.empty(max(0, stop - start), dtype=np.int64)
    for r in range(start, stop):
        x = feistel_encrypt(r, keys, hb)
        while x >= n:
            x = feistel_encrypt(x, keys, hb)
        out[r - start] = x
    return out


# ----------------------------------------------------------------------------
# Sec. II-C: seed-coverage probability, Eq. 12
# ----------------------------------------------------------------------------

def eq12_coverage(n_min: int, M: int) -> float:
    """Eq. 12 exactly as printed: C(N_min-1, M-1) / C(N_min+M-1, M-1).

    This is the fraction of the C(N+M-1, M-1) occupancy vectors (N seeds into
    M clusters) with every cluster non-empty, i.e. the probability when all
    occupancy vectors are equally likely.  Pinned by: enumeration of compositions.
    """
    if n_min < M:
        return 0.0
    return math.comb(n_min - 1, M - 1) / math.comb(n_min + M - 1, M - 1)


def coverage_uniform_draws(N: int, M: int) -> float:
    """P(every one of M equal clusters receives >= 1 of N uniform draws), by inclusion-exclusion.

    Pinned by: Monte Carlo.  (Eq. 12 is not this probability; e.g. N=M=2 gives 1/3 vs 1/2.)
    """
    return float(sum((-1) ** k * math.comb(M, k) * (1.0 - k / M) ** N for k in range(M + 1)))


# ----------------------------------------------------------------------------
# Alg. 2 with Seed Selection and Early Stopping
# ----------------------------------------------------------------------------

@dataclass
class OracleResult:
    modes: np.ndarray             # [M, d] float64, canonical order
    scores: np.ndarray            # [M] KDE sums at the modes
    labels: np.ndarray            # [n] int32
    margins: np.ndarray           # [n] float64
    n_seeds: int                  # N at the end
    n_history: list = field(default_factory=list)
    t_star: list = field(default_factory=list)   # stop iteration of each round
    seeds: np.ndarray = None      # seed point indices, rank order
    conv_iter: np.ndarray = None  # per seed
    seed_pos: np.ndarray = None   # per seed final position
    kept: np.ndarray = None       # bool per seed (after the last round)
    premerge_modes: np.ndarray = None   # modes before refinement, merge order
    iters: int = 0


def early_stop(conv_iter: np.ndarray, gamma: float, max_iter: int):
    """Sec. II-C: stop iteration t* and the kept mask.

    t* is the ceil(gamma*N)-th smallest convergence iteration (max_iter if that
    many seeds never converge).  For gamma < 1, kept = converged by t*; for
    gamma = 1 every seed is kept (unconverged ones at their last iterate)
    except failed ones (conv_iter == -2: an undefined update).
    `gamma` is taken as the float32 value the library receives.
    """
    N = conv_iter.shape[0]
    g = float(np.float32(gamma))
    target = int(math.ceil(g * N))
    target = min(max(target, 1), N)
    c = np.where(conv_iter < 0, np.iinfo(np.int64).max, conv_iter.astype(np.int64))
    kth = np.sort(c)[target - 1]
    t_star = int(kth) if kth <= max_iter else int(max_iter)
    if g >= 1.0:
        kept = conv_iter != -2
        t_star = int(max_iter) if np.any(conv_iter == -1) else (
            int(np.max(conv_iter)) if np.any(conv_iter >= 0) else 0)
    else:
        kept = (conv_iter >= 0) & (conv_iter <= t_star)
    return t_star, kept


def merge(X, Y, rank, h, r_merge, kernel="gaussian"):
    """The prune of Alg. 1 and Alg. 2: greedy radius suppression.

    Candidates are visited in order of (density score descending, rank
    ascending); one is accepted unless an accepted mode lies at distance
    < r_merge.  Returns (accepted row indices into Y, scores of all rows).
    """
    Y = _f64(Y)
    if Y.shape[0] == 0:
        return np.zeros(0, dtype=np.int64), np.zeros(0)
    score = kde(X, Y, h, kernel)
    order = np.lexsort((np.asarray(rank), -score))
    acc = []
    for i in order:
        if acc:
            dist = np.sqrt(((Y[acc] - Y[i]) ** 2).sum(axis=1))
            if np.any(dist < r_merge):
                continue
        acc.append(int(i))
    return np.asarray(acc, dtype=np.int64), score


def canonical_order(modes, scores):
    """Score descending, ties by lexicographic coordinates."""
    keys = [modes[:, k] for k in range(modes.shape[1] - 1, -1, -1)] + [-scores]
    return np.lexsort(keys)


def cluster(X32, h, tol, max_iter, *, all_seeds=False, n_initial=128, L=8.0, gamma=0.95,
            merge_radius=0.0, rng_seed=0, seed_indices=None, refine=True,
            refine_tol=1e-5, refine_max_iter=50, kernel="gaussian", metric="euclidean"):
    """Faster Mean-shift (Alg. 2, Sec. II-C/D) or plain mean shift (Alg. 1, all_seeds=True).

    kernel: "gaussian" (the reading used throughout) or "flat" (Eq. 12-15: the
    window mean, density = window count).  metric: "euclidean" or "cosine"
    (points normalised, updates projected onto the unit sphere; see the
    module notes).

    Steps, in the paper's order: select N seeds; iterate every seed to
    convergence (trajectories are independent, so this is done seed by seed);
    Early Stopping decides t* and the kept seeds; prune; if N < L*M and N < n
    double N and repeat for the new seeds; refine and re-merge; label.
    """
    if metric not in METRICS:
        raise ValueError(f"metric must be one of {METRICS}")
    sphere = metric == "cosine"
    X = normalize_rows(X32) if sphere else _f64(X32)
    n, d = X.shape
    r_merge = float(merge_radius) if merge_radius and merge_radius > 0 else float(h)
    if all_seeds:
        gamma = 1.0
    # --- Seed Selection ---
    if all_seeds:
        seeds = np.arange(n, dtype=np.int64)
        N = n
    elif seed_indices is not None:
        seeds = np.asarray(seed_indices, dtype=np.int64)
        N = seeds.shape[0]
    else:
        N = min(int(n_initial), n)
        seeds = seed_permutation(n, rng_seed, 0, N)
    pos, conv, _ = trajectories(X, X[seeds], h, tol, max_iter, kernel, sphere)
    history, tstars = [N], []
    while True:
        t_star, kept = early_stop(conv, gamma, max_iter)
        tstars.append(t_star)
        kidx = np.nonzero(kept)[0]
        acc, _ = merge(X, pos[kidx], kidx, h, r_merge, kernel)
        M = acc.shape[0]
        if all_seeds or seed_indices is not None or not (N < L * M and N < n):
            break
        N_new = min(2 * N, n)
        new = seed_permutation(n, rng_seed, N, N_new)
        p2, c2, _ = trajectories(X, X[new], h, tol, max_iter, kernel, sphere)
        seeds = np.concatenate([seeds, new])
        pos = np.concatenate([pos, p2])
        conv = np.concatenate([conv, c2])
        N = N_new
        history.append(N)
    modes0 = pos[kidx[acc]]
    if refine and M > 0:
        ref, _, _ = trajectories(X, modes0, h, refine_tol * h, refine_max_iter, kernel, sphere)
        acc2, sc2 = merge(X, ref, np.arange(M), h, r_merge, kernel)
        modes, scores = ref[acc2], sc2[acc2]
    else:
        modes = modes0
        scores = kde(X, modes, h, kernel) if M > 0 else np.zeros(0)
    o = canonical_order(modes, scores) if modes.shape[0] else np.zeros(0, dtype=np.int64)
    modes, scores = modes[o], scores[o]
    labels, margins = label(X, modes) if modes.shape[0] else (
        np.full(n, -1, np.int32), np.full(n, np.inf))
    return OracleResult(modes=modes, scores=scores, labels=labels, margins=margins, n_seeds=N,
                        n_history=history, t_star=tstars, seeds=seeds, conv_iter=conv,
                        seed_pos=pos, kept=kept, premerge_modes=modes0, iters=max(tstars))


def next_frame_seed_count(N, M, H=32.0):
    """Seed count carried to the next frame (Sec. II-D, video use): when the
    frame ended with N seeds and M modes and N > H*M, the next frame starts
    with N - M seeds; otherwise with N."""
    return int(N - M) if N > H * M else int(N)


def cluster_frames(frames, h, tol, max_iter, *, n_initial=128, L=8.0, H=32.0, **kw):
    """Faster Mean-shift over a sequence of frames (Sec. II-D): each frame is
    clustered by `cluster` starting from the seed count carried over from the
    previous frame (doubling inside a frame while N < L*M as usual); the count
    carried on is reduced by M when N > H*M.  Returns (per-frame results,
    starting seed counts)."""
    out, starts = [], []
    N = int(n_initial)
    for X in frames:
        starts.append(N)
        r = cluster(X, h, tol, max_iter, n_initial=N, L=L, **kw)
        out.append(r)
        N = max(1, next_frame_seed_count(r.n_seeds, r.modes.shape[0], H))
    return out, starts


# ----------------------------------------------------------------------------
# Unrolled steps and their adjoint (spec pattern; no paper counterpart)
# ----------------------------------------------------------------------------

def unrolled_forward(X, Y0, h, T):
    """T Gaussian mean-shift updates of every row of Y0 against the points X (dense FP64).

    Returns the list [Y_0, ..., Y_T].
    """
    X, Y = _f64(X), _f64(Y0)
    out = [Y.copy()]
    for _ in range(T):
        D = ((Y[:, None, :] - X[None, :, :]) ** 2).sum(-1)
        logw = -(D - D.min(axis=1, keepdims=True)) / (2.0 * h * h)
        W = np.exp(logw)
        P = W / W.sum(axis=1, keepdims=True)
        Y = P @ X
        out.append(Y.copy())
    return out


def unrolled_backward(X, Y0, h, T, G):
    """Adjoint of `unrolled_forward` for an upstream gradient G = dL/dY_T.

    With p_ij = w_ij / sum_j w_ij, mu_i = sum_j p_ij x_j, g_i = dL/dmu_i and
    a_ij = g_i . (x_j - mu_i), one update contributes
      dL/dy_i  = (1/h^2) sum_j p_ij a_ij (x_j - mu_i)
      dL/dx_j += p_ij [g_i - a_ij (x_j - y_i) / h^2]
      dL/dh   += (1/h^3) sum_ij p_ij a_ij ||y_i - x_j||^2
    (derived by differentiating log w_ij = -||y_i - x_j||^2/(2h^2)).
    Returns (dX, dY0, dh).  Pinned by: central finite differences and torch
    autograd of the dense forward, in float64.
    """
    X = _f64(X)
    Ys = unrolled_forward(X, Y0, h, T)
    g = _f64(G).copy()
    dX = np.zeros_like(X)
    dh = 0.0
    h2 = h * h
    for t in range(T - 1, -1, -1):
        Y = Ys[t]
        D = ((Y[:, None, :] - X[None, :, :]) ** 2).sum(-1)
        W = np.exp(-(D - D.min(axis=1, keepdims=True)) / (2.0 * h2))
        P = W / W.sum(axis=1, keepdims=True)
        mu = P @ X
        A = g @ X.T - (g * mu).sum(axis=1, keepdims=True)      # a_ij
        PA = P * A
        dY = (PA @ X - PA.sum(axis=1, keepdims=True) * mu) / h2
        dX += P.T @ g - (PA.sum(axis=0)[:, None] * X - PA.T @ Y) / h2
        dh += float((PA * D).sum()) / (h2 * h)
        g = dY
    return dX, g, dh
