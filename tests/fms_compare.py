"""Helpers that compare a GPU clustering with the FP64 oracle.

Modes are matched one-to-one (Hungarian assignment on distances); labels are
compared after mapping GPU mode indices to oracle indices, excluding points
whose oracle margin (second-nearest minus nearest distance) is below a
threshold -- their nearest mode is decided by rounding.  The mode ORDER is
part of the output contract (canonical order: density score descending, ties
by coordinates), so the matched GPU order must equal the oracle's, except that
two modes whose oracle scores agree within a relative score tolerance may
appear in either order (their GPU scores are FP32 sums at positions within
the mode tolerance, so such a near-tie can be decided either way).
"""
import numpy as np
from scipy.optimize import linear_sum_assignment


def match_modes(gpu_modes, ref_modes):
    g = np.asarray(gpu_modes, dtype=np.float64)
    r = np.asarray(ref_modes, dtype=np.float64)
    if g.shape != r.shape:
        raise AssertionError(f"mode count differs: gpu {g.shape[0]} vs oracle {r.shape[0]}")
    D = np.sqrt(((g[:, None, :] - r[None, :, :]) ** 2).sum(-1))
    gi, ri = linear_sum_assignment(D)
    perm = np.empty(g.shape[0], dtype=np.int64)
    perm[gi] = ri
    return perm, float(D[gi, ri].max()) if len(gi) else 0.0


def order_violations(perm, ref_scores, score_rtol=1e-4):
    """Pairs of GPU positions i < j whose matched oracle modes come in the
    opposite canonical order although their oracle scores differ by more than
    score_rtol (relative to the larger score)."""
    p = np.asarray(perm)
    s = np.asarray(ref_scores, dtype=np.float64)[p]
    i, j = np.triu_indices(p.shape[0], k=1)
    inverted = p[i] > p[j]
    gap = np.abs(s[i] - s[j]) > score_rtol * np.maximum(np.abs(s[i]), np.abs(s[j]))
    return int((inverted & gap).sum())


def compare_clustering(gpu_modes, gpu_labels, ref, h, mode_tol=1e-3, margin_tol=1e-2,
                       score_rtol=1e-4):
    """Returns a dict of errors; raises on a mode-count mismatch.  mode_ok
    requires every matched mode within mode_tol*h and the canonical order."""
    perm, err = match_modes(gpu_modes, ref.modes)
    viol = order_violations(perm, ref.scores, score_rtol)
    lab = np.asarray(gpu_labels).astype(np.int64)
    mapped = np.where(lab >= 0, perm[np.clip(lab, 0, None)], -1)
    keep = ref.margins >= margin_tol * h
    mism = int((mapped[keep] != ref.labels[keep]).sum())
    return {"max_mode_err": err, "max_mode_err_over_h": err / h,
            "label_mismatch": mism, "low_margin_points": int((~keep).sum()),
            "order_violations": viol,
            "mode_ok": err <= mode_tol * h and viol == 0}
