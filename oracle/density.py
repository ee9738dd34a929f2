"""FP64 oracle of adaptive density control (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this module; the
product path never touches it and it imports nothing from the product
package.

The paper trains with densification, pruning and opacity resets (the
hyperparameter table of its appendix gives the percent-dense fraction and
the reset / prune intervals) but does not state the procedure; this is the
adaptive density control of the 3D Gaussian splatting lineage it builds on,
restated:

  * statistics: per Gaussian, the sum over views in which it is visible of
    the norm of the loss gradient with respect to its projected centre in
    normalised device coordinates, (dL/du W/2, dL/dv H/2), and the number of
    such views;
  * densify: a Gaussian whose mean norm is at least grad_thresh is cloned
    (an identical copy is appended) when its largest scale is at most
    dense_scale, and split otherwise: it is replaced by two Gaussians with
    centres mu + R(q) (s * n_i), n_i ~ N(0, I3) drawn by the caller, scales
    s / 1.6, the other parameters copied;
  * prune: Gaussians (and their copies) with sigmoid(opacity logit) below
    min_opacity are dropped;
  * output order: surviving originals in index order, then clones in index
    order, then split children (two per parent, parent order);
  * per-Gaussian optimiser state follows survivors and is zero for new
    Gaussians; the statistics restart at zero;
  * opacity reset: logit <- min(logit, logit(max_opacity)).
"""
from __future__ import annotations

import numpy as np

SPLIT_N = 2
SPLIT_SCALE = 1.0 / (0.8 * SPLIT_N)   # s / 1.6


def screen_grad_stats(d_uv, visible, width: int, height: int, accum=None, count=None):
    """accum += |(du W/2, dv H/2)| and count += 1 for visible Gaussians."""
    d_uv = np.asarray(d_uv, np.float64)
    P = d_uv.shape[0]
    accum = np.zeros(P) if accum is None else np.array(accum, np.float64)
    count = np.zeros(P, np.int64) if count is None else np.array(count, np.int64)
    ndc = d_uv * np.array([width * 0.5, height * 0.5])
    nrm = np.sqrt(np.sum(ndc * ndc, axis=1))
    vis = np.asarray(visible, bool)
    accum[vis] += nrm[vis]
    count[vis] += 1
    return accum, count


def quat_to_rot(q):
    """Rotation matrices of (w, x, y, z) quaternions, normalised first."""
    q = np.asarray(q, np.float64)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    R = np.empty((q.shape[0], 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - w * z)
    R[:, 0, 2] = 2 * (x * z + w * y)
    R[:, 1, 0] = 2 * (x * y + w * z)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - w * x)
    R[:, 2, 0] = 2 * (x * z - w * y)
    R[:, 2, 1] = 2 * (y * z + w * x)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def decide(means, log_scales, quats, logits, accum, count, grad_thresh, dense_scale, min_opacity,
           precision: str = "f64"):
    """Per-Gaussian decision: 0 keep, 1 clone, 2 split, -1 prune.

    precision "f64" is the definition as stated.  "f32" takes the same
    decision in single precision, for comparison with a single-precision
    implementation: since sigmoid and exp are strictly increasing,
    sigmoid(x) < m is x < log(m / (1 - m)) and max exp(ls) > s is
    max ls > log(s); the two thresholds are formed in double and rounded to
    float32 once, and the mean statistic is one float32 division, so the
    decision involves no transcendental function of a per-Gaussian value."""
    if precision == "f32":
        f = np.float32
        cnt = np.asarray(count, np.int64)
        acc = np.asarray(accum, f)
        avg = np.where(cnt > 0, acc / np.maximum(cnt, 1).astype(f), f(0.0))
        m, ds = float(min_opacity), float(dense_scale)
        lmin = f(-np.inf) if m <= 0 else f(np.inf) if m >= 1 else f(np.log(m / (1.0 - m)))
        ldense = f(-np.inf) if ds <= 0 else f(np.log(ds))
        high = avg >= f(grad_thresh)
        big = np.max(np.asarray(log_scales, f), axis=1) > ldense
        d = np.where(high, np.where(big, 2, 1), 0)
        return np.where(np.asarray(logits, f) < lmin, -1, d)
    count = np.asarray(count)
    avg = np.where(count > 0, np.asarray(accum, np.float64) / np.maximum(count, 1), 0.0)
    big = np.max(np.exp(np.asarray(log_scales, np.float64)), axis=1) > dense_scale
    high = avg >= grad_thresh
    op = 1.0 / (1.0 + np.exp(-np.asarray(logits, np.float64)))
    d = np.where(high, np.where(big, 2, 1), 0)
    return np.where(op < min_opacity, -1, d)


def densify(params: dict, state: dict, accum, count, normals, grad_thresh, dense_scale, min_opacity,
            precision: str = "f64"):
    """params: means [P,3], log_scales [P,3], quats [P,4], opacity_logits [P]
    and any other per-Gaussian arrays (copied); state: per-Gaussian optimiser
    arrays (kept for survivors, zero for new ones); normals [P,2,3];
    precision: that of the decision (see decide).  Returns (new params, new
    state, decision)."""
    means = np.asarray(params["means"], np.float64)
    log_scales = np.asarray(params["log_scales"], np.float64)
    quats = np.asarray(params["quats"], np.float64)
    d = decide(means, log_scales, quats, params["opacity_logits"], accum, count, grad_thresh, dense_scale,
               min_opacity, precision)
    keep = np.flatnonzero((d == 0) | (d == 1))
    clone = np.flatnonzero(d == 1)
    split = np.flatnonzero(d == 2)
    R = quat_to_rot(quats[split]) if len(split) else np.zeros((0, 3, 3))
    s = np.exp(log_scales[split])
    kids_mu = []
    for i in range(SPLIT_N):
        off = np.einsum("pij,pj->pi", R, s * np.asarray(normals, np.float64)[split, i])
        kids_mu.append(means[split] + off)
    out = {}
    for k, v in params.items():
        v = np.asarray(v, np.float64)
        if k == "means":
            child = np.stack(kids_mu, axis=1).reshape((-1,) + v.shape[1:])
        elif k == "log_scales":
            child = np.repeat(v[split] + np.log(SPLIT_SCALE), SPLIT_N, axis=0)
        else:
            child = np.repeat(v[split], SPLIT_N, axis=0)
        out[k] = np.concatenate([v[keep], v[clone], child], axis=0)
    new_state = {}
    n_new = len(clone) + SPLIT_N * len(split)
    for k, v in state.items():
        v = np.asarray(v, np.float64)
        new_state[k] = np.concatenate([v[keep], np.zeros((n_new,) + v.shape[1:])], axis=0)
    return out, new_state, d


def reset_opacity(logits, max_opacity: float = 0.01):
    cap = np.log(max_opacity / (1.0 - max_opacity))
    return np.minimum(np.asarray(logits, np.float64), cap)
