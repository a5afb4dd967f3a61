"""Plain FP64 CPU oracle of the adaptive density control of MB3DGS.

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` (through the ``oracle``
package), never by the product path.

What it computes follows Sec. 3.4 "Training and Densification" and App. D
"Adaptive Density Control" of "Moment-Based 3D Gaussian Splatting", step by
step in numpy:

* view-independent opacity (App. D "View-Independent Opacity"): the opacity
  of a particle seen along its shortest axis through its centre, with both
  erf terms of its optical depth at their bound 2:
  o = 1 - exp(-sqrt(2 pi) w min(s));
* initial peak density from an opacity (App. D, same paragraph, with the
  average instead of the minimal scale): w = -log(1 - o) / (sqrt(2 pi) avg(s));
* the densification criterion (App. D "Cloning and Splitting", after AbsGS):
  per step, the absolute values of the components of dL/d(mean) are summed
  per particle; the criterion is the norm of that sum over the number of
  steps the particle was visible, compared with 1e-4;
* clone (small particles): the particle and its copy each carry w / 2;
* split (large particles): two particles at mean +/- delta s_max v, v the
  axis of the largest scale s_max, that scale multiplied by gamma (in
  float32, since the pruning test reads it), everything else copied
  (gamma = 0.6385502815, delta = 0.6128153091, App. D);
* pruning of every resulting particle whose view-independent opacity is
  below the threshold or whose largest scale exceeds big_world x extent
  (the 3DGS rules this ADC keeps).

Thresholds that decide an integer (keep / clone / split / prune) are
evaluated in float32, in the same operation order as the CUDA path: the
opacity test as sqrt(2 pi) w s_min < -log(1 - o_min) (float32 products), the
gradient test as sqrt(ax^2 + ay^2 + az^2) / n >= threshold (float32, no
fused multiply-add).  Output order: input order, each input's outputs
contiguous (clone: original then copy; split: minus then plus offset).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SQRT_2PI = math.sqrt(2.0 * math.pi)
SPLIT_GAMMA = 0.6385502815246582     # App. D, printed
SPLIT_DELTA = 0.6128153090966912     # App. D, printed (in units of the split axis' scale)


@dataclass
class ADCConfig:
    grad_threshold: float = 1e-4      # App. D: 3DGS's 2e-4 reduced to 1e-4
    prune_opacity: float = 0.005      # 3DGS minimum opacity (the ADC the paper keeps)
    percent_dense: float = 0.01       # 3DGS: clone when max(s) <= percent_dense x extent, else split
    scene_extent: float = 1.0
    big_world: float = 0.1            # 3DGS: prune when max(s) > big_world x extent (0: off)
    split_gamma: float = SPLIT_GAMMA
    split_delta: float = SPLIT_DELTA


def view_independent_opacity(weights, scales):
    """o = 1 - exp(-sqrt(2 pi) w min(s_x, s_y, s_z)) (App. D)."""
    w = np.asarray(weights, np.float64)
    s = np.asarray(scales, np.float64)
    return 1.0 - np.exp(-SQRT_2PI * w * s.min(-1))


def init_weights(opacity, scales):
    """Peak density giving opacity o along an axis of the average scale:
    w = -log(1 - o) / (sqrt(2 pi) avg(s)) (App. D)."""
    o = np.asarray(opacity, np.float64)
    s = np.asarray(scales, np.float64)
    return -np.log1p(-o) / (SQRT_2PI * s.mean(-1))


def accumulate_grad_stats(d_means, visible, abs_sum, count):
    """One step of the densification statistics: abs_sum[i] += |dL/dmean_i|
    (component-wise, float32) and count[i] += 1 for the visible particles.
    visible None: a particle is visible when a component of its gradient is
    non-zero.  Updates abs_sum (P, 3) float32 and count (P,) int32 in place."""
    d = np.asarray(d_means, np.float32)
    vis = np.any(d != 0.0, axis=1) if visible is None else np.asarray(visible).astype(bool)
    abs_sum[vis] = (abs_sum[vis] + np.abs(d[vis])).astype(np.float32)
    count[vis] += 1


def _rotmat(q):
    q = np.asarray(q, np.float64)
    q = q / np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def _keep(cfg: ADCConfig, w, s):
    """Pruning test of one resulting particle (float32 decisions)."""
    f = np.float32
    tau_min = f(-math.log1p(-cfg.prune_opacity))
    dens = f(f(SQRT_2PI) * f(w)) * f(min(s[0], s[1], s[2]))
    if not dens >= tau_min:
        return False
    big = f(cfg.big_world * cfg.scene_extent)
    return not (cfg.big_world > 0.0 and f(max(s[0], s[1], s[2])) > big)


def densify(cfg: ADCConfig, means, scales, quats, weights, sh, abs_sum, count):
    """Clone / split / prune (App. D with the 3DGS rules).  Returns
    (means, scales, quats, weights, sh) of the new set, and per input the
    action taken: 0 kept as is, 1 cloned, 2 split (before pruning)."""
    f = np.float32
    P = len(weights)
    out = {k: [] for k in ("means", "scales", "quats", "weights", "sh")}
    action = np.zeros(P, np.int32)
    dense_limit = f(cfg.percent_dense * cfg.scene_extent)
    thr = f(cfg.grad_threshold)
    for i in range(P):
        a = np.asarray(abs_sum[i], np.float32)
        n = int(count[i])
        grad = f(0.0)
        if n > 0:
            n2 = f(f(a[0] * a[0]) + f(a[1] * a[1]))
            n2 = f(n2 + f(a[2] * a[2]))
            grad = f(np.sqrt(n2) / f(n))
        s = np.asarray(scales[i], np.float64)
        smax = f(max(f(s[0]), f(s[1]), f(s[2])))
        cands = []
        if n > 0 and grad >= thr and smax <= dense_limit:
            action[i] = 1
            for _ in range(2):
                cands.append((means[i], s, quats[i], 0.5 * float(weights[i]), sh[i]))
        elif n > 0 and grad >= thr:
            action[i] = 2
            k = int(np.argmax(s))           # first index of the largest scale
            v = _rotmat(quats[i])[:, k]     # its axis (a column of R, Sigma = R S^2 R^T)
            s_new = s.copy()
            s_new[k] = f(f(cfg.split_gamma) * f(s[k]))    # formed in float32: the pruning test reads it
            for sign in (-1.0, 1.0):
                cands.append((np.asarray(means[i], np.float64) + sign * cfg.split_delta * s[k] * v, s_new, quats[i],
                              float(weights[i]), sh[i]))
        else:
            cands.append((means[i], s, quats[i], float(weights[i]), sh[i]))
        for m, sc, q, w, c in cands:
            if _keep(cfg, w, sc):
                out["means"].append(np.asarray(m, np.float64))
                out["scales"].append(np.asarray(sc, np.float64))
                out["quats"].append(np.asarray(q, np.float64))
                out["weights"].append(w)
                out["sh"].append(np.asarray(c, np.float64))
    res = {k: np.array(v, np.float64) for k, v in out.items()}
    if len(res["weights"]) == 0:
        res = dict(means=np.zeros((0, 3)), scales=np.zeros((0, 3)), quats=np.zeros((0, 4)), weights=np.zeros(0),
                   sh=np.zeros((0,) + np.asarray(sh).shape[1:]))
    return res, action
