"""Pins for the oracle's adaptive density control (Sec. 3.4; App. D
"Adaptive Density Control"): each check compares it with something other
than its own formulas (the oracle's 1D Gaussian of Eq. 4-6, the density of
the 3D Gaussians, an eigendecomposition, a numerical optimisation of the
App. D split objective, invariants of the rules)."""
import json
import math
import os

import numpy as np
import torch
from scipy import integrate, optimize, special

import oracle as O
import scenes

A = O.adc
GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


def test_printed_constants():
    g = json.load(open(GOLD))
    cfg = A.ADCConfig()
    assert cfg.grad_threshold == g["adc_grad_threshold"]["value"]
    assert cfg.split_gamma == g["split_gamma"]["value"]
    assert cfg.split_delta == g["split_delta"]["value"]


def _density(x, mean, scales, quat, w):
    """3D density w exp(-1/2 (x - mu)^T Sigma^-1 (x - mu)), Sigma = R S^2 R^T (Sec. 3.1)."""
    R = O.quat_to_rotmat(torch.as_tensor(np.asarray(quat, np.float64))).numpy()
    Sinv = R @ np.diag(1.0 / np.asarray(scales, np.float64) ** 2) @ R.T
    d = x - mean
    return w * np.exp(-0.5 * np.einsum("ni,ij,nj->n", d, Sinv, d))


def test_view_independent_opacity_is_the_opacity_along_the_shortest_axis():
    """1 - exp(-tau) of a ray through the centre along the axis of the smallest
    scale, from the oracle's ray-parameterised Gaussian (Eq. 4-6) with both
    erf terms of the optical depth at their bound: tau = w-hat Sigma sqrt(2 pi)."""
    rng = np.random.default_rng(0)
    for _ in range(20):
        s = np.exp(rng.normal(-2.0, 0.7, 3))
        q = rng.normal(size=4)
        w = rng.uniform(0.1, 20.0)
        R = O.quat_to_rotmat(torch.as_tensor(q)).numpy()
        k = int(np.argmin(s))
        d = R[:, k]                                   # unit axis of the smallest scale
        o = -7.0 * d                                  # ray origin on that axis, Gaussian at 0
        o_g = torch.as_tensor(R.T @ (o - 0.0) / s)    # S^-1 R^T (o - mu)
        d_g = torch.as_tensor(R.T @ d / s)
        Sig, mu, what = O.gaussian_1d(o_g, d_g, torch.tensor(w, dtype=torch.float64))
        tau = float(what * Sig) * math.sqrt(2.0 * math.pi)
        # the exponent of w-hat cancels (|o_g|^2 ~ 4e4 here): FP64 rounding ~1e-12
        assert abs(A.view_independent_opacity(w, s) - (1.0 - math.exp(-tau))) < 1e-10


def test_init_weights_inverts_the_opacity():
    rng = np.random.default_rng(1)
    o = rng.uniform(0.01, 0.99, 50)
    s_iso = np.repeat(np.exp(rng.normal(-2.0, 0.5, (50, 1))), 3, 1)
    assert np.allclose(A.view_independent_opacity(A.init_weights(o, s_iso), s_iso), o, rtol=1e-12)
    s = np.exp(rng.normal(-2.0, 0.5, (50, 3)))
    # the average scale is at least the minimal one: the opacity along the
    # shortest axis of the initialised particle is at most the target
    assert np.all(A.view_independent_opacity(A.init_weights(o, s), s) <= o + 1e-15)


def test_split_constants_minimise_the_appendix_objective():
    """App. D: children at +/- c (1 - gamma), scale gamma (units of the split
    axis' scale, peak density 1, t_n -> -inf) minimising the squared change of
    the opacity contribution T(t) sigma(t).  The objective is flat near its
    minimum; the printed (gamma, delta) lie within 0.1 % of the minimal value
    and within 0.01 of the numerical minimiser."""
    def objective(x):
        c, g = x
        d = c * (1.0 - g)
        def f(t):
            so = math.exp(-0.5 * t * t)
            to = math.exp(-math.sqrt(math.pi / 2) * (1 + special.erf(t / math.sqrt(2))))
            sn = math.exp(-0.5 * ((t - d) / g) ** 2) + math.exp(-0.5 * ((t + d) / g) ** 2)
            tn = math.exp(-g * math.sqrt(math.pi / 2) * ((1 + special.erf((t - d) / (math.sqrt(2) * g)))
                                                        + (1 + special.erf((t + d) / (math.sqrt(2) * g)))))
            return (to * so - tn * sn) ** 2
        return integrate.quad(f, -12, 12, limit=400)[0]
    best = min((optimize.minimize(objective, x0, method="Nelder-Mead",
                                  options=dict(xatol=1e-9, fatol=1e-14, maxiter=2000))
                for x0 in ([1.5, 0.6], [2.0, 0.7])), key=lambda r: r.fun)
    g, d = A.SPLIT_GAMMA, A.SPLIT_DELTA
    at_printed = objective([d / (1.0 - g), g])
    assert at_printed <= best.fun * 1.001, (at_printed, best.fun)
    assert abs(best.x[1] - g) < 0.01 and abs(best.x[0] * (1 - best.x[1]) - d) < 0.01, best.x


def _scene(P, seed):
    sc = scenes.scene_uniform(P, seed)
    return (sc.means.astype(np.float64), sc.scales.astype(np.float64), sc.quats.astype(np.float64),
            sc.weights.astype(np.float64), sc.sh.astype(np.float64))


def test_clone_conserves_the_density():
    """Every particle cloned (threshold 0, all small): twice the particles,
    and the density of the new set equals the old one everywhere."""
    m, s, q, w, sh = _scene(60, 3)
    cfg = A.ADCConfig(grad_threshold=0.0, percent_dense=1e9, prune_opacity=0.0, big_world=0.0)
    out, act = A.densify(cfg, m, s, q, w, sh, np.ones((60, 3), np.float32), np.ones(60, np.int32))
    assert np.all(act == 1) and len(out["weights"]) == 120
    x = np.random.default_rng(4).normal(0.0, 1.0, (200, 3))
    old = sum(_density(x, m[i], s[i], q[i], w[i]) for i in range(60))
    new = sum(_density(x, out["means"][i], out["scales"][i], out["quats"][i], out["weights"][i]) for i in range(120))
    assert np.allclose(new, old, rtol=1e-12, atol=1e-300)


def test_split_moves_along_the_principal_axis():
    """Every particle split: the children sit at mean -/+ delta s_max v with v
    the eigenvector of the largest eigenvalue of Sigma (numpy eigh), and their
    covariance has that eigenvalue scaled by gamma^2, the others unchanged."""
    m, s, q, w, sh = _scene(40, 5)
    cfg = A.ADCConfig(grad_threshold=0.0, percent_dense=0.0, prune_opacity=0.0, big_world=0.0)
    out, act = A.densify(cfg, m, s, q, w, sh, np.ones((40, 3), np.float32), np.ones(40, np.int32))
    assert np.all(act == 2) and len(out["weights"]) == 80
    for i in range(40):
        R = O.quat_to_rotmat(torch.as_tensor(q[i])).numpy()
        Sig = R @ np.diag(s[i] ** 2) @ R.T
        ev, V = np.linalg.eigh(Sig)
        v, smax = V[:, -1], math.sqrt(ev[-1])
        for j, sign in ((2 * i, -1.0), (2 * i + 1, 1.0)):
            off = out["means"][j] - m[i]
            assert abs(abs(off @ v) - A.SPLIT_DELTA * smax) < 1e-9 * (1 + smax)
            assert np.linalg.norm(off - (off @ v) * v) < 1e-9
            Rc = O.quat_to_rotmat(torch.as_tensor(out["quats"][j])).numpy()
            evc = np.linalg.eigvalsh(Rc @ np.diag(out["scales"][j] ** 2) @ Rc.T)
            expect = np.sort(np.concatenate([ev[:2], [ev[-1] * A.SPLIT_GAMMA ** 2]]))
            assert np.allclose(evc, expect, rtol=1e-6, atol=0.0)   # gamma s_max is formed in float32
        assert np.allclose(out["means"][2 * i] + out["means"][2 * i + 1], 2 * m[i], atol=1e-12)


def test_rules_identity_threshold_and_pruning():
    m, s, q, w, sh = _scene(80, 6)
    rng = np.random.default_rng(7)
    abs_sum = rng.uniform(0.0, 3e-4, (80, 3)).astype(np.float32)
    count = rng.integers(0, 4, 80).astype(np.int32)
    # nothing reaches an infinite threshold and nothing is pruned: identity
    ident, act = A.densify(A.ADCConfig(grad_threshold=np.inf, prune_opacity=0.0, big_world=0.0),
                           m, s, q, w, sh, abs_sum, count)
    assert np.all(act == 0) and np.array_equal(ident["means"], m) and np.array_equal(ident["weights"], w)
    # the criterion: norm of the summed absolute gradients over the visible steps
    grad = np.linalg.norm(abs_sum.astype(np.float64), axis=1) / np.maximum(count, 1)
    _, act = A.densify(A.ADCConfig(prune_opacity=0.0, big_world=0.0), m, s, q, w, sh, abs_sum, count)
    sel = (count > 0) & (grad >= 1e-4)
    near = np.abs(grad - 1e-4) < 1e-9
    assert np.array_equal((act > 0)[~near], sel[~near])
    # pruning removes exactly the particles below the opacity threshold
    o = A.view_independent_opacity(w, s)
    thr = float(np.median(o))
    kept, _ = A.densify(A.ADCConfig(grad_threshold=np.inf, prune_opacity=thr, big_world=0.0),
                        m, s, q, w, sh, abs_sum, count)
    far = np.abs(o - thr) > 1e-6
    assert np.array_equal(np.isin(w, kept["weights"])[far], (o >= thr)[far])


def test_grad_stats_accumulate_absolute_components():
    rng = np.random.default_rng(8)
    abs_sum = np.zeros((30, 3), np.float32)
    count = np.zeros(30, np.int32)
    total = np.zeros((30, 3))
    seen = np.zeros(30, int)
    for step in range(5):
        d = rng.normal(size=(30, 3)).astype(np.float32)
        d[rng.random(30) < 0.3] = 0.0                  # not visible this step
        A.accumulate_grad_stats(d, None, abs_sum, count)
        vis = np.any(d != 0, axis=1)
        total[vis] += np.abs(d[vis])
        seen += vis
    assert np.array_equal(count, seen)
    assert np.allclose(abs_sum, total, rtol=1e-6)
