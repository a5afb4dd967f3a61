"""The oracle's gradient (autograd through the FP64 oracle, roots
differentiated implicitly) against central finite differences of the oracle
loss, with the proxy rectangles held fixed: power moments (Eq. 10-12, N = 3)
and trigonometric moments (Eq. 13-14, N = 5)."""
import numpy as np
import pytest
import torch

import oracle as O
import scenes


def _perturbed(sc, name, idx, h):
    s2 = scenes.Scene(sc.means.copy(), sc.scales.copy(), sc.quats.copy(), sc.weights.copy(), sc.sh.copy(),
                      sc.sh_degree)
    arr = getattr(s2, name).astype(np.float64)
    arr.reshape(-1)[idx] += h
    # the oracle reads float64 values from float32 arrays; keep float64 arrays for the perturbation
    setattr(s2, name, arr)
    return s2


@pytest.mark.parametrize("basis", ["power", "trig"])
@pytest.mark.parametrize("seed", [0, 1])
def test_oracle_gradient_matches_central_differences(seed, basis):
    sc = scenes.tiny_scene(P=7, seed=30 + seed, spread=0.3, log_scale=(-1.7, 0.25), deg=1)
    sc = scenes.Scene(sc.means.astype(np.float64), sc.scales.astype(np.float64), sc.quats.astype(np.float64),
                      sc.weights.astype(np.float64), sc.sh.astype(np.float64), sc.sh_degree)
    cam = scenes.look_at((0.05, 0.1, -2.4), width=20, height=18, fov_deg=45)
    cfg = O.OracleConfig(bg=(0.1, 0.2, 0.3), basis=basis, n_intervals=5 if basis == "trig" else 3)
    rng = np.random.default_rng(seed)
    g = rng.normal(size=(18, 20, 3))
    gP = rng.normal(size=(18, 20)) * 0.3
    res = O.render_grad(sc, cam, cfg, g, gP)
    rect0 = res["out"]["pre"].rect
    checked = 0
    # h = 1e-4: the oracle's FP64 noise floor (~1e-9, Hankel conditioning) makes smaller steps noisy
    for name, rel in [("means", 1e-4), ("scales", 1e-4), ("quats", 1e-4), ("weights", 1e-4), ("sh", 1e-4)]:
        arr = getattr(sc, name)
        for idx in rng.choice(arr.size, size=min(6, arr.size), replace=False):
            h = rel * max(0.1, abs(arr.reshape(-1)[idx]))
            lp, rp = O.render_loss(_perturbed(sc, name, idx, h), cam, cfg, g, gP)
            lm, rm = O.render_loss(_perturbed(sc, name, idx, -h), cam, cfg, g, gP)
            if not (torch.equal(rp, rect0) and torch.equal(rm, rect0)):
                continue                      # a rectangle edge moved: FD across a discontinuity
            fd = (lp - lm) / (2 * h)
            an = res[name].reshape(-1)[idx]
            assert abs(fd - an) <= 2e-5 * max(1.0, abs(an)) + 2e-5, (name, idx, fd, an)
            checked += 1
    assert checked >= 20
