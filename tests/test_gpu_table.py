"""GPU parity of the tabulated transmittance: the quadrature pass
interpolates a per-pixel table of tau(eta) (48 Chebyshev-spaced knots on each
segment between the Gauss nodes, cubic Hermite with the bound's exact
derivative) instead of solving each bound query of Eq. 8.  Checked against the
oracle's solved bounds at the parity bar, 1e-4 on RGB and transmittance, on
the 2k scene and a crop of the 1M-Gaussian 1080p frame; the adjoint (of the
solved bounds) against the oracle gradient at the backward bar."""
import os

import numpy as np
import pytest
import torch

import helpers
import oracle as O
import scenes
from helpers import oracle_config

pytestmark = pytest.mark.gpu
TOL = 1e-4
M = 48
torch.set_num_threads(os.cpu_count() or 8)


def _rasterizer(**kw):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_11800_gb300 import RasterConfig, Rasterizer
    return Rasterizer(RasterConfig(tau_table=M, **kw))


def G(sc):
    from paper_2512_11800_gb300 import GaussianTensors
    return GaussianTensors.from_scene(sc)


def _img(t, cam):
    return t.detach().cpu().double().numpy().reshape(cam.height, cam.width, *t.shape[1:])


def test_table_uniform2k():
    R = _rasterizer(bg=(0.2, 0.5, 0.1))
    sc, cam = scenes.workload("uniform2k_128")
    out = R.render(G(sc), cam)
    ref = O.render(sc, cam, oracle_config(R.config))
    e_rgb = float(np.abs(_img(out["rgb"], cam) - ref["rgb"].numpy()).max())
    e_T = float(np.abs(_img(out["T"], cam) - ref["T"].numpy()).max())
    print("table M=%d uniform2k: rgb %.2e T %.2e" % (M, e_rgb, e_T))
    assert e_rgb <= TOL and e_T <= TOL


def test_table_full_size_crop():
    R = _rasterizer()
    sc, cam = helpers.workload("shells1M_1080p")
    out = R.render(G(sc), cam)
    assert R.status()[0] == 0
    region = ((cam.width - 48) // 2, (cam.height - 48) // 2, 48, 48)
    ref = helpers.oracle_crop("shells1M_1080p", region)
    x0, y0, w, h = region
    e_rgb = float(np.abs(_img(out["rgb"], cam)[y0:y0 + h, x0:x0 + w] - ref["rgb"].numpy()).max())
    print("table M=%d shells1M crop: rgb %.2e" % (M, e_rgb))
    assert e_rgb <= TOL


def test_table_backward_matches_oracle_gradient():
    """With a table the adjoint differentiates the solved bounds that the
    table approximates (pass 1 solves its queries again): held to the
    backward bar against the oracle gradient (relative L2 <= 1e-3 per group,
    element by element within 1e-3 of the group's largest oracle element)."""
    R = _rasterizer(bg=(0.1, 0.2, 0.3))
    sc = scenes.tiny_scene(P=40, seed=9, deg=3, spread=0.5)
    cam = scenes.look_at((0.1, 0.2, -2.0), width=48, height=40, fov_deg=55)
    rng = np.random.default_rng(7)
    g_img = rng.normal(size=(cam.height, cam.width, 3))
    gP_img = rng.normal(size=(cam.height, cam.width)) * 0.1
    g = G(sc)
    out = R.render(g, cam)
    dr = torch.as_tensor(g_img.reshape(-1, 3), dtype=torch.float32, device="cuda")
    dp = torch.as_tensor(gP_img.reshape(-1), dtype=torch.float32, device="cuda")
    grads = R.backward(g, cam, out["capacity"], dr, dp)
    torch.cuda.synchronize()
    assert R.status()[0] == 0
    ref = O.render_grad(sc, cam, oracle_config(R.config), g_img, gP_img)
    err = {}
    for k in ["means", "scales", "quats", "weights", "sh"]:
        a = grads[k].detach().cpu().double().numpy().reshape(-1)
        b = ref[k].reshape(-1)
        err[k] = max(float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)),
                     float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-30)))
    print("table backward sh3 near camera", err)
    assert max(err.values()) <= 1e-3, err
