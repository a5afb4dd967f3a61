"""GPU parity of the trigonometric-moment basis (Sec. 3.2, Eq. 13-14;
App. C "Trigonometric Moments"): the CUDA path through the C ABI against the
oracle's trigonometric path.

Bar: 1e-4 absolute on RGB and final transmittance, at N = 3 and N = 5
intervals.  The transmittance T(eta) at fixed probe depths is held to 1e-4
plus, for nearly atomic pixels (|m1/m0| close to 1, where the circle bounds
are ill-conditioned and the FP32 moments decide the fourth digit), the change
of the oracle's own T(eta) under a 2e-6 (of m0) perturbation of its moments
(helpers.probe_excess).

The adjoint of this basis (Verblunsky-coefficient query adjoints, reverse
Levinson-Durbin, the reverse of Eq. 14) is held to the backward bar against
the oracle's autograd gradient through its trigonometric bounds: relative L2
<= 1e-3 per parameter group and, element by element, within 1e-3 of the
group's largest oracle element.
"""
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
torch.set_num_threads(os.cpu_count() or 8)
PROBES = np.linspace(0.0, 1.0, 17)


def _rasterizer(N, **kw):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_11800_gb300 import RasterConfig, Rasterizer
    return Rasterizer(RasterConfig(basis="trig", n_intervals=N, **kw))


def G(sc):
    from paper_2512_11800_gb300 import GaussianTensors
    return GaussianTensors.from_scene(sc)


def _img(t, cam):
    return t.detach().cpu().double().numpy().reshape(cam.height, cam.width, *t.shape[1:])


def _errors(out, ref, cam, region=None):
    x0, y0, w, h = region or (0, 0, cam.width, cam.height)
    sl = (slice(y0, y0 + h), slice(x0, x0 + w))
    err = dict(rgb=float(np.abs(_img(out["rgb"], cam)[sl] - ref["rgb"].numpy()).max()),
               T=float(np.abs(_img(out["T"], cam)[sl] - ref["T"].numpy()).max()))
    if out.get("T_eta") is not None and "tau_probe" in ref:
        err["T_eta"] = float(np.abs(_img(out["T_eta"], cam)[sl] - np.exp(-ref["tau_probe"].numpy())).max())
    return err


@pytest.mark.parametrize("N", [3, 5])
def test_trig_uniform2k(N):
    """The 2k-Gaussian 128x128 frame, checked on its 64x64 centre (where the
    scene is): image, transmittance probes and the moments themselves."""
    R = _rasterizer(N)
    sc, cam = scenes.workload("uniform2k_128")
    npix = cam.width * cam.height
    eta = torch.tensor(PROBES, dtype=torch.float32, device="cuda").expand(npix, -1).contiguous()
    out = R.render_staged(G(sc), cam, eta=eta)
    region = (32, 32, 64, 64)
    ref = O.render(sc, cam, oracle_config(R.config), probes=PROBES, region=region)
    err = _errors(out, ref, cam, region)
    sl = (slice(32, 96), slice(32, 96))
    excess, n_allow = helpers.probe_excess(_img(out["T_eta"], cam)[sl], ref, PROBES, oracle_config(R.config))
    print("trig uniform2k N=%d max errors" % N, err, "pixels judged by conditioning", n_allow)
    assert err["rgb"] <= TOL and err["T"] <= TOL and excess <= 0.0, (err, excess)
    # the staged moment output is the trigonometric moments {m0, Re m_k, Im m_k}
    m = _img(out["moments"], cam)[sl]
    mr = ref["m"].numpy()
    mo = np.concatenate([mr[..., :1].real, np.stack([mr[..., 1:].real, mr[..., 1:].imag], -1).reshape(
        mr.shape[0], mr.shape[1], -1)], -1)
    assert np.abs(m - mo).max() <= 1e-5 * max(1.0, float(np.abs(mo[..., 0]).max())) + 1e-6


@pytest.mark.parametrize("N", [3, 5])
def test_trig_ragged_near_camera(N):
    R = _rasterizer(N, bg=(0.2, 0.5, 0.1))
    sc = scenes.scene_uniform(600, 5)
    cam = scenes.look_at((0.1, -0.2, -1.6), width=77, height=45, fov_deg=70)
    out = R.render(G(sc), cam)
    ref = O.render(sc, cam, oracle_config(R.config))
    err = _errors(out, ref, cam)
    assert err["rgb"] <= TOL and err["T"] <= TOL, err


def test_trig_full_size_crop():
    """1M Gaussians at 1920x1080 with N = 5, checked on a 32x32 centre crop."""
    R = _rasterizer(5)
    sc, cam = helpers.workload("shells1M_1080p")
    out = R.render(G(sc), cam)
    assert R.status()[0] == 0
    region = ((cam.width - 32) // 2, (cam.height - 32) // 2, 32, 32)
    cfg = oracle_config(R.config)
    ref = O.render(sc, cam, cfg, region=region, pre=helpers.oracle_pre("shells1M_1080p", cfg))
    err = _errors(out, ref, cam, region)
    print("trig shells1M crop N=5", err, "pairs", ref["n_pairs"])
    assert err["rgb"] <= TOL and err["T"] <= TOL, err
    assert torch.isfinite(out["rgb"]).all()


NAMES = ["means", "scales", "quats", "weights", "sh"]
REL = 1e-3


def _grads(R, sc, cam, g_img, gP_img, gT_img=None):
    g = G(sc)
    out = R.render(g, cam)
    dr = torch.as_tensor(g_img.reshape(-1, 3), dtype=torch.float32, device="cuda")
    dp = torch.as_tensor(gP_img.reshape(-1), dtype=torch.float32, device="cuda")
    dT = None if gT_img is None else torch.as_tensor(gT_img.reshape(-1), dtype=torch.float32, device="cuda")
    grads = R.backward(g, cam, out["capacity"], dr, dp, dL_dT=dT)
    torch.cuda.synchronize()
    assert R.status()[0] == 0
    return {k: v.detach().cpu().double().numpy().reshape(-1) for k, v in grads.items()}


def _rel_errors(gg, ref):
    out = {}
    for k in NAMES:
        a, b = gg[k], ref[k].reshape(-1)
        assert np.isfinite(b).all(), ("oracle gradient not finite", k)
        assert np.isfinite(a).all(), ("GPU gradient not finite", k, int((~np.isfinite(a)).sum()))
        scale = max(float(np.abs(b).max()), 1e-30)
        out[k] = max(float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)), float(np.abs(a - b).max()) / scale)
    return out


@pytest.mark.parametrize("N", [3, 5])
def test_trig_backward_sh3_near_camera(N):
    """SH degree 3, background colour, and losses on RGB, penalty and final
    transmittance."""
    R = _rasterizer(N, bg=(0.1, 0.2, 0.3))
    sc = scenes.tiny_scene(P=40, seed=9, deg=3, spread=0.5)
    cam = scenes.look_at((0.1, 0.2, -2.0), width=48, height=40, fov_deg=55)
    rng = np.random.default_rng(4)
    g_img = rng.normal(size=(cam.height, cam.width, 3))
    gP_img = rng.normal(size=(cam.height, cam.width)) * 0.1
    gT_img = rng.normal(size=(cam.height, cam.width))
    gg = _grads(R, sc, cam, g_img, gP_img, gT_img)
    ref = O.render_grad(sc, cam, oracle_config(R.config), g_img, gP_img, dL_dT=gT_img)
    err = _rel_errors(gg, ref)
    print("trig backward sh3 near camera N=%d" % N, err)
    assert max(err.values()) <= REL, err


def test_trig_backward_uniform2k_centre():
    """The 2k-Gaussian 128x128 frame at N = 5 with the upstream gradient on
    a 48x48 crop of its centre, where the scene is (dense, overlapping
    pixels)."""
    R = _rasterizer(5)
    sc, cam = scenes.workload("uniform2k_128")
    x0, y0, s = 40, 40, 48
    rng = np.random.default_rng(5)
    g_img = np.zeros((cam.height, cam.width, 3))
    gP_img = np.zeros((cam.height, cam.width))
    g_img[y0:y0 + s, x0:x0 + s] = rng.normal(size=(s, s, 3))
    gP_img[y0:y0 + s, x0:x0 + s] = rng.normal(size=(s, s)) * 0.1
    gg = _grads(R, sc, cam, g_img, gP_img)
    ref = O.render_grad(sc, cam, oracle_config(R.config), g_img[y0:y0 + s, x0:x0 + s], gP_img[y0:y0 + s, x0:x0 + s],
                        region=(x0, y0, s, s))
    err = _rel_errors(gg, ref)
    print("trig backward uniform2k centre crop N=5", err)
    assert max(err.values()) <= REL, err


def test_trig_backward_full_size_crop():
    """1M Gaussians at 1920x1080 with N = 5 rendered and differentiated in
    full; the upstream gradient is non-zero on the centre 24x24 crop only."""
    R = _rasterizer(5)
    sc, cam = helpers.workload("shells1M_1080p")
    x0, y0, s = 948, 528, 24
    rng = np.random.default_rng(6)
    g_img = np.zeros((cam.height, cam.width, 3))
    gP_img = np.zeros((cam.height, cam.width))
    g_img[y0:y0 + s, x0:x0 + s] = rng.normal(size=(s, s, 3))
    gP_img[y0:y0 + s, x0:x0 + s] = rng.normal(size=(s, s)) * 0.1
    gg = _grads(R, sc, cam, g_img, gP_img)
    ref = O.render_grad(sc, cam, oracle_config(R.config), g_img[y0:y0 + s, x0:x0 + s], gP_img[y0:y0 + s, x0:x0 + s],
                        region=(x0, y0, s, s))
    err = _rel_errors(gg, ref)
    print("trig backward shells1M crop N=5", err, "pairs", ref["out"]["n_pairs"])
    assert max(err.values()) <= REL, err


def test_trig_kept_queries_match_solved():
    """Trigonometric bound queries kept by the quadrature pass (16 bytes:
    tau, the node angles, j and the node count) for all, half or none of the
    pairs: the image is bit-identical and the gradients equal those of
    queries solved again in pass 1 to rounding."""
    R = _rasterizer(5, bg=(0.1, 0.2, 0.3))
    sc, cam = scenes.workload("uniform2k_128")
    g = G(sc)
    tp, pp = R.pair_counts(g, cam)
    rng = np.random.default_rng(11)
    dr = torch.as_tensor(rng.normal(size=(cam.width * cam.height, 3)), dtype=torch.float32, device="cuda")
    res = {}
    for name, qc in [("all", pp), ("half", pp // 2), ("none", 0)]:
        out = R.render(g, cam, capacity=tp, query_capacity=qc)
        assert R.status()[0] == 0 and R.cfg_c.query_capacity == qc
        grads = R.backward(g, cam, tp, dr, query_capacity=qc)
        torch.cuda.synchronize()
        res[name] = (out["rgb"].clone(), {k: v.clone() for k, v in grads.items()})
    for name in ["all", "half"]:
        assert torch.equal(res[name][0], res["none"][0])
        for k in NAMES:
            a, b = res[name][1][k], res["none"][1][k]
            assert float((a - b).norm() / b.norm().clamp_min(1e-30)) <= 1e-5, (name, k)
