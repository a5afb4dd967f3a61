"""GPU: execution shapes, the autotuner, batched views and CUDA-graph capture.

The tile shape, record batch and tile schedule change only how pixels map to
CTAs: every pixel still visits its Gaussians in ascending id order, so the
forward images are bit-identical across shapes, and per-view images of a
batched multi-view render are bit-identical to single-view renders.  The
backward sums per-Gaussian gradients with float atomics, so across shapes it
agrees to rounding (relative L2 <= 1e-5).  Tile lists of non-square tiles
are compared bit-exactly with the oracle's binning.
"""
import numpy as np
import pytest
import torch

import oracle as O
import scenes

pytestmark = pytest.mark.gpu
NAMES = ["means", "scales", "quats", "weights", "sh"]
SHAPES = [(16, 16), (32, 8), (8, 32), (64, 4)]


def _rast(**kw):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_11800_gb300 import RasterConfig, Rasterizer
    return Rasterizer(RasterConfig(bg=(0.1, 0.2, 0.3), **kw))


def G(sc):
    from paper_2512_11800_gb300 import GaussianTensors
    return GaussianTensors.from_scene(sc)


def _scene_and_views():
    sc = scenes.scene_uniform(3000, 21)
    cams = [scenes.look_at((0, 0, -3), width=100, height=60), scenes.look_at((2, 1, -2), width=37, height=91)]
    return sc, cams


def _rel(a, b):
    return float(torch.linalg.vector_norm(a - b) / max(float(torch.linalg.vector_norm(b)), 1e-30))


def test_execution_shapes_give_identical_images():
    sc, cams = _scene_and_views()
    g = G(sc)
    ref = _rast(tile_w=16, tile_h=16, batch=256, schedule="grid").render(g, cams)
    for tw, th in SHAPES:
        for batch in (32, 128, 256):
            for sched in ("queue", "grid"):
                out = _rast(tile_w=tw, tile_h=th, batch=batch, schedule=sched).render(g, cams)
                for k in ["rgb", "T", "penalty"]:
                    assert torch.equal(out[k], ref[k]), (tw, th, batch, sched, k)


@pytest.mark.parametrize("tw,th", [(32, 8), (8, 32)])
def test_tile_lists_bit_exact_for_other_shapes(tw, th):
    sc, cam = scenes.workload("uniform2k_128")
    cam = scenes.look_at((0, 0, -3), fov_deg=60, width=131, height=77)     # ragged in both directions
    R = _rast(tile_w=tw, tile_h=th)
    out = R.render_staged(G(sc), cam)
    r = out["rects"].cpu().numpy().astype(np.int64)
    empty = (r[:, 0] > r[:, 2]) | (r[:, 1] > r[:, 3])
    r[empty] = [1, 1, 0, 0]
    ids, ranges = O.bin_tiles(torch.as_tensor(r), cam.width, cam.height, tw, th)
    gr = out["ranges"].cpu().numpy().astype(np.int64)
    assert gr.shape[0] == ranges.shape[0] == R.num_tiles(cam)
    assert np.array_equal(gr[:, 1] - gr[:, 0], (ranges[:, 1] - ranges[:, 0]).numpy())
    gids = out["ids"].cpu().numpy()
    for t in range(gr.shape[0]):
        assert np.array_equal(gids[gr[t, 0]:gr[t, 1]], ids[ranges[t, 0]:ranges[t, 1]].numpy()), t


def test_backward_agrees_across_shapes_and_schedules():
    sc, cams = _scene_and_views()
    g = G(sc)
    npix = sum(c.width * c.height for c in cams)
    dl = torch.randn(npix, 3, device="cuda", generator=torch.Generator("cuda").manual_seed(3)) * 1e-2
    R0 = _rast(tile_w=16, tile_h=16, batch=256, schedule="grid")
    out = R0.render(g, cams)
    ref = {k: v.clone() for k, v in R0.backward(g, cams, out["capacity"], dl).items()}
    for tw, th, batch, sched, save in [(32, 8, 128, "queue", True), (8, 32, 64, "queue", False),
                                       (64, 4, 256, "grid", True)]:
        R = _rast(tile_w=tw, tile_h=th, batch=batch, schedule=sched, save_queries=save)
        o = R.render(g, cams)
        gr = R.backward(g, cams, o["capacity"], dl)
        for k in NAMES:
            assert _rel(gr[k], ref[k]) <= 1e-5, (tw, th, batch, sched, k)


def test_autotune_keeps_the_images():
    sc, cam = scenes.workload("uniform2k_128")
    g = G(sc)
    R = _rast()
    ref = R.render(g, cam)["rgb"].clone()
    tw, th, batch, sched, ms = R.autotune(g, cam, backward=True)
    assert (tw, th) in [(16, 16), (32, 8), (8, 32)] and batch in (0, 256) and sched in ("queue", "grid")
    assert ms > 0.0
    assert torch.equal(R.render(g, cam)["rgb"], ref)
    assert R.status()[0] == 0


def test_batched_views_match_single_views():
    """Uneven resolutions in one set of launches (one persistent launch per
    pass over all views' tiles): images bit-identical to single-view renders,
    gradients equal to the sum of the single-view gradients."""
    sc = scenes.scene_uniform(4000, 8)
    cams = [scenes.look_at(e, width=w, height=h) for e, w, h in
            [((0, 0, -3), 96, 54), ((2.5, 0.5, -1.5), 64, 36), ((-1, 2, -2.5), 160, 90), ((0.5, -2, 2), 64, 36)]]
    g = G(sc)
    R = _rast()
    both = R.render(g, cams)
    rgb_b = both["rgb"].clone()
    npix = [c.width * c.height for c in cams]
    dl = torch.randn(sum(npix), 3, device="cuda", generator=torch.Generator("cuda").manual_seed(5)) * 1e-2
    gb = {k: v.clone() for k, v in R.backward(g, cams, both["capacity"], dl).items()}
    o = 0
    acc = {k: torch.zeros_like(v) for k, v in gb.items()}
    for c, n in zip(cams, npix):
        one = R.render(g, c)
        assert torch.equal(one["rgb"], rgb_b[o:o + n])
        gs = R.backward(g, c, one["capacity"], dl[o:o + n].contiguous())
        for k in acc:
            acc[k] += gs[k]
        o += n
    for k in NAMES:
        assert _rel(gb[k], acc[k]) <= 1e-5, k


def test_cuda_graph_capture_of_forward_and_backward():
    """The whole fwd+bwd step (render, L2-loss gradient, backward) captured in
    one CUDA graph and replayed: same images and gradients as eager calls."""
    sc, cams = _scene_and_views()
    g = G(sc)
    R = _rast()
    tp, pp = R.pair_counts(g, cams)
    target = torch.rand(sum(c.width * c.height for c in cams), 3, device="cuda",
                        generator=torch.Generator("cuda").manual_seed(9))
    outbuf = None

    def step():
        nonlocal outbuf
        o = R.render(g, cams, capacity=tp, query_capacity=pp, out=outbuf)
        outbuf = o
        dl = (o["rgb"] - target).mul_(2.0 / o["rgb"].numel())
        return R.backward(g, cams, tp, dl, query_capacity=pp)

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(2):
            eager = step()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    rgb_e = outbuf["rgb"].clone()
    grads_e = {k: v.clone() for k, v in eager.items()}
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        cap_grads = step()
    outbuf["rgb"].zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(outbuf["rgb"], rgb_e)
    for k in NAMES:
        assert _rel(cap_grads[k], grads_e[k]) <= 1e-5, k
    assert R.status()[0] == 0
