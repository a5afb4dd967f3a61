"""mb3dgs_render_noalloc: the render entry point for callers that cannot
allocate device memory (its workspace is a fixed static device array).

Checked through the C ABI against mb3dgs_render (caller-provided workspace)
on two calls in a row, within the parity tolerance of the other GPU tests.
This file is collected last on purpose."""
import ctypes as C

import pytest
import torch

import scenes

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_11800_gb300 import GaussianTensors, Rasterizer
    from paper_2512_11800_gb300 import _binding as B
    R = Rasterizer()
    return R, B, GaussianTensors


def _noalloc(R, B, g, cams, npix):
    arr, nv = R.cameras(cams)
    rgb = torch.full((npix, 3), -1.0, device="cuda")
    T = torch.full((npix,), -1.0, device="cuda")
    P = torch.full((npix,), -1.0, device="cuda")
    st = torch.full((1,), 12345, dtype=torch.int32, device="cuda")
    gc = g.to_c()
    rc = R.lib.mb3dgs_render_noalloc(C.byref(R.cfg_c), C.byref(gc), arr, nv, C.c_void_p(rgb.data_ptr()),
                                     C.c_void_p(T.data_ptr()), C.c_void_p(P.data_ptr()), C.c_void_p(st.data_ptr()),
                                     C.c_void_p(torch.cuda.current_stream().cuda_stream))
    B.check(rc, "render_noalloc")
    torch.cuda.synchronize()
    return rgb, T, P, int(st.item())


@pytest.mark.parametrize("name", ["uniform2k_128", "two_views"])
def test_noalloc_matches_render_twice(setup, name):
    R, B, GaussianTensors = setup
    if name == "two_views":
        sc = scenes.scene_uniform(3000, 21)
        cams = [scenes.look_at((0, 0, -3), width=96, height=64), scenes.look_at((1.5, 0.5, -2.5), width=80, height=80)]
    else:
        sc, cam = scenes.workload(name)
        cams = [cam]
    g = GaussianTensors.from_scene(sc)
    npix = sum(c.width * c.height for c in cams)
    ref = R.render(g, cams)
    torch.cuda.synchronize()
    for _ in range(2):
        rgb, T, P, st = _noalloc(R, B, g, cams, npix)
        assert st == 0
        assert (rgb - ref["rgb"]).abs().max().item() <= TOL
        assert (T - ref["T"]).abs().max().item() <= TOL
        assert (P - ref["penalty"]).abs().max().item() <= TOL * max(1.0, ref["penalty"].abs().max().item())


def test_noalloc_rejects_oversized_problems(setup):
    R, B, GaussianTensors = setup
    sc = scenes.scene_uniform(100, 3)
    g = GaussianTensors.from_scene(sc)
    gc = g.to_c()
    gc.P = 50_000_000                       # records alone exceed the fixed workspace: rejected before any launch
    cam = scenes.look_at((0, 0, -3), width=64, height=64)
    arr, nv = R.cameras(cam)
    buf = torch.empty(64 * 64 * 5 + 1, device="cuda")
    p = buf.data_ptr()
    rc = R.lib.mb3dgs_render_noalloc(C.byref(R.cfg_c), C.byref(gc), arr, nv, C.c_void_p(p), C.c_void_p(p),
                                     C.c_void_p(p), C.c_void_p(p), None)
    assert rc == -3
