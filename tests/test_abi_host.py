"""C ABI checks that need no GPU: the library builds for sm_103a, loads, and
exports every entry point declared in include/mb3dgs.h; host-only calls
validate arguments and size workspaces."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "mb3dgs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mb3dgs_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2512_11800_gb300 import _binding as B
    return B.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_2512_11800_gb300 import _binding as B
    syms = declared_symbols()
    assert len(syms) >= 14
    for s in syms:
        assert hasattr(lib, s), s
    assert sorted(B.EXPORTS) == syms


def test_config_defaults_and_status_strings(lib):
    from paper_2512_11800_gb300 import _binding as B
    c = B.Config()
    assert lib.mb3dgs_config_default(C.byref(c)) == 0
    assert c.n == 4 and c.n_intervals == 3 and abs(c.beta - 0.25) < 1e-7 and abs(c.kappa - 3) < 1e-7
    assert abs(c.conf_c - 0.01) < 1e-8 and abs(c.warp_lambda + 1.5) < 1e-7 and abs(c.bias_alpha - 1e-3) < 1e-9
    for code in [0, -1, -2, -3, -4, -5, -6, -7]:
        assert lib.mb3dgs_status_string(code).decode() == B.STATUS[code]


def _cam(W=1920, H=1080):
    import scenes
    from paper_2512_11800_gb300 import to_camera
    return to_camera(scenes.look_at((0, 0, -3), width=W, height=H))


def test_workspace_size_and_validation(lib):
    from paper_2512_11800_gb300 import _binding as B
    c = B.Config()
    lib.mb3dgs_config_default(C.byref(c))
    cam = _cam()
    n = C.c_size_t(0)
    assert lib.mb3dgs_workspace_size(C.byref(c), C.byref(cam), 1, 1000, 0, C.byref(n)) == 0
    a = n.value
    assert lib.mb3dgs_workspace_size(C.byref(c), C.byref(cam), 1, 1000, 1 << 20, C.byref(n)) == 0
    assert n.value >= a + 16 * (1 << 20)            # four 32-bit pair arrays
    assert lib.mb3dgs_num_tiles(None, C.byref(cam), 1) == 120 * 68
    bad = B.Config()
    lib.mb3dgs_config_default(C.byref(bad))
    bad.n = 3
    assert lib.mb3dgs_workspace_size(C.byref(bad), C.byref(cam), 1, 10, 0, C.byref(n)) == -6
    bad.n, bad.n_intervals = 4, 0
    assert lib.mb3dgs_workspace_size(C.byref(bad), C.byref(cam), 1, 10, 0, C.byref(n)) == -6
    bad.n_intervals, bad.conf_c = 3, 1.5
    assert lib.mb3dgs_workspace_size(C.byref(bad), C.byref(cam), 1, 10, 0, C.byref(n)) == -1
    assert lib.mb3dgs_workspace_size(C.byref(c), C.byref(cam), 0, 10, 0, C.byref(n)) == -1
    assert lib.mb3dgs_workspace_size(C.byref(c), C.byref(cam), 1, 10, 1 << 31, C.byref(n)) == -1
    cam.width = 0
    assert lib.mb3dgs_workspace_size(C.byref(c), C.byref(cam), 1, 10, 0, C.byref(n)) == -1
    # null workspace with a non-empty layout is rejected before any CUDA call
    g = B.Gaussians()
    assert lib.mb3dgs_preprocess(C.byref(c), C.byref(g), C.byref(_cam()), 1, None, 0, 0, None) == -1


def test_multiview_tiles(lib):
    from paper_2512_11800_gb300 import _binding as B
    cams = (B.Camera * 3)(_cam(640, 360), _cam(1280, 720), _cam(1920, 1080))
    assert lib.mb3dgs_num_tiles(None, cams, 3) == 40 * 23 + 80 * 45 + 120 * 68


def test_execution_shape_validation_and_tile_counts(lib):
    """Tile shapes w x h with w in {8, 16, 32, 64} and w h = 256 threads,
    record batches that are multiples of 32 up to 256, two schedules; the
    tile count follows the shape (ragged last row and column)."""
    from paper_2512_11800_gb300 import _binding as B
    cam = _cam(131, 77)
    n = C.c_size_t(0)
    for tw, th in [(8, 32), (16, 16), (32, 8), (64, 4)]:
        c = B.Config()
        lib.mb3dgs_config_default(C.byref(c))
        c.tile_w, c.tile_h = tw, th
        assert lib.mb3dgs_workspace_size(C.byref(c), C.byref(cam), 1, 10, 0, C.byref(n)) == 0
        assert lib.mb3dgs_num_tiles(C.byref(c), C.byref(cam), 1) == ((131 + tw - 1) // tw) * ((77 + th - 1) // th)
    for tw, th, batch, sched, code in [(16, 8, 256, 0, -6), (24, 16, 256, 0, -6), (128, 2, 256, 0, -6),
                                       (16, 16, 48, 0, -6), (16, 16, 512, 0, -6), (16, 16, 64, 7, -1)]:
        c = B.Config()
        lib.mb3dgs_config_default(C.byref(c))
        c.tile_w, c.tile_h, c.batch, c.schedule = tw, th, batch, sched
        assert lib.mb3dgs_workspace_size(C.byref(c), C.byref(cam), 1, 10, 0, C.byref(n)) == code, (tw, th, batch)


def test_query_capacity_policy():
    """Query slots (16 B x (N+1) a pair, 8 B x (N+1) in the compact form): all
    of the frame's pairs while they fit the budget, else as many as the
    budget holds (the backward solves the other pixels' queries again).  None
    without saved queries or with a table; the trigonometric basis keeps the
    16-byte form.  The C layout accepts capacities beyond 2^31."""
    from paper_2512_11800_gb300 import RasterConfig, Rasterizer
    from paper_2512_11800_gb300 import _binding as B
    R = Rasterizer(RasterConfig(query_budget_gb=1.0, query_format="full"))
    per_pair = 16 * (R.config.n_intervals + 1)
    fit = (1 << 30) // per_pair
    assert R.set_query_capacity(fit) == fit
    assert R.set_query_capacity(fit + 1) == fit
    assert R.set_query_capacity(10 * fit) == fit and R.cfg_c.compact_queries == 0
    assert R.set_query_capacity(0) == 0
    R.config.query_format = "compact"
    assert R.set_query_capacity(fit) == fit and R.cfg_c.compact_queries == 1
    assert R.set_query_capacity(fit + 1) == fit + 1
    assert R.set_query_capacity(10 * fit) == 2 * fit and R.cfg_c.compact_queries == 1
    n8, n16 = C.c_size_t(0), C.c_size_t(0)
    cam = _cam(128, 128)
    R.set_query_capacity(fit)                            # the same slots in both forms
    assert R.lib.mb3dgs_workspace_size(C.byref(R.cfg_c), C.byref(cam), 1, 100, 0, C.byref(n8)) == 0
    R.config.query_format = "full"
    R.set_query_capacity(fit)
    assert R.lib.mb3dgs_workspace_size(C.byref(R.cfg_c), C.byref(cam), 1, 100, 0, C.byref(n16)) == 0
    assert n16.value - n8.value >= fit * per_pair // 2 - 4096
    R.config.query_budget_gb = 1e6
    assert R.set_query_capacity(2 ** 33) == 2 ** 33
    n = C.c_size_t(0)
    cam = _cam(128, 128)
    assert R.lib.mb3dgs_workspace_size(C.byref(R.cfg_c), C.byref(cam), 1, 100, 0, C.byref(n)) == 0
    assert n.value >= 2 ** 33 * per_pair
    R.config.save_queries = False
    assert R.set_query_capacity(1000) == 0
    Rt = Rasterizer(RasterConfig(basis="trig", query_format="compact"))
    assert Rt.set_query_capacity(1000) == 1000 and Rt.cfg_c.compact_queries == 0   # 16-byte trig queries
    Rtab = Rasterizer(RasterConfig(tau_table=48))
    assert Rtab.set_query_capacity(1000) == 0


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No CPU fallback: without libmb3dgs.so the loader and the Rasterizer raise."""
    from paper_2512_11800_gb300 import RasterConfig, Rasterizer
    from paper_2512_11800_gb300 import _binding as B
    monkeypatch.setattr(B, "_lib", None)
    monkeypatch.setattr(B._build, "LIB", str(tmp_path / "missing" / "libmb3dgs.so"))
    monkeypatch.setattr(B._build, "build", lambda *a, **k: None)     # as if the build produced nothing
    with pytest.raises(ImportError):
        B.load()
    with pytest.raises(ImportError):
        Rasterizer(RasterConfig())


def test_workspace_size_is_monotone_in_pair_capacity(lib):
    """The allocation-free render finds the largest pair capacity that fits
    its fixed workspace by bisection, which needs the workspace size to be
    non-decreasing in the pair capacity."""
    import numpy as np
    from paper_2512_11800_gb300 import _binding as B
    c = B.Config()
    lib.mb3dgs_config_default(C.byref(c))
    cam = _cam(128, 128)
    n = C.c_size_t(0)
    caps = sorted(set([0, 1, 2, 3, 4095, 4096, 4097] + list(np.random.default_rng(0).integers(0, 1 << 30, 200))))
    sizes = []
    for cap in caps:
        assert lib.mb3dgs_workspace_size(C.byref(c), C.byref(cam), 1, 2000, int(cap), C.byref(n)) == 0
        sizes.append(n.value)
    assert all(a <= b for a, b in zip(sizes, sizes[1:]))
    # the largest capacity below a byte budget: it fits and the next one does not
    budget = 64 << 20

    def fits(cap):
        assert lib.mb3dgs_workspace_size(C.byref(c), C.byref(cam), 1, 2000, cap, C.byref(n)) == 0
        return n.value <= budget
    lo, hi = 0, (1 << 31) - 1
    while lo < hi:
        mid = lo + (hi - lo + 1) // 2
        lo, hi = (mid, hi) if fits(mid) else (lo, mid - 1)
    assert fits(lo) and not fits(lo + 1)


def test_adc_defaults_and_validation(lib):
    """mb3dgs_adc_config_default holds the paper's printed density-control
    constants (App. D) and the oracle's defaults; the calls validate their
    arguments on the host (no device work)."""
    import json
    import oracle as O
    from paper_2512_11800_gb300 import _binding as B
    c = B.AdcConfig()
    assert lib.mb3dgs_adc_config_default(C.byref(c)) == 0
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
    f32 = lambda x: float(C.c_float(x).value)
    assert c.grad_threshold == f32(gold["adc_grad_threshold"]["value"])
    assert c.split_gamma == f32(gold["split_gamma"]["value"]) and c.split_delta == f32(gold["split_delta"]["value"])
    ref = O.adc.ADCConfig()
    for k in ["prune_opacity", "percent_dense", "scene_extent", "big_world"]:
        assert getattr(c, k) == f32(getattr(ref, k)), k
    n = C.c_size_t(0)
    assert lib.mb3dgs_densify_workspace_size(1000, C.byref(n)) == 0 and n.value >= 8000
    assert lib.mb3dgs_densify_workspace_size(-1, C.byref(n)) == -1
    g = B.Gaussians()
    g.P = 10
    out = B.GaussiansOut()
    out.capacity = 19                                   # below 2P
    assert lib.mb3dgs_densify(C.byref(c), C.byref(g), None, None, None, 0, C.byref(out), None, None, None,
                              None) == -1
    bad = B.AdcConfig()
    lib.mb3dgs_adc_config_default(C.byref(bad))
    bad.split_gamma = 1.5
    out.capacity = 20
    assert lib.mb3dgs_densify(C.byref(bad), C.byref(g), None, None, None, 0, C.byref(out), None, None, None,
                              None) == -1
    assert lib.mb3dgs_view_independent_opacity(None, None, 5, None, None) == -1
