"""ctypes declarations of the C ABI in include/mb3dgs.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

c_float3 = C.c_float * 3


class Config(C.Structure):
    _fields_ = [("n", C.c_int), ("n_intervals", C.c_int), ("kappa", C.c_float), ("beta", C.c_float),
                ("conf_c", C.c_float), ("warp_lambda", C.c_float), ("t_near", C.c_float), ("t_far", C.c_float),
                ("eps", C.c_float), ("bias_alpha", C.c_float), ("m_min", C.c_float), ("r_mult", C.c_float),
                ("bg", c_float3), ("moment_dtype", C.c_int), ("strict", C.c_int),
                ("tile_w", C.c_int), ("tile_h", C.c_int), ("batch", C.c_int), ("schedule", C.c_int),
                ("query_capacity", C.c_int64), ("basis", C.c_int), ("trig_theta", C.c_float),
                ("tau_table", C.c_int), ("compact_queries", C.c_int)]


class Gaussians(C.Structure):
    _fields_ = [("means", C.c_void_p), ("scales", C.c_void_p), ("quats", C.c_void_p), ("weights", C.c_void_p),
                ("sh", C.c_void_p), ("P", C.c_int64), ("sh_degree", C.c_int)]


class Camera(C.Structure):
    _fields_ = [("viewmat", C.c_float * 16), ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float),
                ("cy", C.c_float), ("width", C.c_int), ("height", C.c_int)]


class AluPeaks(C.Structure):
    _fields_ = [("fp32_tflops", C.c_double), ("ex2_tops", C.c_double), ("rsqrt_tops", C.c_double),
                ("rcp_tops", C.c_double), ("sin_tops", C.c_double), ("sm_count", C.c_int)]


class GaussianGrads(C.Structure):
    _fields_ = [("means", C.c_void_p), ("scales", C.c_void_p), ("quats", C.c_void_p), ("weights", C.c_void_p),
                ("sh", C.c_void_p)]


class AdcConfig(C.Structure):
    _fields_ = [("grad_threshold", C.c_float), ("prune_opacity", C.c_float), ("percent_dense", C.c_float),
                ("scene_extent", C.c_float), ("big_world", C.c_float), ("split_gamma", C.c_float),
                ("split_delta", C.c_float)]


class GaussiansOut(C.Structure):
    _fields_ = [("means", C.c_void_p), ("scales", C.c_void_p), ("quats", C.c_void_p), ("weights", C.c_void_p),
                ("sh", C.c_void_p), ("capacity", C.c_int64)]


MOMENTS = {"f32": 0, "bf16": 1, "f16": 2}
BASES = {"power": 0, "trig": 1}
SCHEDULES = {"queue": 0, "grid": 1}
STATUS = {0: "ok", -1: "invalid argument", -2: "CUDA error", -3: "workspace too small", -4: "device wait timed out",
          -5: "non-finite Gaussian parameters", -6: "unsupported configuration", -7: "tile-pair capacity exceeded"}

EXPORTS = ["mb3dgs_status_string", "mb3dgs_last_cuda_error", "mb3dgs_config_default", "mb3dgs_workspace_size", "mb3dgs_preprocess",
           "mb3dgs_bin_tiles", "mb3dgs_accumulate_moments", "mb3dgs_reconstruct_transmittance", "mb3dgs_shade",
           "mb3dgs_render", "mb3dgs_render_noalloc", "mb3dgs_backward", "mb3dgs_backward_quadrature",
           "mb3dgs_backward_moments", "mb3dgs_backward_preprocess", "mb3dgs_get_status", "mb3dgs_get_pair_counts", "mb3dgs_autotune", "mb3dgs_debug_tile_lists", "mb3dgs_num_tiles", "mb3dgs_launch_count",
           "mb3dgs_probe_alu_peaks", "mb3dgs_adc_config_default", "mb3dgs_view_independent_opacity",
           "mb3dgs_init_weights", "mb3dgs_accumulate_grad_stats", "mb3dgs_densify_workspace_size", "mb3dgs_densify"]

_lib = None


def _declare(lib):
    P = C.POINTER
    vp, i64, sz = C.c_void_p, C.c_int64, C.c_size_t
    cfg, cam, gs, gg = P(Config), P(Camera), P(Gaussians), P(GaussianGrads)
    sig = {
        "mb3dgs_status_string": (C.c_char_p, [C.c_int]),
        "mb3dgs_last_cuda_error": (C.c_char_p, []),
        "mb3dgs_config_default": (C.c_int, [cfg]),
        "mb3dgs_workspace_size": (C.c_int, [cfg, cam, C.c_int, i64, i64, P(sz)]),
        "mb3dgs_preprocess": (C.c_int, [cfg, gs, cam, C.c_int, vp, sz, i64, vp]),
        "mb3dgs_bin_tiles": (C.c_int, [cfg, cam, C.c_int, i64, i64, vp, sz, vp]),
        "mb3dgs_accumulate_moments": (C.c_int, [cfg, cam, C.c_int, i64, i64, vp, sz, vp, vp]),
        "mb3dgs_reconstruct_transmittance": (C.c_int, [cfg, cam, C.c_int, i64, i64, vp, sz, vp, C.c_int, vp, vp]),
        "mb3dgs_shade": (C.c_int, [cfg, cam, C.c_int, i64, i64, vp, sz, vp, vp, vp, vp]),
        "mb3dgs_render": (C.c_int, [cfg, gs, cam, C.c_int, vp, sz, i64, vp, vp, vp, vp]),
        "mb3dgs_render_noalloc": (C.c_int, [cfg, gs, cam, C.c_int, vp, vp, vp, vp, vp]),
        "mb3dgs_backward": (C.c_int, [cfg, gs, cam, C.c_int, vp, sz, i64, vp, vp, vp, gg, vp]),
        "mb3dgs_backward_quadrature": (C.c_int, [cfg, cam, C.c_int, i64, i64, vp, sz, vp, vp, vp, vp]),
        "mb3dgs_backward_moments": (C.c_int, [cfg, cam, C.c_int, i64, i64, vp, sz, vp]),
        "mb3dgs_backward_preprocess": (C.c_int, [cfg, gs, cam, C.c_int, vp, sz, i64, gg, vp]),
        "mb3dgs_get_status": (C.c_int, [vp, sz, P(C.c_int), P(i64), vp]),
        "mb3dgs_get_pair_counts": (C.c_int, [vp, sz, P(i64), P(i64), vp]),
        "mb3dgs_autotune": (C.c_int, [cfg, gs, cam, C.c_int, vp, sz, vp, vp, vp, gg, P(C.c_float), vp]),
        "mb3dgs_debug_tile_lists": (C.c_int, [cfg, cam, C.c_int, i64, i64, vp, sz, vp, vp, vp, vp]),
        "mb3dgs_num_tiles": (i64, [cfg, cam, C.c_int]),
        "mb3dgs_launch_count": (i64, []),
        "mb3dgs_probe_alu_peaks": (C.c_int, [P(AluPeaks), vp]),
        "mb3dgs_adc_config_default": (C.c_int, [P(AdcConfig)]),
        "mb3dgs_view_independent_opacity": (C.c_int, [vp, vp, i64, vp, vp]),
        "mb3dgs_init_weights": (C.c_int, [vp, vp, i64, vp, vp]),
        "mb3dgs_accumulate_grad_stats": (C.c_int, [vp, vp, i64, vp, vp, vp]),
        "mb3dgs_densify_workspace_size": (C.c_int, [i64, P(sz)]),
        "mb3dgs_densify": (C.c_int, [P(AdcConfig), gs, vp, vp, vp, sz, P(GaussiansOut), vp, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


def library_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load libmb3dgs.so (building it with nvcc if missing or stale).  Raises if
    the library cannot be built or loaded: there is no fallback path."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError("libmb3dgs.so is not built (run paper_2512_11800_gb300/build.py)")
    _lib = _declare(C.CDLL(_build.LIB))
    return _lib


def check(rc, what=""):
    if rc != 0:
        extra = ""
        if rc == -2 and _lib is not None:
            extra = ": " + _lib.mb3dgs_last_cuda_error().decode()
        raise RuntimeError("mb3dgs %s failed: %s (%d)%s" % (what, STATUS.get(rc, "unknown"), rc, extra))
