"""Adaptive density control between optimiser steps (Sec. 3.4 "Training and
Densification"; App. D "Adaptive Density Control"): argument marshalling for
the mb3dgs_view_independent_opacity, mb3dgs_init_weights,
mb3dgs_accumulate_grad_stats and mb3dgs_densify calls of the C ABI.  Every
step runs in the library's CUDA kernels."""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import torch

from . import _binding as B


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _f32(x):
    if not (x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()):
        raise ValueError("expected a contiguous float32 CUDA tensor")
    return x


@dataclass
class AdcConfig:
    grad_threshold: float = 1e-4        # App. D: 3DGS's 2e-4 reduced to 1e-4
    prune_opacity: float = 0.005        # 3DGS minimum opacity, on the view-independent opacity
    percent_dense: float = 0.01         # clone when max(s) <= percent_dense x extent, else split
    scene_extent: float = 1.0
    big_world: float = 0.1              # prune when max(s) > big_world x extent (0: off)
    split_gamma: float = 0.6385502815246582    # App. D
    split_delta: float = 0.6128153090966912    # App. D

    def to_c(self) -> B.AdcConfig:
        c = B.AdcConfig()
        for k in self.__dataclass_fields__:
            setattr(c, k, float(getattr(self, k)))
        return c


def view_independent_opacity(weights, scales, stream=None):
    """o = 1 - exp(-sqrt(2 pi) w min(s)) per Gaussian (App. D)."""
    lib = B.load()
    w, s = _f32(weights), _f32(scales)
    out = torch.empty_like(w)
    B.check(lib.mb3dgs_view_independent_opacity(_ptr(w), _ptr(s), w.numel(), _ptr(out), _stream(stream)),
            "view_independent_opacity")
    return out


def init_weights(opacity, scales, stream=None):
    """Peak densities w = -log(1 - o) / (sqrt(2 pi) avg(s)) (App. D)."""
    lib = B.load()
    o, s = _f32(opacity), _f32(scales)
    out = torch.empty_like(o)
    B.check(lib.mb3dgs_init_weights(_ptr(o), _ptr(s), o.numel(), _ptr(out), _stream(stream)), "init_weights")
    return out


class DensityStats:
    """Running densification statistics of P Gaussians: the summed absolute
    components of dL/dmean (P, 3) and the number of steps each was visible."""

    def __init__(self, P, device="cuda"):
        self.abs_sum = torch.zeros(P, 3, dtype=torch.float32, device=device)
        self.count = torch.zeros(P, dtype=torch.int32, device=device)

    def accumulate(self, d_means, visible=None, stream=None):
        lib = B.load()
        d = _f32(d_means)
        vis = None
        if visible is not None:
            vis = visible.to(torch.uint8).contiguous()
        B.check(lib.mb3dgs_accumulate_grad_stats(_ptr(d), _ptr(vis), self.abs_sum.shape[0], _ptr(self.abs_sum),
                                                 _ptr(self.count), _stream(stream)), "accumulate_grad_stats")

    def reset(self):
        self.abs_sum.zero_()
        self.count.zero_()


def densify(g, stats: DensityStats, cfg: AdcConfig | None = None, stream=None):
    """Clone / split / prune (mb3dgs_densify).  Returns (GaussianTensors of the
    new set, per-input action int8: 0 kept, 1 cloned, 2 split, per-input index
    of its first output int32: input i's outputs are first[i] .. first[i+1] - 1,
    the map for per-particle optimiser state).  Reads the new count back to the
    host (one synchronisation)."""
    from . import GaussianTensors
    lib = B.load()
    cfg = cfg or AdcConfig()
    P = g.P
    gc = g.to_c()
    dev = g.means.device
    K3 = 3 * (g.sh_degree + 1) ** 2
    cap = max(2 * P, 1)
    out_t = dict(means=torch.empty(cap, 3, device=dev), scales=torch.empty(cap, 3, device=dev),
                 quats=torch.empty(cap, 4, device=dev), weights=torch.empty(cap, device=dev),
                 sh=torch.empty(cap, K3 // 3, 3, device=dev))
    o = B.GaussiansOut()
    o.means, o.scales, o.quats = (out_t[k].data_ptr() for k in ["means", "scales", "quats"])
    o.weights, o.sh = out_t["weights"].data_ptr(), out_t["sh"].data_ptr()
    o.capacity = cap
    nb = C.c_size_t(0)
    B.check(lib.mb3dgs_densify_workspace_size(P, C.byref(nb)), "densify_workspace_size")
    ws = torch.empty(max(int(nb.value), 256), dtype=torch.uint8, device=dev)
    p_out = torch.zeros(1, dtype=torch.int64, device=dev)
    action = torch.empty(max(P, 1), dtype=torch.int8, device=dev)
    first = torch.empty(max(P, 1), dtype=torch.int32, device=dev)
    c = cfg.to_c()
    B.check(lib.mb3dgs_densify(C.byref(c), C.byref(gc), _ptr(stats.abs_sum), _ptr(stats.count), _ptr(ws),
                               ws.numel(), C.byref(o), _ptr(p_out), _ptr(action), _ptr(first), _stream(stream)),
            "densify")
    n = int(p_out.item())
    new = GaussianTensors(*(out_t[k][:n].contiguous() for k in ["means", "scales", "quats", "weights", "sh"]),
                          g.sh_degree)
    return new, action[:P], first[:P]
