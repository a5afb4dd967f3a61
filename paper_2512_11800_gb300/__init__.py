"""GB300-native moment-based Gaussian rasterizer (MB3DGS hot path).

Thin Python layer over the C ABI of ``include/mb3dgs.h``: it only marshals
arguments, owns device memory through PyTorch tensors and passes PyTorch's
current CUDA stream.  Every step of the rendering path runs in the sm_103a
kernels of ``libmb3dgs.so``; if the library cannot be loaded the import of
the rendering functions raises (there is no CPU or PyTorch fallback).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _binding as B

__all__ = ["RasterConfig", "GaussianTensors", "Rasterizer", "to_camera", "load_library", "render", "adc"]


def load_library():
    return B.load()


@dataclass
class RasterConfig:
    n: int = 4
    n_intervals: int = 3
    kappa: float = 3.0
    beta: float = 0.25
    conf_c: float = 0.01
    warp_lambda: float = -1.5
    t_near: float = 0.01
    t_far: float = 1.0e6
    eps: float = 1.0e-6
    bias_alpha: float = 1.0e-3
    m_min: float = 1.0e-7
    r_mult: float = 3.0
    bg: tuple = (0.0, 0.0, 0.0)
    moment_dtype: str = "f32"
    strict: int = 0
    # keep every pair's bound queries from the forward for the backward
    # (64 B per (pixel, Gaussian) pair at N = 3); False: backward recomputes them
    save_queries: bool = True
    query_budget_gb: float = 48.0  # device memory for kept queries; pixels beyond it recompute theirs
    # kept-query form: "full" (16 B a query) or "compact" (8 B: roots as 16-bit
    # positions in their brackets, restored by one Laguerre step in the
    # backward; twice the pairs in the same memory, but the restore costs more
    # than solving the remaining pixels' queries again at the 16-view frame's
    # 57 % kept fraction)
    query_format: str = "full"
    # execution shape (results do not depend on it; Rasterizer.autotune sets it)
    tile_w: int = 16
    tile_h: int = 16
    batch: int = 256
    schedule: str = "queue"        # "queue" | "grid"
    # moment basis: "power" (Eq. 10-12) or "trig" (Eq. 13-14)
    basis: str = "power"
    trig_theta: float = 0.5 * np.pi   # wrapping angle of the trigonometric moments
    # tabulated transmittance: M knots a segment, 0 = solve every query (the backward
    # differentiates the solved bounds the table approximates)
    tau_table: int = 0

    def to_c(self) -> B.Config:
        c = B.Config()
        for f in ["n", "n_intervals", "strict", "tile_w", "tile_h", "batch"]:
            setattr(c, f, int(getattr(self, f)))
        for f in ["kappa", "beta", "conf_c", "warp_lambda", "t_near", "t_far", "eps", "bias_alpha", "m_min", "r_mult"]:
            setattr(c, f, float(getattr(self, f)))
        c.bg = B.c_float3(*[float(x) for x in self.bg])
        c.moment_dtype = B.MOMENTS[self.moment_dtype]
        c.schedule = B.SCHEDULES[self.schedule]
        c.basis = B.BASES[self.basis]
        c.trig_theta = float(self.trig_theta)
        c.tau_table = int(self.tau_table)
        return c


@dataclass
class GaussianTensors:
    """Float32 CUDA tensors: means (P,3), scales (P,3), quats (P,4), weights (P,), sh (P,K,3)."""
    means: torch.Tensor
    scales: torch.Tensor
    quats: torch.Tensor
    weights: torch.Tensor
    sh: torch.Tensor
    sh_degree: int

    @property
    def P(self):
        return int(self.means.shape[0])

    @staticmethod
    def from_scene(scene, device="cuda"):
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=device)
        return GaussianTensors(t(scene.means), t(scene.scales), t(scene.quats), t(scene.weights), t(scene.sh),
                               int(scene.sh_degree))

    def to_c(self) -> B.Gaussians:
        for name in ["means", "scales", "quats", "weights", "sh"]:
            x = getattr(self, name)
            if not (x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()):
                raise ValueError("%s must be a contiguous float32 CUDA tensor" % name)
        g = B.Gaussians()
        g.means, g.scales, g.quats = self.means.data_ptr(), self.scales.data_ptr(), self.quats.data_ptr()
        g.weights, g.sh = self.weights.data_ptr(), self.sh.data_ptr()
        g.P = self.P
        g.sh_degree = int(self.sh_degree)
        return g


def to_camera(cam) -> B.Camera:
    """Any object with viewmat (4x4), fx, fy, cx, cy, width, height."""
    c = B.Camera()
    vm = np.asarray(cam.viewmat, dtype=np.float32).reshape(16)
    c.viewmat = (C.c_float * 16)(*vm.tolist())
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height = int(cam.width), int(cam.height)
    return c


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class Rasterizer:
    """Renders Gaussians through the C ABI.  Holds a reusable workspace."""

    def __init__(self, config: RasterConfig | None = None, device="cuda"):
        self.lib = B.load()
        self.config = config or RasterConfig()
        self.cfg_c = self.config.to_c()
        self.device = torch.device(device)
        self._ws = None
        self._last_qcap = 0
        self.generation = 0   # renders so far: the workspace holds the last one's state

    # ------------------------------------------------------------ plumbing
    def cameras(self, cams):
        cams = list(cams) if isinstance(cams, (list, tuple)) else [cams]
        arr = (B.Camera * len(cams))(*[to_camera(c) for c in cams])
        return arr, len(cams)

    def workspace_bytes(self, cams, P, capacity):
        arr, nv = self.cameras(cams)
        n = C.c_size_t(0)
        B.check(self.lib.mb3dgs_workspace_size(C.byref(self.cfg_c), arr, nv, int(P), int(capacity), C.byref(n)),
                "workspace_size")
        return int(n.value)

    def workspace(self, nbytes):
        if self._ws is None or self._ws.numel() < nbytes:
            self._ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
        return self._ws

    def num_pixels(self, cams):
        cams = list(cams) if isinstance(cams, (list, tuple)) else [cams]
        return sum(int(c.width) * int(c.height) for c in cams)

    def num_tiles(self, cams):
        arr, nv = self.cameras(cams)
        return int(self.lib.mb3dgs_num_tiles(C.byref(self.cfg_c), arr, nv))

    def status(self, stream=None):
        st = C.c_int(0)
        n = C.c_int64(0)
        B.check(self.lib.mb3dgs_get_status(_ptr(self._ws), self._ws.numel(), C.byref(st), C.byref(n),
                                           _stream(stream)), "get_status")
        return int(st.value), int(n.value)

    # ------------------------------------------------------------ API
    def pair_counts(self, g: GaussianTensors, cams, stream=None):
        """((tile, Gaussian) pairs, (pixel, Gaussian) pairs) of this frame:
        preprocess + binning with zero capacities, then one host read."""
        arr, nv = self.cameras(cams)
        self.cfg_c.query_capacity = 0
        ws = self.workspace(self.workspace_bytes(cams, g.P, 0))
        gc = g.to_c()
        s = _stream(stream)
        self.generation += 1
        B.check(self.lib.mb3dgs_preprocess(C.byref(self.cfg_c), C.byref(gc), arr, nv, _ptr(ws), ws.numel(), 0, s),
                "preprocess")
        B.check(self.lib.mb3dgs_bin_tiles(C.byref(self.cfg_c), arr, nv, g.P, 0, _ptr(ws), ws.numel(), s), "bin_tiles")
        tp, pp = C.c_int64(0), C.c_int64(0)
        B.check(self.lib.mb3dgs_get_pair_counts(_ptr(ws), ws.numel(), C.byref(tp), C.byref(pp), _stream(stream)),
                "get_pair_counts")
        return int(tp.value), int(pp.value)

    def count_pairs(self, g: GaussianTensors, cams, stream=None):
        """(tile, Gaussian) pairs of this frame (the pair capacity it needs)."""
        return self.pair_counts(g, cams, stream)[0]

    def autotune(self, g: GaussianTensors, cams, backward=True, stream=None):
        """Times the frame under each execution shape (tile shape, batch,
        schedule) and keeps the fastest (mb3dgs_autotune); the images do not
        depend on it.  Returns (tile_w, tile_h, batch, schedule, ms)."""
        arr, nv = self.cameras(cams)
        shapes = [(16, 16), (32, 8), (8, 32)]
        need, qcap = 0, 0
        for tw, th in shapes:
            self.cfg_c.tile_w, self.cfg_c.tile_h = tw, th
            tp, pp = self.pair_counts(g, cams, stream)
            qcap = self.set_query_capacity(pp)
            need = max(need, self.workspace_bytes(cams, g.P, tp))
        ws = self.workspace(need)
        self.generation += 1
        npix = self.num_pixels(cams)
        rgb = torch.empty(npix, 3, device=self.device)
        T = torch.empty(npix, device=self.device)
        gc = g.to_c()
        dl, gg = None, None
        if backward:
            dl = torch.full((npix, 3), 1.0 / (3 * npix), device=self.device)
            grads = {k: torch.empty_like(getattr(g, k)) for k in ["means", "scales", "quats", "weights", "sh"]}
            gg = B.GaussianGrads()
            gg.means, gg.scales, gg.quats = grads["means"].data_ptr(), grads["scales"].data_ptr(), grads["quats"].data_ptr()
            gg.weights, gg.sh = grads["weights"].data_ptr(), grads["sh"].data_ptr()
        ms = C.c_float(0.0)
        B.check(self.lib.mb3dgs_autotune(C.byref(self.cfg_c), C.byref(gc), arr, nv, _ptr(ws), ws.numel(), _ptr(rgb),
                                         _ptr(T), _ptr(dl), C.byref(gg) if gg is not None else None, C.byref(ms),
                                         _stream(stream)), "autotune")
        c = self.cfg_c
        self.config.tile_w, self.config.tile_h, self.config.batch = int(c.tile_w), int(c.tile_h), int(c.batch)
        self.config.schedule = {v: k for k, v in B.SCHEDULES.items()}[int(c.schedule)]
        return self.config.tile_w, self.config.tile_h, self.config.batch, self.config.schedule, float(ms.value)

    def set_query_capacity(self, n):
        """Query slots of the following calls for a frame of n pixel pairs:
        as many as the budget holds (0 without saved queries: the backward
        solves every query again; pixels beyond the slots do so too)."""
        n = int(n)
        nq = self.config.n_intervals + 1
        room = int(self.config.query_budget_gb * 2 ** 30)
        fmt = self.config.query_format
        if fmt not in ("full", "compact"):
            raise ValueError("query_format must be full or compact")
        compact = fmt == "compact" and self.config.basis == "power"
        self.cfg_c.compact_queries = 1 if compact else 0
        budget = room // ((8 if compact else 16) * nq)
        keep = self.config.save_queries and not self.config.tau_table
        self.cfg_c.query_capacity = min(n, budget) if keep else 0
        return int(self.cfg_c.query_capacity)

    def render(self, g: GaussianTensors, cams, capacity=None, stream=None, penalty=True, out=None,
               query_capacity=None):
        """Full forward (mb3dgs_render).  Returns dict(rgb (Npix,3), T (Npix,),
        penalty (Npix,)) over the concatenated views.  Without ``capacity`` (and,
        when queries are saved, ``query_capacity``) one counting pass with a
        host read sizes the frame."""
        arr, nv = self.cameras(cams)
        if capacity is None or (query_capacity is None and self.config.save_queries):
            tp, pp = self.pair_counts(g, cams, stream)
            capacity = tp if capacity is None else capacity
            query_capacity = pp if query_capacity is None else query_capacity
        qcap = self.set_query_capacity(query_capacity or 0)
        nbytes = self.workspace_bytes(cams, g.P, capacity)
        ws = self.workspace(nbytes)
        npix = self.num_pixels(cams)
        if out is None:
            out = dict(rgb=torch.empty(npix, 3, device=self.device), T=torch.empty(npix, device=self.device),
                       penalty=torch.empty(npix, device=self.device) if penalty else None)
        gc = g.to_c()
        self.generation += 1
        B.check(self.lib.mb3dgs_render(C.byref(self.cfg_c), C.byref(gc), arr, nv, _ptr(ws), ws.numel(), int(capacity),
                                       _ptr(out["rgb"]), _ptr(out["T"]), _ptr(out.get("penalty")), _stream(stream)),
                "render")
        out["capacity"] = int(capacity)
        out["query_capacity"] = qcap
        self._last_qcap = qcap
        return out

    def render_staged(self, g: GaussianTensors, cams, capacity=None, eta=None, stream=None):
        """The five stage calls one by one; also returns the power moments
        (Npix, 9), the transmittance at the warped depths ``eta`` (Npix, Q) and
        the tile lists for inspection."""
        arr, nv = self.cameras(cams)
        if capacity is None:
            capacity = self.count_pairs(g, cams, stream)
        self.set_query_capacity(0)
        ws = self.workspace(self.workspace_bytes(cams, g.P, capacity))
        self.generation += 1
        npix = self.num_pixels(cams)
        s = _stream(stream)
        cfg = C.byref(self.cfg_c)
        gc = g.to_c()
        P = g.P
        B.check(self.lib.mb3dgs_preprocess(cfg, C.byref(gc), arr, nv, _ptr(ws), ws.numel(), int(capacity), s),
                "preprocess")
        B.check(self.lib.mb3dgs_bin_tiles(cfg, arr, nv, P, int(capacity), _ptr(ws), ws.numel(), s), "bin_tiles")
        mom = torch.empty(npix, 9, device=self.device)
        B.check(self.lib.mb3dgs_accumulate_moments(cfg, arr, nv, P, int(capacity), _ptr(ws), ws.numel(), _ptr(mom), s),
                "accumulate_moments")
        Tq = None
        Q = 0
        if eta is not None:
            eta = eta.contiguous().float()
            Q = int(eta.shape[1])
            Tq = torch.empty(npix, Q, device=self.device)
        B.check(self.lib.mb3dgs_reconstruct_transmittance(cfg, arr, nv, P, int(capacity), _ptr(ws), ws.numel(),
                                                          _ptr(eta), Q, _ptr(Tq), s), "reconstruct")
        rgb = torch.empty(npix, 3, device=self.device)
        T = torch.empty(npix, device=self.device)
        pen = torch.empty(npix, device=self.device)
        B.check(self.lib.mb3dgs_shade(cfg, arr, nv, P, int(capacity), _ptr(ws), ws.numel(), _ptr(rgb), _ptr(T),
                                      _ptr(pen), s), "shade")
        ntiles = self.num_tiles(cams)
        ids = torch.empty(max(int(capacity), 1), dtype=torch.int32, device=self.device)
        ranges = torch.empty(ntiles, 2, dtype=torch.int32, device=self.device)
        rects = torch.empty(nv * P, 4, dtype=torch.int32, device=self.device)
        B.check(self.lib.mb3dgs_debug_tile_lists(cfg, arr, nv, P, int(capacity), _ptr(ws), ws.numel(), _ptr(ids),
                                                 _ptr(ranges), _ptr(rects), s), "debug_tile_lists")
        return dict(rgb=rgb, T=T, penalty=pen, moments=mom, T_eta=Tq, ids=ids[:capacity], ranges=ranges, rects=rects,
                    capacity=int(capacity))

    def backward(self, g: GaussianTensors, cams, capacity, dL_drgb, dL_dP=None, stream=None, grads=None,
                 query_capacity=None, dL_dT=None):
        """Adjoint of the last ``render`` (same Gaussians, cameras, capacity and
        query capacity, by default the last render's): gradients of
        sum(dL_drgb * rgb) + sum(dL_dP * penalty) + sum(dL_dT * T) with respect
        to the Gaussian parameters (mb3dgs_backward)."""
        arr, nv = self.cameras(cams)
        self.set_query_capacity(self._last_qcap if query_capacity is None else query_capacity)
        ws = self._ws
        if grads is None:
            grads = {k: torch.empty_like(getattr(g, k)) for k in ["means", "scales", "quats", "weights", "sh"]}
        gc = g.to_c()
        gg = B.GaussianGrads()
        gg.means, gg.scales, gg.quats = grads["means"].data_ptr(), grads["scales"].data_ptr(), grads["quats"].data_ptr()
        gg.weights, gg.sh = grads["weights"].data_ptr(), grads["sh"].data_ptr()
        dL_drgb = dL_drgb.contiguous().float()
        if dL_dP is not None:
            dL_dP = dL_dP.contiguous().float()
        if dL_dT is not None:
            dL_dT = dL_dT.contiguous().float()
        B.check(self.lib.mb3dgs_backward(C.byref(self.cfg_c), C.byref(gc), arr, nv, _ptr(ws), ws.numel(),
                                         int(capacity), _ptr(dL_drgb), _ptr(dL_dP), _ptr(dL_dT), C.byref(gg),
                                         _stream(stream)),
                "backward")
        return grads


class _RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rast, cams, sh_degree, means, scales, quats, weights, sh):
        g = GaussianTensors(means.contiguous(), scales.contiguous(), quats.contiguous(), weights.contiguous(),
                            sh.contiguous(), sh_degree)
        out = rast.render(g, cams)
        ctx.rast, ctx.cams, ctx.g, ctx.capacity, ctx.qcap = rast, cams, g, out["capacity"], out["query_capacity"]
        ctx.generation = rast.generation
        return out["rgb"], out["T"], out["penalty"]

    @staticmethod
    def backward(ctx, d_rgb, d_T, d_pen):
        if ctx.rast.generation != ctx.generation:
            raise RuntimeError("the Rasterizer rendered again after this forward: its workspace no longer holds "
                               "this forward's state; use one Rasterizer per pending backward")
        if d_rgb is None:
            d_rgb = torch.zeros(ctx.rast.num_pixels(ctx.cams), 3, device=ctx.rast.device)
        grads = ctx.rast.backward(ctx.g, ctx.cams, ctx.capacity, d_rgb, d_pen, query_capacity=ctx.qcap, dL_dT=d_T)
        return None, None, None, grads["means"], grads["scales"], grads["quats"], grads["weights"], grads["sh"]


def render(rast: "Rasterizer", cams, means, scales, quats, weights, sh, sh_degree):
    """Differentiable render: returns (rgb [Npix,3], T [Npix], penalty [Npix]);
    all three are differentiable (T = e^{-m0} through the total optical depth).
    Backward runs the adjoint passes of mb3dgs_backward; it raises if the same
    Rasterizer rendered again in between (its workspace holds one forward)."""
    return _RenderFn.apply(rast, cams, sh_degree, means, scales, quats, weights, sh)


from . import adc  # noqa: E402  (adaptive density control, Sec. 3.4 / App. D)
