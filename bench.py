"""Benchmark of the moment-based Gaussian rasterizer on one GB300.

Default workload: the 1,000,000-Gaussian scene (64 anisotropic clusters +
interpenetrating low-density shells, SH degree 3) at 1920x1080.  One step =
the whole hot path: preprocess -> tile binning -> moment pass -> per-pixel
reconstruction -> quadrature pass -> L2-loss gradient against a random
target -> backward (quadrature/bound adjoint, moment adjoint, preprocessing
adjoint).  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--forward-only] [--workload shells1M_1080p|batch16|adc]

--workload batch16: the same scene seen by 16 views of uneven resolution
(640x360 / 1280x720 / 1920x1080), the whole fwd+bwd step captured in one
CUDA graph and replayed, next to 16 sequential single-view render+backward
calls (--batch16-frames F: F frames of 16/F views one after the other in the
graph).  --workload adc: one adaptive-density-control step on the scene's 1M
Gaussians (gradient statistics, then clone / split / prune).  The default
line carries short records of both, batch16 as one frame and as two.

With N > 1 (launched by torchrun) every rank renders its own replica of the
workload (the path has no data exchange); rank 0 prints the aggregate.
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import scenes  # noqa: E402

WORKLOAD = "shells1M_1080p"
METRIC = "Mpixel/s fwd and fwd+bwd, 1M Gaussians @1080p; fraction of roofline; err vs FP64"
# Algorithmic work per unit of each per-pair kernel: the operations the
# method itself needs, counted from its formulas (not this build's executed
# instructions).  FP32 flops (an FMA counts 2) and MUFU special-function
# operations.  Unit: the (pixel, Gaussian) pair with the pixel centre inside
# the Gaussian's proxy rectangle.
#   quadrature pass, N intervals (N+1 samples):
#     40 flop + 4 MUFU per pair: the ray-parameterised 1D Gaussian (Eq. 4-6:
#       d_g, o_g.d_g, |d_g|^2, Sigma, mu, w-hat) and the colour sums;
#     250 flop + 12 MUFU per sample: the depth warp (10), the bound query of
#       Eq. 8 -- orthogonal-polynomial values and kernel coefficients at eta
#       (30), the Christoffel weight of eta (10), two roots of the degree-4
#       kernel polynomial by four Laguerre steps each (160) and their weights
#       (30) -- and the interval's quadrature and penalty terms (Eq. 7,
#       App. D; 10);
#   moment pass: 70 flop + 6 MUFU per pair (Eq. 4-6 and the nine-moment
#     recurrence of Eq. 10-12);
#   adjoint passes: twice their forward counterparts (reverse mode costs at
#     least the forward arithmetic again).
def alg_ops(kernel, n_intervals):
    """(FP32 flops, MUFU ops) per pixel pair of the method's work."""
    q = n_intervals + 1
    shade = (40 + 250 * q, 4 + 12 * q)
    moments = (70, 6)
    return {"k_shade": shade, "k_bwd_quadrature": (2 * shade[0], 2 * shade[1]),
            "k_moments": moments, "k_bwd_moments": (2 * moments[0], 2 * moments[1])}[kernel]


# Executed work of the current kernels from ncu captures on the 200k/720p
# workload (per pixel pair): FP32 flops = FADD + FMUL + 2 FFMA thread
# instructions, all thread instructions, and DRAM bytes (read + write; the
# kept bound queries dominate).  Scaled to a launch by its pairs.
EXECUTED_PER_PAIR = {
    "k_shade": dict(flops=1014.6, thread_inst=1613.6, dram_bytes=76.7),
    "k_bwd_quadrature": dict(flops=1135.7, thread_inst=1590.8, dram_bytes=70.5),
}
# MUFU (XU) pipe utilisation of the same captures (ncu
# sm__inst_executed_pipe_xu.avg.pct_of_peak_sustained_active / 100).
XU_PIPE_FRAC = {"k_shade": 0.105, "k_bwd_quadrature": 0.052}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            dev = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[torch.cuda.current_device()]
            self.proc = subprocess.Popen(["nvidia-smi", "-i", dev, "--query-gpu=" + q, "--format=csv,noheader,nounits",
                                          "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(n_gpus):
    if n_gpus > 1 or int(os.environ.get("WORLD_SIZE", "1")) > 1:
        import torch.distributed as dist
        local = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
        return dist, dist.get_rank(), dist.get_world_size()
    return None, 0, 1


def max_over_ranks(dist, ms, device):
    """The slowest rank's step time (every rank gets it)."""
    if not dist:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mpix_s(world, pixels_per_rank, ms):
    """Whole-job throughput of N replicas: all ranks' pixels over the slowest rank's time."""
    return world * pixels_per_rank / (ms * 1e-3) / 1e6


def oracle_step(sc, cam, size, with_bwd, target, basis="power", n_intervals=3):
    """One oracle step on a centred size x size crop: forward, or forward +
    gradient of the L2 loss against the target crop (autograd in FP64)."""
    import oracle as O
    cfg = O.OracleConfig(basis=basis, n_intervals=n_intervals)
    x0, y0 = (cam.width - size) // 2, (cam.height - size) // 2
    region = (x0, y0, size, size)
    if not with_bwd:
        return O.render(sc, cam, cfg, region=region)["n_pairs"]
    # d/drgb of mean((rgb - target)^2) over the full frame, restricted to the crop
    rgb = O.render(sc, cam, cfg, region=region)["rgb"].numpy()
    tg = target.reshape(cam.height, cam.width, 3)[y0:y0 + size, x0:x0 + size]
    g = 2.0 * (rgb - tg) / (cam.width * cam.height * 3)
    return O.render_grad(sc, cam, cfg, g, None, region=region)["out"]["n_pairs"]


def cpu_oracle_sample(sc, cam, with_bwd, size=32, name=WORKLOAD, basis="power", n_intervals=3):
    """Time the FP64 oracle on a centred crop of the same workload (bounded sample)."""
    torch.set_num_threads(os.cpu_count() or 1)
    target = scenes.target_image(cam.height, cam.width)
    t0 = time.perf_counter()
    n_pairs = oracle_step(sc, cam, size, with_bwd, target, basis, n_intervals)
    dt = time.perf_counter() - t0
    return dict(value=size * size / dt / 1e6, unit="Mpixel/s", cores=torch.get_num_threads(), kind="oracle",
                sample="centre %dx%d crop of the %dx%d frame of %s (%d pixel pairs), %s, %.1f s" %
                       (size, size, cam.width, cam.height, name, n_pairs,
                        "forward+backward" if with_bwd else "forward", dt))


def run_reference(args):
    """--impl reference: the FP64 CPU oracle timed on a bounded sample per step."""
    if int(os.environ.get("RANK", "0")) != 0:
        return
    torch.set_num_threads(os.cpu_count() or 1)
    sc, cam = scenes.workload(WORKLOAD)
    target = scenes.target_image(cam.height, cam.width)
    size = 16
    with_bwd = not args.forward_only
    for _ in range(args.warmup):
        oracle_step(sc, cam, size, with_bwd, target)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_step(sc, cam, size, with_bwd, target)
    dt = (time.perf_counter() - t0) / args.steps
    val = size * size / dt / 1e6
    what = "forward+backward" if with_bwd else "forward"
    line = dict(metric=METRIC, value=val, unit="Mpixel/s", impl="reference", n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=dt * 1e3, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic",
                config={"workload": WORKLOAD + " (centre %dx%d crop per step)" % (size, size),
                        "gaussians": 1_000_000, "width": 1920, "height": 1080, "pass": what},
                cpu_baseline=dict(kind="oracle", cores=torch.get_num_threads(), value=val, unit="Mpixel/s",
                                  sample="centre %dx%d crop per step, %s" % (size, size, what)),
                e2e=dict(value=val, unit="Mpixel/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line))


def probe_peaks(dev):
    """Measured FP32 FMA and MUFU throughput of this GPU (library probe)."""
    from paper_2512_11800_gb300 import _binding as B
    lib = B.load()
    pk = B.AluPeaks()
    B.check(lib.mb3dgs_probe_alu_peaks(C.byref(pk), C.c_void_p(torch.cuda.current_stream(dev).cuda_stream)),
            "probe_alu_peaks")
    return dict(fp32_tflops=pk.fp32_tflops, ex2_tops=pk.ex2_tops, rsqrt_tops=pk.rsqrt_tops, rcp_tops=pk.rcp_tops,
                sin_tops=pk.sin_tops, sm_count=pk.sm_count)


def roofline(kernel, ms, pairs, n_intervals, peaks, sm_mhz, captured=True):
    """ALU roofline of one per-pair kernel from its CUDA-event time.
    frac = algorithmic FP32 flops / time over the measured FP32 peak;
    frac_xu = algorithmic MUFU ops / time over the measured MUFU rate of the
    slower non-exponential kinds (rsqrt, rcp); issue_frac = executed thread
    instructions (ncu) / time over SMs x 4 schedulers x 32 lanes x the SM
    clock sampled during the timed steps.  captured=False: the launch is a
    variant without an ncu capture of its own (k_shade keeping no queries),
    so traffic is null."""
    flops, mufu = alg_ops(kernel, n_intervals)
    ex = EXECUTED_PER_PAIR[kernel]
    sec = ms * 1e-3
    achieved = flops * pairs / sec / 1e12
    mufu_peak = min(peaks["rsqrt_tops"], peaks["rcp_tops"])
    issue_peak = peaks["sm_count"] * 4 * 32 * sm_mhz * 1e6
    return dict(kernel=kernel, bound="alu", achieved=achieved, peak=peaks["fp32_tflops"], unit="TFLOP/s",
                frac=achieved / peaks["fp32_tflops"],
                traffic=ex["dram_bytes"] * pairs if captured else None,
                frac_fp32_algorithmic=achieved / peaks["fp32_tflops"],
                frac_xu=mufu * pairs / sec / 1e12 / mufu_peak,
                issue_frac=ex["thread_inst"] * pairs / sec / issue_peak,
                frac_fp32_executed=ex["flops"] * pairs / sec / 1e12 / peaks["fp32_tflops"],
                xu_pipe_frac_ncu=XU_PIPE_FRAC[kernel],
                alg_flops_per_pair=flops, alg_mufu_per_pair=mufu, sm_count=peaks["sm_count"],
                peak_note="peak = measured FP32 FMA throughput of this GPU (library probe, 2 flop per FFMA); "
                          "achieved = the method's FP32 flops per pixel pair (op model in bench.py) x pairs / "
                          "kernel time; frac_xu against the measured rsqrt/rcp MUFU rate; issue_frac and "
                          "frac_fp32_executed from ncu per-pair counts of the kernel on the 200k/720p "
                          "workload; traffic = ncu DRAM bytes per pair x pairs")


class Frame:
    """Device buffers and the C-ABI stage calls of one frame (one or more views)."""

    def __init__(self, R, g, cams, target, ws=None, save_queries=True):
        from paper_2512_11800_gb300 import _binding as B
        self.B, self.R, self.g, self.cams = B, R, g, cams
        self.cap, qcap = R.pair_counts(g, cams)
        qcap = qcap if save_queries else 0      # a forward-only step keeps no queries
        self.qcap = R.set_query_capacity(qcap)
        nbytes = R.workspace_bytes(cams, g.P, self.cap)
        if ws is not None:          # a shared workspace (frames run one after the other)
            assert ws.numel() >= nbytes
            R._ws = ws
        out = R.render(g, cams, capacity=self.cap, query_capacity=qcap)
        self.arr, self.nv = R.cameras(cams)
        self.ws = R.workspace(nbytes)
        self.gc = g.to_c()
        self.rgb, self.T, self.pen = out["rgb"], out["T"], out["penalty"]
        self.target = target
        self.dl = torch.empty_like(self.rgb)
        self.grads = {k: torch.empty_like(getattr(g, k)) for k in ["means", "scales", "quats", "weights", "sh"]}
        gg = B.GaussianGrads()
        gg.means, gg.scales, gg.quats = (self.grads[k].data_ptr() for k in ["means", "scales", "quats"])
        gg.weights, gg.sh = self.grads["weights"].data_ptr(), self.grads["sh"].data_ptr()
        self.gg = gg

    def step(self, stream, with_bwd, ev=None):
        B, R, lib = self.B, self.R, self.R.lib
        R.set_query_capacity(self.qcap)
        s = C.c_void_p(stream.cuda_stream)
        cfg = C.byref(R.cfg_c)
        wsp, wsn, cap, P = C.c_void_p(self.ws.data_ptr()), self.ws.numel(), self.cap, self.g.P
        rec = (lambda i: ev[i].record(stream)) if ev is not None else (lambda i: None)
        rec(0)
        B.check(lib.mb3dgs_preprocess(cfg, C.byref(self.gc), self.arr, self.nv, wsp, wsn, cap, s), "preprocess")
        B.check(lib.mb3dgs_bin_tiles(cfg, self.arr, self.nv, P, cap, wsp, wsn, s), "bin")
        rec(1)
        B.check(lib.mb3dgs_accumulate_moments(cfg, self.arr, self.nv, P, cap, wsp, wsn, None, s), "moments")
        rec(2)
        B.check(lib.mb3dgs_reconstruct_transmittance(cfg, self.arr, self.nv, P, cap, wsp, wsn, None, 0, None, s),
                "recon")
        rec(3)
        B.check(lib.mb3dgs_shade(cfg, self.arr, self.nv, P, cap, wsp, wsn, C.c_void_p(self.rgb.data_ptr()),
                                 C.c_void_p(self.T.data_ptr()), C.c_void_p(self.pen.data_ptr()), s), "shade")
        rec(4)
        if with_bwd:
            # L2 loss against the target image (the loss itself is the caller's)
            torch.sub(self.rgb, self.target, out=self.dl).mul_(2.0 / self.rgb.numel())
            B.check(lib.mb3dgs_backward_quadrature(cfg, self.arr, self.nv, P, cap, wsp, wsn,
                                                   C.c_void_p(self.dl.data_ptr()), None, None, s),
                    "backward_quadrature")
            rec(5)
            B.check(lib.mb3dgs_backward_moments(cfg, self.arr, self.nv, P, cap, wsp, wsn, s), "backward_moments")
            rec(6)
            B.check(lib.mb3dgs_backward_preprocess(cfg, C.byref(self.gc), self.arr, self.nv, wsp, wsn, cap,
                                                   C.byref(self.gg), s), "backward_preprocess")
        else:
            rec(5)
            rec(6)
        rec(7)


STAGES = ["preprocess+bin", "moments", "reconstruct", "shade", "bwd_quadrature", "bwd_moments", "bwd_preprocess"]


def pair_counts(R, frame):
    st, _ = R.status()
    tp, pp = C.c_int64(0), C.c_int64(0)
    frame.B.check(R.lib.mb3dgs_get_pair_counts(C.c_void_p(frame.ws.data_ptr()), frame.ws.numel(), C.byref(tp),
                                               C.byref(pp), C.c_void_p(torch.cuda.current_stream().cuda_stream)),
                  "pair_counts")
    return st, int(tp.value), int(pp.value)


def run_single(args, dist, rank, world, dev):
    from paper_2512_11800_gb300 import GaussianTensors, RasterConfig, Rasterizer
    sc, cam = scenes.workload(args.workload)
    npix = cam.width * cam.height
    R = Rasterizer(RasterConfig(basis=args.basis, n_intervals=args.n_intervals, moment_dtype=args.moment_dtype,
                                tau_table=args.tau_table), device=dev)
    g = GaussianTensors.from_scene(sc, dev)
    target = torch.as_tensor(scenes.target_image(cam.height, cam.width).reshape(-1, 3), device=dev)
    with_bwd = not args.forward_only
    if with_bwd:
        # kept bound queries in up to 60 % of the free device memory (the 3M
        # frame needs 70 GB of them; the library's default budget is 48 GB)
        tp0, _ = R.pair_counts(g, cam)
        R.set_query_capacity(0)
        base = R.workspace_bytes(cam, g.P, tp0)
        torch.cuda.empty_cache()
        R.config.query_budget_gb = max(R.config.query_budget_gb,
                                       0.6 * (torch.cuda.mem_get_info(dev)[0] - base) / 2 ** 30)
    fr = Frame(R, g, cam, target, save_queries=with_bwd)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        fr.step(stream, with_bwd)
    torch.cuda.synchronize()
    peaks = probe_peaks(dev)
    clocks = ClockSampler()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    l0 = R.lib.mb3dgs_launch_count()
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(8)] for _ in range(args.steps)]
    t_start.record(stream)
    for k in range(args.steps):
        fr.step(stream, with_bwd, evs[k])
    t_end.record(stream)
    torch.cuda.synchronize()
    launches = R.lib.mb3dgs_launch_count() - l0
    clk = clocks.stop()
    ms = t_start.elapsed_time(t_end) / args.steps
    stage_ms = {name: statistics.median(e[i].elapsed_time(e[i + 1]) for e in evs) for i, name in enumerate(STAGES)}
    ms = max_over_ranks(dist, ms, dev)
    st, tile_pairs, pairs = pair_counts(R, fr)

    # end to end through the public API: pinned host inputs -> device, render,
    # backward, image back to host
    host = {k: torch.from_numpy(np.ascontiguousarray(getattr(sc, k))).pin_memory()
            for k in ["means", "scales", "quats", "weights", "sh"]}
    dev_in = {k: torch.empty_like(v, device=dev) for k, v in host.items()}
    rgb_host = torch.empty(npix, 3, dtype=torch.float32).pin_memory()
    h2d = sum(v.numel() * 4 for v in host.values())
    d2h = rgb_host.numel() * 4
    g2 = GaussianTensors(dev_in["means"], dev_in["scales"], dev_in["quats"], dev_in["weights"], dev_in["sh"],
                         sc.sh_degree)
    outbuf = dict(rgb=torch.empty(npix, 3, device=dev), T=torch.empty(npix, device=dev),
                  penalty=torch.empty(npix, device=dev))
    grads2 = {k: torch.empty_like(v) for k, v in dev_in.items()}

    def e2e_step():
        for k in host:
            dev_in[k].copy_(host[k], non_blocking=True)
        o = R.render(g2, cam, capacity=fr.cap, out=outbuf, penalty=True, query_capacity=fr.qcap)
        if with_bwd:
            dl = (o["rgb"] - target).mul_(2.0 / o["rgb"].numel())
            R.backward(g2, cam, fr.cap, dl, None, grads=grads2, query_capacity=fr.qcap)
        rgb_host.copy_(o["rgb"], non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / args.steps
    if rank != 0:
        return None

    sm_mhz = clk.get("sm_mhz") or measured_peaks().get("sm_max_mhz", 2070.0)
    n_int = R.config.n_intervals
    fwd_ms = sum(stage_ms[k] for k in STAGES[:4])
    dominant = "k_bwd_quadrature" if with_bwd and stage_ms["bwd_quadrature"] > stage_ms["shade"] else "k_shade"
    dom_ms = stage_ms["bwd_quadrature" if dominant == "k_bwd_quadrature" else "shade"]
    line = dict(
        metric=METRIC,
        value=job_mpix_s(world, npix, ms),
        unit="Mpixel/s",
        n_gpus=world, steps=args.steps, warmup=args.warmup, ms_per_step=ms,
        higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32", data="synthetic",
        fwd_mpix_s=world * npix / (fwd_ms * 1e-3) / 1e6,
        config={"workload": args.workload, "gaussians": g.P, "width": cam.width, "height": cam.height,
                "sh_degree": sc.sh_degree,
                "n_moments": 9, "n_intervals": n_int, "basis": args.basis, "moment_storage": args.moment_dtype,
                "tau_table_knots": args.tau_table,
                "pass": "forward+backward (L2 loss vs random target)" if with_bwd else "forward",
                "saved_queries": fr.qcap > 0,
                "tiling": dict(tile=[R.config.tile_w, R.config.tile_h], batch=R.config.batch,
                               schedule=R.config.schedule),
                "l2": "inputs larger than L2 (236 MB Gaussian parameters + 128 MB records per step)"
                      if args.workload == WORKLOAD else "see workload",
                "parallelism": "replicas" if world > 1 else "1 GPU"},
        stage_ms=stage_ms,
        pairs=pairs, tile_pairs=tile_pairs, status=st,
        roofline=roofline(dominant, dom_ms, pairs, n_int, peaks, sm_mhz, captured=fr.qcap > 0)
        if args.basis == "power" and not args.tau_table else None,
        roofline_shade=roofline("k_shade", stage_ms["shade"], pairs, n_int, peaks, sm_mhz, captured=fr.qcap > 0)
        if args.basis == "power" and not args.tau_table else None,
        alu_peaks=peaks,
        e2e=dict(value=world * npix / (e2e_ms * 1e-3) / 1e6, unit="Mpixel/s", h2d_bytes_per_step=h2d,
                 d2h_bytes_per_step=d2h),
        gpu_launches=int(launches),
        clocks=clk,
    )
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_oracle_sample(sc, cam, with_bwd, name=args.workload, basis=args.basis,
                                                 n_intervals=n_int)
    if (world == 1 and args.workload == WORKLOAD and with_bwd and args.basis == "power" and not args.tau_table
            and args.moment_dtype == "f32" and not args.no_batch16):
        # the many-view configuration (16 views of uneven resolution), short form
        del fr, g2, dev_in, outbuf, grads2
        R._ws = None
        torch.cuda.empty_cache()
        line["batch16"] = run_batch16(args, None, rank, world, dev, summary=True)
        # the same 16 views as two frames of 8 in the graph: each frame keeps
        # all of its bound queries
        a2 = argparse.Namespace(**vars(args))
        a2.batch16_frames = 2
        line["batch16_two_frames"] = run_batch16(a2, None, rank, world, dev, summary=True)
        line["adc"] = run_adc(args, None, rank, world, dev, summary=True)
    return line


def run_batch16(args, dist, rank, world, dev, summary=False):
    """16 views of uneven resolution: fwd+bwd in one CUDA graph vs 16 sequential
    single-view calls (eager).  summary=True: the short form nested in the
    default bench line (default execution shape instead of the autotuner, 2
    sequential steps, no end-to-end leg); returns a dict."""
    from paper_2512_11800_gb300 import GaussianTensors, RasterConfig, Rasterizer
    sc, _ = scenes.workload(WORKLOAD)
    cams = scenes.multiview_cameras(16, seed=4, radius=3.0, fov_deg=60.0)
    npix = [c.width * c.height for c in cams]
    g = GaussianTensors.from_scene(sc, dev)
    R = Rasterizer(RasterConfig(), device=dev)
    # execution shape tuned on the largest view (fwd+bwd), shared by all views
    big = max(range(len(cams)), key=lambda i: npix[i])
    c0 = R.config
    tuned = (c0.tile_w, c0.tile_h, c0.batch, c0.schedule, None) if summary else R.autotune(g, cams[big], backward=True)
    rng = np.random.default_rng(12)
    target = torch.as_tensor(rng.random((sum(npix), 3), dtype=np.float32), device=dev)
    stream = torch.cuda.current_stream()
    with_bwd = not args.forward_only

    # sequential: one Frame per view sharing one workspace, eager calls
    offs = np.concatenate([[0], np.cumsum(npix)])
    need = 0
    for c in cams:
        tp, pp = R.pair_counts(g, c)
        R.set_query_capacity(pp)
        need = max(need, R.workspace_bytes(c, g.P, tp))
    R._ws = None
    shared = R.workspace(need)
    frames = [Frame(R, g, c, target[offs[i]:offs[i + 1]], ws=shared) for i, c in enumerate(cams)]

    def seq_step():
        for f in frames:
            f.step(stream, with_bwd)

    seq_warm, seq_steps = (1, 2) if summary else (args.warmup, args.steps)
    for _ in range(seq_warm):
        seq_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(seq_steps):
        seq_step()
    e1.record(stream)
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1) / seq_steps
    del frames, shared
    R._ws = None
    torch.cuda.empty_cache()

    # batched: all 16 views in one frame (one set of persistent launches over
    # all views' tiles; --batch16-frames F: F frames of 16/F views one after
    # the other), the whole step captured in one CUDA graph.  The bound
    # queries are kept for as many pixels as the free device memory allows
    # (60 % of it after the workspace); the backward solves the rest again.
    counts = [R.pair_counts(g, c) for c in cams]
    nf = max(1, min(len(cams), getattr(args, "batch16_frames", 1)))
    groups = [list(range(k * len(cams) // nf, (k + 1) * len(cams) // nf)) for k in range(nf)]
    gcams = [[cams[i] for i in grp] for grp in groups]
    gcounts = [R.pair_counts(g, gc) for gc in gcams]
    tp, pp = R.pair_counts(g, cams)
    R.set_query_capacity(0)
    base = max(R.workspace_bytes(gc, g.P, gtp) for gc, (gtp, _) in zip(gcams, gcounts))
    torch.cuda.empty_cache()
    free = torch.cuda.mem_get_info(dev)[0]
    R.config.query_budget_gb = max(0.0, 0.6 * (free - base)) / 2 ** 30
    need = 0
    for gc, (gtp, gpp) in zip(gcams, gcounts):
        R.set_query_capacity(gpp)
        need = max(need, R.workspace_bytes(gc, g.P, gtp))
    R._ws = None
    shared = R.workspace(need)
    fbs = [Frame(R, g, [cams[i] for i in grp], target[offs[grp[0]]:offs[grp[-1] + 1]], ws=shared)
           for grp in groups]

    def batch_step(st):
        for f in fbs:
            f.step(st, with_bwd)

    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        for _ in range(args.warmup):
            batch_step(side)
    stream.wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    l0 = R.lib.mb3dgs_launch_count()
    with torch.cuda.graph(graph):
        batch_step(torch.cuda.current_stream())
    launches = R.lib.mb3dgs_launch_count() - l0
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler()
    clocks.start()
    e0.record(stream)
    for _ in range(args.steps):
        graph.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = max_over_ranks(dist, e0.elapsed_time(e1) / args.steps, dev)
    st = max((pair_counts(R, f)[0] for f in fbs), key=abs)
    tile_pairs = sum(c[0] for c in counts)
    pairs = sum(c[1] for c in counts)
    if summary:
        tot = sum(npix)
        return dict(workload="batch16_shells1M: 16 views (640x360 / 1280x720 / 1920x1080), %s in one CUDA "
                             "graph, forward + backward" % ("one frame" if len(fbs) == 1 else
                                                           "%d frames of %d views" % (len(fbs), len(cams) // len(fbs))),
                    value=world * tot / (ms * 1e-3) / 1e6, unit="Mpixel/s", ms_per_step=ms, steps=args.steps,
                    sequential_ms_per_step=seq_ms, sequential_mpix_s=world * tot / (seq_ms * 1e-3) / 1e6,
                    speedup_vs_sequential=seq_ms / ms, pixels=tot, pixel_pairs=pairs,
                    query_bytes=8 if R.cfg_c.compact_queries else 16,
                    kept_queries_frac=sum(f.qcap for f in fbs) / max(pp, 1), frames=len(fbs),
                    gpu_launches=int(launches), status=st, clocks=clk)

    # end to end: inputs from pinned host memory into the graph's input
    # buffers, replay, rgb back to host
    host = {k: torch.from_numpy(np.ascontiguousarray(getattr(sc, k))).pin_memory()
            for k in ["means", "scales", "quats", "weights", "sh"]}
    rgb_host = torch.empty(sum(npix), 3, dtype=torch.float32).pin_memory()

    def e2e_step():
        for k in host:
            getattr(g, k).copy_(host[k], non_blocking=True)
        graph.replay()
        o = 0
        for f in fbs:
            rgb_host[o:o + f.rgb.shape[0]].copy_(f.rgb, non_blocking=True)
            o += f.rgb.shape[0]

    e2e_step()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / args.steps
    if rank != 0:
        return None
    tot = sum(npix)
    return dict(
        metric=METRIC,
        value=job_mpix_s(world, tot, ms),
        unit="Mpixel/s",
        n_gpus=world, steps=args.steps, warmup=args.warmup, ms_per_step=ms,
        higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32", data="synthetic",
        config={"workload": "batch16_shells1M", "gaussians": g.P, "views": [[c.width, c.height] for c in cams],
                "pixels": tot, "pass": "forward+backward" if with_bwd else "forward",
                "query_slots": fbs[0].qcap, "pixel_pairs": pp,
                "kept_queries": "%.0f %% of the pixel pairs (60 %% of free device memory), %d B a query"
                                % (100.0 * sum(f.qcap for f in fbs) / max(pp, 1), 8 if R.cfg_c.compact_queries else 16),
                "groups": groups,
                "tiling": dict(tile=list(tuned[:2]), batch=tuned[2], schedule=tuned[3], tuned_ms=tuned[4]),
                "graph": "whole step in one CUDA graph (%s)" % (
                    "one set of persistent launches over all 16 views" if len(fbs) == 1 else
                    "%d frames of %d views, one set of persistent launches each" % (len(fbs), len(cams) // len(fbs))),
                "l2": "inputs larger than L2",
                "parallelism": "replicas" if world > 1 else "1 GPU"},
        sequential=dict(ms_per_step=seq_ms, mpix_s=world * tot / (seq_ms * 1e-3) / 1e6,
                        how="16 x (render + backward) single-view eager calls"),
        speedup_vs_sequential=seq_ms / ms,
        pairs=pairs, tile_pairs=tile_pairs, status=st,
        e2e=dict(value=world * tot / (e2e_ms * 1e-3) / 1e6, unit="Mpixel/s",
                 h2d_bytes_per_step=sum(v.numel() * 4 for v in host.values()),
                 d2h_bytes_per_step=rgb_host.numel() * 4),
        gpu_launches=int(launches),
        clocks=clk,
    )


def run_adc(args, dist, rank, world, dev, summary=False):
    """One step of the adaptive density control (Sec. 3.4, App. D) on the 1M
    scene: accumulate one step of |dL/dmean| statistics, then clone / split /
    prune into a preallocated set (C ABI, no host synchronisation inside the
    timed steps).  HBM-bound: algorithmic bytes = P (44 statistics + 252 read)
    + P_out 236 written per step.  summary=True: the short form nested in the
    default line."""
    from paper_2512_11800_gb300 import GaussianTensors
    from paper_2512_11800_gb300 import _binding as B
    lib = B.load()
    sc, _ = scenes.workload(WORKLOAD)
    g = GaussianTensors.from_scene(sc, dev)
    P = g.P
    rng = np.random.default_rng(13)
    dmeans = torch.as_tensor((rng.normal(size=(P, 3)) * 6e-5).astype(np.float32), device=dev)
    abs_sum = torch.zeros(P, 3, device=dev)
    count = torch.zeros(P, dtype=torch.int32, device=dev)
    K3 = 3 * (sc.sh_degree + 1) ** 2
    cap = 2 * P
    outs = [torch.empty(cap, 3, device=dev), torch.empty(cap, 3, device=dev), torch.empty(cap, 4, device=dev),
            torch.empty(cap, device=dev), torch.empty(cap, K3, device=dev)]
    o = B.GaussiansOut()
    o.means, o.scales, o.quats, o.weights, o.sh = (t.data_ptr() for t in outs)
    o.capacity = cap
    nb = C.c_size_t(0)
    B.check(lib.mb3dgs_densify_workspace_size(P, C.byref(nb)), "densify_workspace_size")
    ws = torch.empty(int(nb.value), dtype=torch.uint8, device=dev)
    p_out = torch.zeros(1, dtype=torch.int64, device=dev)
    action = torch.empty(P, dtype=torch.int8, device=dev)
    cfg = B.AdcConfig()
    lib.mb3dgs_adc_config_default(C.byref(cfg))
    cfg.scene_extent = 3.0          # camera distance of the scene
    gc = g.to_c()
    stream = torch.cuda.current_stream()
    sp = C.c_void_p(stream.cuda_stream)
    vp = lambda t: C.c_void_p(t.data_ptr())

    def step():
        B.check(lib.mb3dgs_accumulate_grad_stats(vp(dmeans), None, P, vp(abs_sum), vp(count), sp), "grad_stats")
        B.check(lib.mb3dgs_densify(C.byref(cfg), C.byref(gc), vp(abs_sum), vp(count), vp(ws), ws.numel(),
                                   C.byref(o), vp(p_out), vp(action), None, sp), "densify")

    for _ in range(args.warmup):
        abs_sum.zero_()
        count.zero_()
        step()
    torch.cuda.synchronize()
    steps = args.steps
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    l0 = lib.mb3dgs_launch_count()
    for k in range(steps):
        abs_sum.zero_()          # one statistics step before each densification (outside the events)
        count.zero_()
        evs[k][0].record(stream)
        step()
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    launches = lib.mb3dgs_launch_count() - l0
    ms = statistics.median(a.elapsed_time(b) for a, b in evs)
    n_out = int(p_out.item())
    acts = np.bincount(action.cpu().numpy().astype(np.int64), minlength=3)
    bytes_step = P * (44 + 252) + n_out * 236
    peak = measured_peaks().get("hbm_gbs")
    achieved = bytes_step / (ms * 1e-3) / 1e9
    roof = dict(kernel="statistics + densify (count, scan, write)", bound="hbm", achieved=achieved, peak=peak,
                unit="GB/s", frac=achieved / peak if peak else None, traffic=None,
                peak_note="peak = MEASURED_PEAKS.json hbm_gbs (copy); achieved = algorithmic bytes "
                          "P (44 + 252) + P_out 236 per step / median step time")
    res = dict(workload="adc_shells1M: %d Gaussians (SH 3), statistics + clone/split/prune" % P,
               value=P / (ms * 1e-3) / 1e6, unit="Mgaussian/s", ms_per_step=ms, steps=steps,
               P_out=n_out, actions=dict(kept=int(acts[0]), cloned=int(acts[1]), split=int(acts[2])),
               gpu_launches=int(launches), roofline=roof)
    if summary:
        return res
    line = dict(metric="Mgaussian/s of one adaptive density control step, 1M Gaussians", value=res["value"],
                unit="Mgaussian/s", n_gpus=world, steps=steps, warmup=args.warmup, ms_per_step=ms,
                higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32", data="synthetic",
                config={"workload": "adc_shells1M", "gaussians": P, "sh_degree": sc.sh_degree,
                        "l2": "inputs larger than L2 (236 MB parameters)"},
                P_out=n_out, actions=res["actions"], roofline=roof, gpu_launches=int(launches))
    return line if rank == 0 else None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(scenes.WORKLOADS) + ["batch16", "adc"],
                    help="the default is the headline workload; the others are for profiling")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch16-frames", type=int, default=1,
                    help="batch16: split the 16 views into this many frames run one after the other in the graph")
    ap.add_argument("--no-batch16", action="store_true",
                    help="leave out the short 16-view record the default workload adds to its line")
    ap.add_argument("--forward-only", action="store_true")
    ap.add_argument("--basis", default="power", choices=["power", "trig"],
                    help="moment basis; trig (Eq. 13-14) reports no roofline (its node solve has no fixed op count)")
    ap.add_argument("--n-intervals", type=int, default=3)
    ap.add_argument("--tau-table", type=int, default=0,
                    help="tabulated transmittance with this many knots a segment (0: off)")
    ap.add_argument("--moment-dtype", default="f32", choices=["f32", "bf16", "f16"],
                    help="storage of the per-pixel moments (accumulation is FP32 in every case)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        run_reference(args)
        return
    dist, rank, world = dist_setup(args.gpus)
    dev = torch.device("cuda", torch.cuda.current_device())
    run = {"batch16": run_batch16, "adc": run_adc}.get(args.workload, run_single)
    line = run(args, dist, rank, world, dev)
    if line is not None:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
