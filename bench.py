"""Benchmark of the moment-based Gaussian rasterizer on one GB300.

One step = one pass of the hot path over the 1,000,000-Gaussian scene
(64 anisotropic clusters + interpenetrating low-density shells, SH degree 3)
rendered at 1920x1080: preprocess -> tile binning -> moment pass ->
per-pixel reconstruction -> quadrature pass (+ backward when enabled).
Prints one JSON line (see the module's contract in the design doc).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (launched by torchrun) every rank renders its own replica of the
workload (the path has no data exchange); rank 0 prints the aggregate.
"""
from __future__ import annotations

import argparse
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
SM_COUNT = 152
FP32_LANES_PER_SM = 128


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# Algorithmic FP32 work per (pixel, Gaussian) pair of the quadrature pass,
# counted from the per-pair arithmetic ("op model").
def shade_flops_per_pair(n_intervals=3):
    return SHADE_FLOPS_BASE + (n_intervals + 1) * SHADE_FLOPS_PER_QUERY


SHADE_FLOPS_BASE = 60.0        # pair geometry, sample points, quadrature/penalty bookkeeping
SHADE_FLOPS_PER_QUERY = 330.0  # warp, standardise, pi_k, K(eta,eta), one Laguerre root solve + weight


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


def cpu_oracle_sample(sc, cam, seconds_target=20.0):
    """Time the FP64 oracle on a centred crop of the same workload (bounded sample)."""
    import oracle as O
    torch.set_num_threads(os.cpu_count() or 1)
    cfg = O.OracleConfig()
    size = 48
    region = ((cam.width - size) // 2, (cam.height - size) // 2, size, size)
    t0 = time.perf_counter()
    out = O.render(sc, cam, cfg, region=region)
    dt = time.perf_counter() - t0
    return dict(value=size * size / dt / 1e6, unit="Mpixel/s", cores=torch.get_num_threads(), kind="oracle",
                sample="centre %dx%d crop of the 1920x1080 frame of %s (%d pairs), %.1f s" %
                       (size, size, WORKLOAD, out["n_pairs"], dt))


def run_reference(args):
    """--impl reference: the FP64 CPU oracle timed on a bounded sample per step."""
    if int(os.environ.get("RANK", "0")) != 0:
        return
    import oracle as O
    torch.set_num_threads(os.cpu_count() or 1)
    sc, cam = scenes.workload(WORKLOAD)
    cfg = O.OracleConfig()
    size = 16
    region = ((cam.width - size) // 2, (cam.height - size) // 2, size, size)
    for _ in range(args.warmup):
        O.render(sc, cam, cfg, region=region)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.render(sc, cam, cfg, region=region)
    dt = (time.perf_counter() - t0) / args.steps
    val = size * size / dt / 1e6
    line = dict(metric=METRIC, value=val, unit="Mpixel/s", impl="reference", n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=dt * 1e3, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic",
                config=dict(workload=WORKLOAD + " (centre %dx%d crop per step)" % (size, size), gaussians=1_000_000,
                            width=1920, height=1080),
                cpu_baseline=dict(kind="oracle", cores=torch.get_num_threads(), value=val, unit="Mpixel/s",
                                  sample="centre %dx%d crop per step" % (size, size)),
                e2e=dict(value=val, unit="Mpixel/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--forward-only", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        run_reference(args)
        return

    from paper_2512_11800_gb300 import GaussianTensors, RasterConfig, Rasterizer
    from paper_2512_11800_gb300 import _binding as B
    import ctypes as C

    dist, rank, world = dist_setup(args.gpus)
    dev = torch.device("cuda", torch.cuda.current_device())
    sc, cam = scenes.workload(WORKLOAD)
    npix = cam.width * cam.height
    R = Rasterizer(RasterConfig(), device=dev)
    g = GaussianTensors.from_scene(sc, dev)
    cap = R.count_pairs(g, cam)
    out = R.render(g, cam, capacity=cap)
    stream = torch.cuda.current_stream()
    s = C.c_void_p(stream.cuda_stream)
    lib = R.lib
    arr, nv = R.cameras(cam)
    ws = R.workspace(R.workspace_bytes(cam, g.P, cap))
    gc = g.to_c()
    cfg = C.byref(R.cfg_c)
    wsp, wsn = C.c_void_p(ws.data_ptr()), ws.numel()
    rgb, T, pen = out["rgb"], out["T"], out["penalty"]

    target = torch.as_tensor(scenes.target_image(cam.height, cam.width).reshape(-1, 3), device=dev)
    dL_drgb = torch.empty_like(rgb)
    grads = {k: torch.empty_like(getattr(g, k)) for k in ["means", "scales", "quats", "weights", "sh"]}
    gg = B.GaussianGrads()
    gg.means, gg.scales, gg.quats = grads["means"].data_ptr(), grads["scales"].data_ptr(), grads["quats"].data_ptr()
    gg.weights, gg.sh = grads["weights"].data_ptr(), grads["sh"].data_ptr()
    with_bwd = not args.forward_only

    def step(record=None):
        if record is not None:
            record[0].record(stream)
        B.check(lib.mb3dgs_preprocess(cfg, C.byref(gc), arr, nv, wsp, wsn, cap, s), "preprocess")
        B.check(lib.mb3dgs_bin_tiles(cfg, arr, nv, g.P, cap, wsp, wsn, s), "bin")
        if record is not None:
            record[1].record(stream)
        B.check(lib.mb3dgs_accumulate_moments(cfg, arr, nv, g.P, cap, wsp, wsn, None, s), "moments")
        if record is not None:
            record[2].record(stream)
        B.check(lib.mb3dgs_reconstruct_transmittance(cfg, arr, nv, g.P, cap, wsp, wsn, None, 0, None, s), "recon")
        if record is not None:
            record[3].record(stream)
        B.check(lib.mb3dgs_shade(cfg, arr, nv, g.P, cap, wsp, wsn, C.c_void_p(rgb.data_ptr()),
                                 C.c_void_p(T.data_ptr()), C.c_void_p(pen.data_ptr()), s), "shade")
        if record is not None:
            record[4].record(stream)
        if with_bwd:
            # L2 loss against the random target image (the loss itself is the caller's)
            torch.sub(rgb, target, out=dL_drgb).mul_(2.0 / rgb.numel())
            B.check(lib.mb3dgs_backward(cfg, C.byref(gc), arr, nv, wsp, wsn, cap, C.c_void_p(dL_drgb.data_ptr()),
                                        None, C.byref(gg), s), "backward")
        if record is not None:
            record[5].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # per-stage times (device, CUDA events on the launching stream)
    stage = {"preprocess+bin": [], "moments": [], "reconstruct": [], "shade": [], "backward": []}
    clocks = ClockSampler()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    l0 = lib.mb3dgs_launch_count()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(args.steps)]
    t_start.record(stream)
    for k in range(args.steps):
        step(evs[k])
    t_end.record(stream)
    torch.cuda.synchronize()
    launches = lib.mb3dgs_launch_count() - l0
    clk = clocks.stop()
    ms = t_start.elapsed_time(t_end) / args.steps
    for e in evs:
        stage["preprocess+bin"].append(e[0].elapsed_time(e[1]))
        stage["moments"].append(e[1].elapsed_time(e[2]))
        stage["reconstruct"].append(e[2].elapsed_time(e[3]))
        stage["shade"].append(e[3].elapsed_time(e[4]))
        stage["backward"].append(e[4].elapsed_time(e[5]))
    stage_ms = {k: statistics.median(v) for k, v in stage.items()}
    if dist:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    st, npairs_tiles = R.status()
    # algorithmic pairs (pixel centre inside the Gaussian's rectangle), counted exactly
    rects = torch.empty(g.P, 4, dtype=torch.int32, device=dev)
    B.check(lib.mb3dgs_debug_tile_lists(cfg, arr, nv, g.P, cap, wsp, wsn, None, None, C.c_void_p(rects.data_ptr()), s),
            "debug")
    r = rects.long()
    pairs = int(((r[:, 2] - r[:, 0] + 1).clamp(min=0) * (r[:, 3] - r[:, 1] + 1).clamp(min=0)).sum().item())

    # end to end through the public API: pinned host inputs -> device, render, image back to host
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
        o = R.render(g2, cam, capacity=cap, out=outbuf, penalty=True)
        if with_bwd:
            dl = (o["rgb"] - target).mul_(2.0 / o["rgb"].numel())
            R.backward(g2, cam, cap, dl, None, grads=grads2)
        rgb_host.copy_(o["rgb"], non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / args.steps

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    peaks = measured_peaks()
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = SM_COUNT * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12        # TFLOP/s at max SM clock
    fwd_ms = sum(stage_ms[k] for k in ["preprocess+bin", "moments", "reconstruct", "shade"])
    flops = pairs * shade_flops_per_pair(3)
    achieved = flops / (stage_ms["shade"] * 1e-3) / 1e12
    line = dict(
        metric=METRIC,
        value=world * npix / (ms * 1e-3) / 1e6,
        unit="Mpixel/s",
        n_gpus=world, steps=args.steps, warmup=args.warmup, ms_per_step=ms,
        higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32", data="synthetic",
        fwd_mpix_s=world * npix / (fwd_ms * 1e-3) / 1e6,
        config=dict(workload=WORKLOAD, gaussians=g.P, width=cam.width, height=cam.height, sh_degree=3,
                    n_moments=9, n_intervals=3, pass_="forward+backward (L2 loss vs random target)" if with_bwd
                    else "forward", l2="inputs larger than L2 (236 MB Gaussian "
                    "parameters + 128 MB records per step)", parallelism="replicas" if world > 1 else "1 GPU"),
        stage_ms=stage_ms,
        pairs=pairs, tile_pairs=npairs_tiles, status=st,
        roofline=dict(kernel="k_shade", bound="alu", achieved=achieved, peak=fp32_peak, unit="TFLOP/s",
                      frac=achieved / fp32_peak, traffic=None,
                      peak_note="FP32: %d SMs x %d lanes x 2 flop x %.0f MHz (max SM clock, MEASURED_PEAKS.json)"
                                % (SM_COUNT, FP32_LANES_PER_SM, sm_max),
                      flops_per_pair=shade_flops_per_pair(3)),
        e2e=dict(value=world * npix / (e2e_ms * 1e-3) / 1e6, unit="Mpixel/s", h2d_bytes_per_step=h2d,
                 d2h_bytes_per_step=d2h),
        gpu_launches=int(launches),
        clocks=clk,
    )
    line["config"]["pass"] = line["config"].pop("pass_")
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_oracle_sample(sc, cam)
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
