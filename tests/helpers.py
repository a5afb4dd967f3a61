"""Shared test helpers: map the CUDA path's float32 configuration onto the
oracle's (the oracle consumes exactly the same float32 input values), keep
the oracle's expensive results for the large workloads once per test session
(scene draws, FP64 preprocessing of 1M-3M Gaussians, crop renders), and run
many small independent oracle renders on a pool of worker processes."""
import multiprocessing
import os
from concurrent.futures import ProcessPoolExecutor

import numpy as np

import oracle as O
import scenes

FLOAT_FIELDS = ["kappa", "beta", "conf_c", "warp_lambda", "t_near", "t_far", "eps", "bias_alpha", "m_min", "r_mult"]


def f32(x):
    return float(np.float32(x))


def oracle_config(rc=None, **over):
    """OracleConfig with the float32-rounded values of a RasterConfig."""
    from paper_2512_11800_gb300 import RasterConfig
    rc = rc or RasterConfig()
    kw = {k: f32(getattr(rc, k)) for k in FLOAT_FIELDS}
    kw.update(n=rc.n, n_intervals=rc.n_intervals, bg=tuple(f32(b) for b in rc.bg), basis=rc.basis,
              trig_theta=f32(rc.trig_theta))
    kw.update(over)
    return O.OracleConfig(**kw)


_WORKLOADS = {}
_PRE = {}
_REFS = {}


def workload(name):
    """scenes.workload(name), drawn once per session (tests that change a
    scene work on a copy: Scene.subset)."""
    if name not in _WORKLOADS:
        _WORKLOADS[name] = scenes.workload(name)
    return _WORKLOADS[name]


def _cfg_key(cfg):
    return tuple(sorted((k, v) for k, v in vars(cfg).items()))


def oracle_pre(name, cfg):
    key = (name, _cfg_key(cfg))
    if key not in _PRE:
        sc, cam = workload(name)
        _PRE[key] = O.preprocess(sc, cam, cfg)
    return _PRE[key]


def oracle_crop(name, region, cfg=None):
    """O.render of one pixel region of a named workload, computed once per
    session and shared by every test that checks that region."""
    cfg = cfg or oracle_config()
    key = (name, tuple(region), _cfg_key(cfg))
    if key not in _REFS:
        sc, cam = workload(name)
        _REFS[key] = O.render(sc, cam, cfg, region=region, pre=oracle_pre(name, cfg))
    return _REFS[key]


def crops(cam, seed, n, size):
    """The centre crop and n seeded crops of size x size pixels."""
    rng = np.random.default_rng(seed)
    out = [((cam.width - size) // 2, (cam.height - size) // 2, size, size)]
    for _ in range(n):
        out.append((int(rng.integers(0, cam.width - size)), int(rng.integers(0, cam.height - size)), size, size))
    return out


def _worker_init():
    import torch
    torch.set_num_threads(2)


def _loss_task(args):
    scene, cam, cfg, dL_drgb, region = args
    loss, rect = O.render_loss(scene, cam, cfg, dL_drgb, region=region)
    return loss, rect.numpy()


def oracle_losses(tasks):
    """O.render_loss for each (scene, cam, cfg, dL_drgb, region) task, on
    worker processes started with spawn (never forked from a process that
    has used the GPU).  Returns [(loss, rect), ...] in task order."""
    workers = max(1, min(8, (os.cpu_count() or 2) // 2))
    ctx = multiprocessing.get_context("spawn")
    with ProcessPoolExecutor(max_workers=workers, mp_context=ctx, initializer=_worker_init) as ex:
        return list(ex.map(_loss_task, tasks, chunksize=4))


def probe_excess(T_got, ref, probes, cfg, rel=2e-6, trials=16, seed=0):
    """Transmittance probes T(eta) against the oracle, judged against the
    oracle's own conditioning: for every pixel whose error exceeds 1e-4 the
    oracle's optical depths are recomputed with every one of its FP64 moments
    perturbed by rel * m0 (rel = 2e-6: the rounding of a FP32 sum of a few
    hundred terms whose magnitudes add up to about m0, sqrt(n) eps m0 plus
    each term's own rounding) and the largest change of T is that pixel's
    allowance.  Returns the largest
    error in excess of 1e-4 + allowance (<= 0 when every probe passes) and
    the number of pixels that needed an allowance."""
    import torch
    T_ref = np.exp(-ref["tau_probe"].numpy())
    err = np.abs(T_got - T_ref).max(-1)
    bad = np.argwhere(err > 1e-4)
    worst = float(err.max()) - 1e-4 if bad.size == 0 else -1.0
    depth = O.trig_optical_depth if cfg.basis == "trig" else O.optical_depth
    rng = np.random.default_rng(seed)
    eta = torch.as_tensor(np.asarray(probes, dtype=np.float64))[None]
    for iy, ix in bad:
        m = ref["m"][iy, ix][None]
        base = np.exp(-depth(m, eta, cfg).numpy()[0])
        spread = 0.0
        for _ in range(trials):
            noise = torch.as_tensor(rng.normal(size=m.shape))
            if m.is_complex():
                im = torch.as_tensor(rng.normal(size=m.shape))
                im[..., 0] = 0.0                      # m0 is real
                noise = torch.complex(noise, im)
            pm = m + rel * m[..., :1].real * noise
            spread = max(spread, float(np.abs(np.exp(-depth(pm, eta, cfg).numpy()[0]) - base).max()))
        worst = max(worst, float(err[iy, ix]) - 1e-4 - spread)
    return worst, len(bad)
