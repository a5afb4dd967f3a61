"""CPU regression guard for the CUDA path's forward arithmetic.

tests/host/emulate_forward.cu compiles the device functions of the forward
(preprocess_one, pair_gaussian, legendre_moments, reconstruct_pixel,
pair_quadrature, the Eq. 15 epilogue) for the host.  The emulation runs them
per pixel over the Gaussians whose rectangle holds the pixel centre, in
ascending id order as the kernels do, and is compared with the FP64 oracle at
the parity bar (1e-4 on RGB and final transmittance).

This is a guard, not the parity evidence.  Host libm replaces the device's
exp and erf, division is exact, and binning, tiling and launches are not
exercised.  Parity of the CUDA path itself is established by the -m gpu tests.
Needs nvcc (host compilation only; no GPU)."""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

import oracle as O
import scenes
from helpers import oracle_config

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
TOL = 1e-4


def _nvcc():
    for c in [os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"]:
        if c and os.path.exists(c):
            return c
    return None


@pytest.fixture(scope="module")
def emulator(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("emu") / "emulate_forward")
    cmd = [nvcc, "-O2", "-std=c++17", "--expt-relaxed-constexpr", "-I" + os.path.join(ROOT, "include"),
           "-gencode", "arch=compute_103a,code=sm_103a", os.path.join(HERE, "host", "emulate_forward.cu"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    return exe


def emulate(exe, tmp, sc, cam, region):
    fin, fout = str(tmp / "in.bin"), str(tmp / "out.bin")
    with open(fin, "wb") as f:
        f.write(struct.pack("<qi", sc.P, sc.sh_degree))
        for a in [sc.means, sc.scales, sc.quats, sc.weights, sc.sh]:
            f.write(np.ascontiguousarray(a, np.float32).tobytes())
        f.write(np.asarray(cam.viewmat, np.float32).tobytes())
        f.write(struct.pack("<ffffii", cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height))
        f.write(struct.pack("<4i", *region))
    subprocess.run([exe, fin, fout], check=True, timeout=600)
    w, h = region[2], region[3]
    d = np.fromfile(fout, np.float32).astype(np.float64)
    return d[:3 * w * h].reshape(h, w, 3), d[3 * w * h:].reshape(h, w)


def _case(name):
    if name == "uniform2k_full":
        sc, cam = scenes.workload("uniform2k_128")
        return sc, cam, (0, 0, cam.width, cam.height)
    if name == "ragged_near_camera":
        sc = scenes.scene_uniform(600, 5)
        cam = scenes.look_at((0.1, -0.2, -1.6), width=77, height=45, fov_deg=70)
        return sc, cam, (0, 0, cam.width, cam.height)
    if name == "camera_inside_cloud":
        sc = scenes.scene_uniform(400, 31)
        sc.means[:, 2] -= 1.5
        sc.scales *= 3.0
        cam = scenes.look_at((0, 0, -1.6), width=40, height=32, fov_deg=70)
        return sc, cam, (0, 0, cam.width, cam.height)
    if name == "clusters200k_crop":
        sc, cam = scenes.workload("clusters200k_720p")
        return sc, cam, (608, 328, 24, 24)
    raise KeyError(name)


@pytest.mark.parametrize("name", ["uniform2k_full", "ragged_near_camera", "camera_inside_cloud", "clusters200k_crop"])
def test_host_emulated_forward_matches_oracle(emulator, tmp_path, name):
    sc, cam, region = _case(name)
    rgb, T = emulate(emulator, tmp_path, sc, cam, region)
    ref = O.render(sc, cam, oracle_config(), region=region)
    e_rgb = float(np.abs(rgb - ref["rgb"].numpy()).max())
    e_T = float(np.abs(T - ref["T"].numpy()).max())
    assert np.isfinite(rgb).all() and np.isfinite(T).all()
    assert e_rgb <= TOL and e_T <= TOL, (name, e_rgb, e_T)
