"""bench.py pieces that need no GPU: the reference arm (the FP64 oracle on a
bounded sample) prints one well-formed JSON line, and the roofline and
throughput arithmetic."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "Mpixel/s" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and "crop" in d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "Mpixel/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_roofline_and_throughput_arithmetic():
    sys.path.insert(0, ROOT)
    import bench
    pairs, ms, clk = 368_206_242, 31.5, 2070.0
    peaks = dict(fp32_tflops=80.0, ex2_tops=10.0, rsqrt_tops=5.0, rcp_tops=5.2, sin_tops=5.0, sm_count=152)
    r = bench.roofline("k_shade", ms, pairs, 3, peaks, clk)
    # the method's op model at N = 3: 40 + 250 x 4 flop and 4 + 12 x 4 MUFU ops a pair
    assert bench.alg_ops("k_shade", 3) == (1040, 52)
    assert bench.alg_ops("k_bwd_quadrature", 3) == (2080, 104)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s" and r["sm_count"] == 152
    assert r["peak"] == pytest.approx(80.0)
    assert r["achieved"] == pytest.approx(1040 * pairs / (ms * 1e-3) / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 80.0) == pytest.approx(r["frac_fp32_algorithmic"])
    assert r["frac_xu"] == pytest.approx(52 * pairs / (ms * 1e-3) / 1e12 / 5.0)
    ex = bench.EXECUTED_PER_PAIR["k_shade"]
    assert r["issue_frac"] == pytest.approx(ex["thread_inst"] * pairs / (ms * 1e-3) / (152 * 4 * 32 * clk * 1e6))
    assert r["frac_fp32_executed"] == pytest.approx(ex["flops"] * pairs / (ms * 1e-3) / 1e12 / 80.0)
    assert r["traffic"] == pytest.approx(ex["dram_bytes"] * pairs)
    assert bench.roofline("k_shade", ms, pairs, 3, peaks, clk, captured=False)["traffic"] is None
    # whole-job throughput of N replicas: all ranks' pixels over the slowest rank's time
    assert bench.job_mpix_s(4, 1920 * 1080, 100.0) == pytest.approx(4 * 1920 * 1080 / 0.1 / 1e6)
