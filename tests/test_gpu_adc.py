"""GPU parity of the adaptive density control (Sec. 3.4; App. D) through the
C ABI against the oracle (oracle/mb3dgs_adc.py, pinned in
test_oracle_adc.py).

Bar: decisions, counts and output order bit-exact (they are integer work,
taken in float32 on both sides in the same operation order); the float32
sums of the gradient statistics bit-exact (correctly rounded additions in
the same order); copied and halved values bit-exact; the split offsets, the
view-independent opacity and the initial weights within 2e-6 relative (FP32
against the FP64 oracle)."""
import numpy as np
import pytest
import torch

import helpers
import oracle as O
import scenes

pytestmark = pytest.mark.gpu
A = O.adc
NAMES = ["means", "scales", "quats", "weights", "sh"]


def _adc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_11800_gb300 import GaussianTensors, adc
    return GaussianTensors, adc


def test_opacity_and_initial_weights():
    GaussianTensors, adc = _adc()
    sc = scenes.scene_uniform(100_000, 21)
    g = GaussianTensors.from_scene(sc)
    o = adc.view_independent_opacity(g.weights, g.scales).cpu().double().numpy()
    ref = A.view_independent_opacity(sc.weights.astype(np.float64), sc.scales.astype(np.float64))
    assert np.abs(o - ref).max() <= 2e-6 * np.maximum(ref, 1e-3).max()
    assert np.all(np.abs(o - ref) <= 2e-6 * ref + 1e-9)
    target = np.random.default_rng(2).uniform(0.01, 0.95, sc.P).astype(np.float32)
    w = adc.init_weights(torch.as_tensor(target, device="cuda"), g.scales).cpu().double().numpy()
    wref = A.init_weights(target.astype(np.float64), sc.scales.astype(np.float64))
    assert np.all(np.abs(w - wref) <= 2e-6 * np.abs(wref))


def test_gradient_statistics_are_exact():
    GaussianTensors, adc = _adc()
    P = 50_000
    rng = np.random.default_rng(3)
    st = adc.DensityStats(P)
    abs_sum = np.zeros((P, 3), np.float32)
    count = np.zeros(P, np.int32)
    for step in range(6):
        d = (rng.normal(size=(P, 3)) * 10.0 ** rng.uniform(-6, -2, (P, 1))).astype(np.float32)
        d[rng.random(P) < 0.25] = 0.0                           # not visible (no gradient)
        vis = None
        if step % 2:
            vis = rng.random(P) < 0.8                           # explicit mask on odd steps
        st.accumulate(torch.as_tensor(d, device="cuda"),
                      None if vis is None else torch.as_tensor(vis, device="cuda"))
        A.accumulate_grad_stats(d, vis, abs_sum, count)
    assert np.array_equal(st.count.cpu().numpy(), count)
    assert np.array_equal(st.abs_sum.cpu().numpy(), abs_sum)


def _stats_for(sc, seed):
    """Summed absolute gradients around the threshold and visible-step counts
    0..3, so that every action and most pruning outcomes occur."""
    rng = np.random.default_rng(seed)
    abs_sum = rng.uniform(0.0, 3.2e-4, (sc.P, 3)).astype(np.float32)
    count = rng.integers(0, 4, sc.P).astype(np.int32)
    return abs_sum, count


def _config(sc):
    smax = sc.scales.max(1)
    o = A.view_independent_opacity(sc.weights, sc.scales)
    return A.ADCConfig(percent_dense=float(np.float32(np.median(smax))), scene_extent=1.0,
                       prune_opacity=float(np.float32(np.quantile(o, 0.2))),
                       big_world=float(np.float32(np.quantile(smax, 0.98))))


def _run(sc, cfg, abs_sum, count):
    GaussianTensors, adc = _adc()
    g = GaussianTensors.from_scene(sc)
    st = adc.DensityStats(sc.P)
    st.abs_sum.copy_(torch.as_tensor(abs_sum))
    st.count.copy_(torch.as_tensor(count))
    c = adc.AdcConfig(**{k: getattr(cfg, k) for k in adc.AdcConfig.__dataclass_fields__})
    new, action, first = adc.densify(g, st, c)
    torch.cuda.synchronize()
    got = {k: getattr(new, k).cpu().double().numpy() for k in NAMES}
    return got, action.cpu().numpy(), first.cpu().numpy()


def _compare(got, ref, split_rows):
    assert len(got["weights"]) == len(ref["weights"])
    if len(ref["weights"]) == 0:
        return
    for k in ["scales", "quats", "weights", "sh"]:
        assert np.array_equal(got[k].reshape(len(got[k]), -1), ref[k].reshape(len(ref[k]), -1)), k
    m, r = got["means"], ref["means"]
    same = ~split_rows
    assert np.array_equal(m[same], r[same])
    if split_rows.any():
        scale = np.abs(r[split_rows]).max(1, keepdims=True) + ref["scales"][split_rows].max(1, keepdims=True)
        assert np.all(np.abs(m[split_rows] - r[split_rows]) <= 2e-6 * scale)


def test_densify_matches_oracle():
    sc = scenes.tiny_scene(P=20_000, seed=22, spread=1.0, deg=1)
    cfg = _config(sc)
    abs_sum, count = _stats_for(sc, 5)
    got, action, first = _run(sc, cfg, abs_sum, count)
    ref, ref_action = A.densify(cfg, sc.means, sc.scales, sc.quats, sc.weights, sc.sh, abs_sum, count)
    print("actions", np.bincount(action, minlength=3), "P_out", len(got["weights"]), "of", sc.P)
    assert np.array_equal(action, ref_action)
    assert len(got["weights"]) == len(ref["weights"])
    assert all(np.bincount(action, minlength=3) > 1000)          # every action occurs
    assert len(ref["weights"]) < 2 * sc.P - 1000                  # and pruning removes particles
    # rows produced by a split
    counts = np.diff(np.append(first, len(got["weights"])))
    split_rows = np.repeat(action == 2, counts)
    _compare(got, ref, split_rows)


def test_densify_edge_cases():
    sc = scenes.scene_uniform(3000, 23)
    abs_sum, count = _stats_for(sc, 6)
    # nothing densified, nothing pruned: the identity
    got, action, first = _run(sc, A.ADCConfig(grad_threshold=np.inf, prune_opacity=0.0, big_world=0.0),
                              abs_sum, count)
    assert np.all(action == 0) and np.array_equal(first, np.arange(sc.P))
    assert np.array_equal(got["means"], sc.means.astype(np.float64))
    # everything pruned: an empty set
    got, action, first = _run(sc, A.ADCConfig(prune_opacity=float(np.float32(0.999999))), abs_sum, count)
    assert len(got["weights"]) == 0 and np.all(first == 0)
    # no Gaussians at all
    none = scenes.scene_uniform(0, 24)
    got, action, first = _run(none, A.ADCConfig(), np.zeros((0, 3), np.float32), np.zeros(0, np.int32))
    assert len(got["weights"]) == 0 and len(action) == 0
    # everything cloned, everything split
    ones = np.ones((sc.P, 3), np.float32)
    cnt = np.ones(sc.P, np.int32)
    for pd, act in [(1e9, 1), (0.0, 2)]:
        cfg = A.ADCConfig(grad_threshold=0.0, percent_dense=pd, prune_opacity=0.0, big_world=0.0)
        got, action, first = _run(sc, cfg, ones, cnt)
        ref, _ = A.densify(cfg, sc.means, sc.scales, sc.quats, sc.weights, sc.sh, ones, cnt)
        assert np.all(action == act) and len(got["weights"]) == 2 * sc.P
        assert np.array_equal(first, 2 * np.arange(sc.P))
        _compare(got, ref, np.full(2 * sc.P, act == 2))


def test_densify_full_size_sampled():
    """The 1M-Gaussian scene: total count and actions of all inputs from the
    GPU, and for 1500 sampled inputs the oracle's outputs of that input alone
    against the GPU's outputs at first[i] .. first[i+1] - 1."""
    sc, _ = helpers.workload("shells1M_1080p")
    cfg = _config(sc)
    abs_sum, count = _stats_for(sc, 7)
    got, action, first = _run(sc, cfg, abs_sum, count)
    end = np.append(first[1:], len(got["weights"]))
    assert np.all(end >= first) and np.all(end - first <= 2)
    idx = np.random.default_rng(8).choice(sc.P, 1500, replace=False)
    for i in idx:
        sl = slice(i, i + 1)
        ref, ref_action = A.densify(cfg, sc.means[sl], sc.scales[sl], sc.quats[sl], sc.weights[sl], sc.sh[sl],
                                    abs_sum[sl], count[sl])
        assert action[i] == ref_action[0], i
        assert end[i] - first[i] == len(ref["weights"]), i
        part = {k: got[k][first[i]:end[i]] for k in NAMES}
        _compare(part, ref, np.full(len(ref["weights"]), action[i] == 2))
