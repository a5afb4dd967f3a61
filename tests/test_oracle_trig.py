"""Pins of the oracle's trigonometric-moment path (Eq. 13-14, App. C
"Trigonometric Moments") against facts that do not come from the oracle:

* the closed form of one Gaussian's moment, with the complex erf evaluated
  exactly (scipy), equals numerical integration of the linearised integrand
  (this pins alpha, beta, the damping factor, the phase and the boundary
  argument v_n, before the method's first-order erf step);
* the first-order erf step of App. C is exact for a real argument and its
  error shrinks quadratically with the imaginary part;
* k = 0 is the exact total optical depth (the power path's m0);
* the canonical representation on the unit circle reproduces the moments,
  puts its nodes on the circle (a theorem, not imposed by the solver) and
  agrees with the zeros of the para-orthogonal polynomial built by the Szego
  recursion (a different algorithm, written here);
* a measure that is itself a Gauss-Szego rule is its own representation, so
  its bounds at that rule's prescribed node are exact;
* the bounds lie in [0, 1] with L <= U, and contain the exact distribution
  function of random measures on the support arc in all but a small share of
  queries (they are the circle analogue of the Eq. 8 bounds with the cut in
  the wrapping zone, not strict bounds);
* a scene of one colour renders with the monochrome identity of Eq. 15.
"""
import math

import numpy as np
import pytest
import scipy.integrate as si
import scipy.special as ss
import torch

import oracle as O
import scenes

DT = torch.float64


def _lin(mu, cfg):
    """Linearised warp u_t = a + s (t - mu) at c = max(mu, t_n)."""
    c = max(mu, cfg.t_near)
    g, dg = O.warp(torch.tensor(c, dtype=DT), cfg)
    return float(g) + float(dg) * (mu - c), float(dg)


@pytest.mark.parametrize("mu,Sigma,w", [(2.0, 0.05, 3.0), (0.5, 0.2, 1.0), (0.02, 0.03, 2.0),
                                        (-0.1, 0.3, 0.7), (5.0, 1.5, 0.2)])
def test_trig_closed_form_with_exact_erf_matches_integration(mu, Sigma, w):
    cfg = O.OracleConfig(basis="trig")

    def erfc_exact(re, im):
        z = re.numpy() + 1j * im.numpy()
        return torch.as_tensor(ss.erfc(z))

    m = O.trig_gaussian_moments(torch.tensor([mu], dtype=DT), torch.tensor([Sigma], dtype=DT),
                                torch.tensor([w], dtype=DT), cfg, erfc_fn=erfc_exact)[0].numpy()
    a, s = _lin(mu, cfg)
    lo, hi = cfg.t_near, mu + 40.0 * Sigma
    for k in range(cfg.n + 1):
        al = k * (2.0 * math.pi - cfg.trig_theta)

        def f(t, part):
            v = w * np.exp(-(t - mu) ** 2 / (2 * Sigma ** 2)) * np.exp(1j * al * (a + s * (t - mu)))
            return v.real if part == 0 else v.imag
        pts = [mu] if lo < mu < hi else None
        re = si.quad(f, lo, hi, args=(0,), limit=400, epsabs=1e-14, epsrel=1e-12, points=pts)[0]
        im = si.quad(f, lo, hi, args=(1,), limit=400, epsabs=1e-14, epsrel=1e-12, points=pts)[0]
        scale = w * Sigma
        assert abs(m[k].real - re) <= 1e-9 * scale and abs(m[k].imag - im) <= 1e-9 * scale, (k, m[k], re, im)


def test_first_order_erf_step():
    a = torch.linspace(-3.0, 3.0, 61, dtype=DT)
    exact0 = torch.as_tensor(ss.erfc(a.numpy() + 0j))
    assert torch.allclose(O.erfc_first_order(a, torch.zeros_like(a)), exact0, atol=1e-15)
    errs = []
    for b in [0.2, 0.1, 0.05]:
        bb = torch.full_like(a, b)
        ex = torch.as_tensor(ss.erfc(a.numpy() + 1j * b))
        errs.append(float((O.erfc_first_order(a, bb) - ex).abs().max()))
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5, errs
    # the error is localised: far from the axis origin it carries e^{-a^2}
    far = torch.tensor([4.0, -4.0], dtype=DT)
    ex = torch.as_tensor(ss.erfc(far.numpy() + 0.5j))
    assert float((O.erfc_first_order(far, torch.full_like(far, 0.5)) - ex).abs().max()) < 1e-6


def test_zeroth_trig_moment_is_the_exact_optical_depth():
    cfg = O.OracleConfig(basis="trig")
    rng = np.random.default_rng(0)
    mu = torch.as_tensor(rng.uniform(-0.5, 6.0, 50))
    Sig = torch.as_tensor(rng.uniform(0.01, 1.0, 50))
    w = torch.as_tensor(rng.uniform(0.1, 5.0, 50))
    mt = O.trig_gaussian_moments(mu, Sig, w, cfg)[:, 0]
    mp = O.gaussian_moments(mu, Sig, w, O.OracleConfig())[:, 0]
    assert torch.allclose(mt.real, mp, rtol=1e-13, atol=0) and float(mt.imag.abs().max()) == 0.0


def _random_measure(rng, cfg, n_atoms):
    A = 2.0 * math.pi - cfg.trig_theta
    ang = rng.uniform(0.0, A, n_atoms)
    wts = rng.uniform(0.1, 1.0, n_atoms)
    k = np.arange(cfg.n + 1)
    mom = (wts[None, :] * np.exp(1j * k[:, None] * ang[None, :])).sum(1)
    return ang, wts / wts.sum(), torch.as_tensor(mom / wts.sum())


def test_canonical_representation_reproduces_moments_on_the_circle():
    cfg = O.OracleConfig(basis="trig")
    rng = np.random.default_rng(1)
    for trial in range(40):
        _, _, mom = _random_measure(rng, cfg, int(rng.integers(2, 20)))
        c = O.trig_biased_moments(mom[None], cfg)[0]
        phi = torch.as_tensor(rng.uniform(0.0, 2.0 * math.pi - cfg.trig_theta, 3))
        z, w = O.trig_canonical_representation(c[None].expand(3, -1), phi, cfg.n)
        assert torch.allclose(z.abs(), torch.ones_like(w), atol=1e-10)
        assert (w > 0).all()
        for k in range(cfg.n + 1):
            rep = (w * z ** k).sum(-1)
            assert torch.allclose(rep, c[k].expand(3), atol=1e-10), (k, rep, c[k])


def _szego_nodes(c, w0, n):
    """Zeros of the para-orthogonal polynomial z phi_n(z) - t phi_n^*(z) with
    t chosen so that w0 is a zero, phi_n from the Szego recursion (Levinson)."""
    def ip(p, q):   # int conj(p) q d(measure)
        s = 0j
        for j, pj in enumerate(p):
            for l, ql in enumerate(q):
                d = l - j
                s += np.conj(pj) * ql * (c[d] if d >= 0 else np.conj(c[-d]))
        return s
    P = np.array([1.0 + 0j])
    for k in range(n):
        Ps = np.conj(P[::-1])
        zP = np.concatenate([[0], P])
        Psp = np.concatenate([Ps, [0]])
        a = ip(np.array([1.0]), zP) / ip(np.array([1.0]), Psp)
        P = zP - a * Psp
    Ps = np.conj(P[::-1])
    ev = lambda p, z: np.polyval(p[::-1], z)
    t = w0 * ev(P, w0) / ev(Ps, w0)
    para = np.concatenate([[0], P]) - t * np.concatenate([Ps, [0]])
    return np.roots(para[::-1])


def test_nodes_are_the_para_orthogonal_zeros():
    cfg = O.OracleConfig(basis="trig")
    rng = np.random.default_rng(2)
    for trial in range(25):
        _, _, mom = _random_measure(rng, cfg, int(rng.integers(3, 15)))
        c = O.trig_biased_moments(mom[None], cfg)[0]
        phi = float(rng.uniform(0.0, 2.0 * math.pi - cfg.trig_theta))
        z, _ = O.trig_canonical_representation(c[None], torch.tensor([phi], dtype=DT), cfg.n)
        ref = _szego_nodes(c.numpy(), np.exp(1j * phi), cfg.n)
        a = np.sort(np.mod(np.angle(z[0].numpy()), 2 * np.pi))
        b = np.sort(np.mod(np.angle(ref), 2 * np.pi))
        assert np.allclose(a, b, atol=1e-9), (a, b)


def test_a_gauss_szego_measure_is_its_own_representation():
    cfg = O.OracleConfig(basis="trig", bias_alpha=0.0)
    rng = np.random.default_rng(3)
    A = 2.0 * math.pi - cfg.trig_theta
    cut = 2.0 * math.pi - 0.5 * cfg.trig_theta
    for trial in range(20):
        _, _, mom = _random_measure(rng, cfg, 12)
        phi0 = float(rng.uniform(0.1, A - 0.1))
        z, w = O.trig_canonical_representation(mom[None], torch.tensor([phi0], dtype=DT), cfg.n)
        z, w = z[0], w[0]
        # the rule's own moments, and its bounds at its prescribed node
        mom2 = torch.stack([(w * z ** k).sum() for k in range(cfg.n + 1)])
        L, U = O.trig_moment_bounds(mom2[None], torch.tensor([phi0], dtype=DT), cfg)
        rel = np.mod(np.angle(z.numpy()) - cut, 2 * np.pi)
        exact_L = float(w[1:][torch.as_tensor(rel[1:] < rel[0])].sum())
        assert abs(float(L[0]) - exact_L) < 1e-9 and abs(float(U[0]) - (exact_L + float(w[0]))) < 1e-9


def test_bounds_range_and_containment_rate():
    cfg = O.OracleConfig(basis="trig")
    rng = np.random.default_rng(4)
    A = 2.0 * math.pi - cfg.trig_theta
    cut = 2.0 * math.pi - 0.5 * cfg.trig_theta
    n_bad, n_all, worst = 0, 0, 0.0
    for trial in range(300):
        ang, wts, mom = _random_measure(rng, cfg, int(rng.integers(1, 30)))
        c = O.trig_biased_moments(mom[None], cfg)[0]
        phi = torch.as_tensor(rng.uniform(0.0, A, 6))
        L, U = O.trig_moment_bounds(c[None].expand(6, -1), phi, cfg)
        assert (L >= -1e-12).all() and (U <= 1.0 + 1e-9).all() and (L <= U + 1e-12).all()
        # exact distribution function of the biased measure on [cut, phi)
        a = cfg.bias_alpha
        rel = np.mod(ang - cut, 2 * np.pi)
        for q in range(6):
            rq = np.mod(float(phi[q]) - cut, 2 * np.pi)
            F = (1 - a) * wts[rel < rq].sum() + a * float(phi[q]) / A
            v = max(float(L[q]) - F, F - float(U[q]), 0.0)
            n_all += 1
            n_bad += v > 1e-9
            worst = max(worst, v)
    assert n_bad / n_all < 0.01 and worst < 0.02, (n_bad, n_all, worst)


def test_monochrome_identity_with_trig_moments():
    sc = scenes.scene_uniform(200, 8)
    sc.sh[:] = 0.0
    sc.sh[:, 0, :] = (np.array([0.3, 0.6, 0.9]) - 0.5) / (0.5 / math.sqrt(math.pi))
    cam = scenes.look_at((0, 0, -3), width=24, height=20)
    out = O.render(sc, cam, O.OracleConfig(basis="trig", n_intervals=5))
    col = torch.tensor([0.3, 0.6, 0.9], dtype=DT)
    T = out["T"][..., None]
    ok = out["O"] >= 1e-6
    ref = (1.0 - T) * col
    assert torch.allclose(out["rgb"][ok], ref[ok], atol=1e-12)
