"""Plain, slow FP64 CPU oracle of the MB3DGS rendering path.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline / reference legs, never by the product path.

Everything is float64 PyTorch on the CPU, vectorised over (pixel, Gaussian)
pairs but otherwise written step by step in the paper's order and notation.
Library primitives used as steps: ``torch.linalg.solve`` (Hankel and
Vandermonde systems), ``torch.linalg.eigvals`` (companion-matrix roots of the
kernel polynomial), ``torch.special.erf/erfc`` and ``scipy.special.ndtri``
(inverse normal CDF).  Autograd through these functions gives the oracle's
gradient (roots are differentiated implicitly by one Newton step).

Paper references are to "Moment-Based 3D Gaussian Splatting" (MB3DGS):
Eq. 1-3 (volume rendering), Eq. 4-6 (ray-parameterised 1D Gaussian, App. A),
Eq. 7 (quadrature, App. B), Eq. 8 (moment bounds, Sec. 3.2), Eq. 10-12
(power-moment recurrence, App. C), Eq. 15 (opacity rescaling), Eq. 17-21
(confidence-interval proxy, App. C "Rasterisation"), consistency penalty
(Sec. 3.4, App. D "Regularisation").

Readings adopted where the paper is silent or garbled: power transform of Barron (2025), f(x) = |l-1|/l * ((x/|l-1|
+ 1)^l - 1) with l = -1.5 applied to 2t; near bound t_n = 0.01, far bound
t_f = 1e6 (moments use the t_f -> inf closed forms); boundary term of the
recurrence with a "+" sign and the linearised distance u_n (the appendix
derivation); moment bias b <- (1-alpha) b + alpha b*, b* the moments of
U[0,1]; bounds interpolated as tau = m0 ((1-beta) L + beta U); sample nodes
x_j = Phi^-1((j+1/2)/(N+1)), j = 0..N; the 0/0 limit of the quadrature
weight; axis-aligned proxy rectangle with pixel-centre inclusion; frustum
culling with a sphere of radius r_mult * max(s).

Parity pins: every function here is checked by ``tests/test_oracle_pins.py``
against closed forms, brute-force integration / ray marching, exact discrete
measures and invariants.  None of those checks re-types the formula under
test.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch
from scipy.special import ndtri

DT = torch.float64


# ----------------------------------------------------------------------------
# configuration
# ----------------------------------------------------------------------------
@dataclass
class OracleConfig:
    n: int = 4                  # 2n+1 power moments (Sec. 3.2, n = 4)
    n_intervals: int = 3        # N quadrature intervals (power-moment figures use N = 3)
    kappa: float = 3.0          # sample-spacing scale (App. B, kappa = 3)
    beta: float = 0.25          # bound interpolation (Sec. 3.2, beta = 0.25)
    conf_c: float = 0.01        # proxy confidence level (App. C, c = 0.01)
    warp_lambda: float = -1.5   # power-transform lambda (Sec. 3.2)
    t_near: float = 0.01
    t_far: float = 1.0e6
    eps: float = 1.0e-6         # rescaling clamp (Eq. 15)
    bias_alpha: float = 1.0e-3  # moment bias towards U[0,1] (reading; see module docstring)
    m_min: float = 1.0e-7       # below this total optical depth the pixel is treated as empty
    r_mult: float = 3.0         # culling sphere radius in units of max scale
    bg: tuple = (0.0, 0.0, 0.0)
    basis: str = "power"        # "power" (Eq. 10-12) or "trig" (Eq. 13-14)
    trig_theta: float = 0.5 * math.pi   # wrapping angle theta of the trigonometric moments (reading)


# ----------------------------------------------------------------------------
# warp g-hat (Sec. 3.2, power transform of Barron 2025)
# ----------------------------------------------------------------------------
def power_transform(x, lam):
    """Barron's power transform f_lambda(x) = |l-1|/l * ((x/|l-1| + 1)^l - 1)."""
    a = abs(lam - 1.0)
    return (a / lam) * ((x / a + 1.0) ** lam - 1.0)


def power_transform_deriv(x, lam):
    a = abs(lam - 1.0)
    return (x / a + 1.0) ** (lam - 1.0)


def warp(t, cfg: OracleConfig):
    """g-hat(t) = (f(t) - f(t_n)) / (f(t_f) - f(t_n)) with f(t) = f_lambda(2t)
    (Sec. 3.2); returns (g-hat, d g-hat / dt)."""
    lam = cfg.warp_lambda
    fn = power_transform(2.0 * cfg.t_near, lam)
    ff = power_transform(2.0 * cfg.t_far, lam)
    den = ff - fn
    g = (power_transform(2.0 * t, lam) - fn) / den
    dg = 2.0 * power_transform_deriv(2.0 * t, lam) / den
    return g, dg


# ----------------------------------------------------------------------------
# Gaussian parameterisation (Sec. 3.1: Sigma = R S S^T R^T, 3DGS quaternions)
# ----------------------------------------------------------------------------
def quat_to_rotmat(q):
    q = q / torch.linalg.norm(q, dim=-1, keepdim=True)
    w, x, y, z = q.unbind(-1)
    R = torch.stack([
        1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
        2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
        2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)
    return R.reshape(q.shape[:-1] + (3, 3))


def sh_basis(d, deg):
    """Real spherical harmonics (Condon-Shortley phase) up to degree 3,
    index l*l + l + m.  Sec. 3.1: emission (L_e)_i(d) from SH up to l = 3."""
    x, y, z = d.unbind(-1)
    pi = math.pi
    out = [torch.full_like(x, 0.5 / math.sqrt(pi))]
    if deg >= 1:
        c1 = math.sqrt(3.0 / (4.0 * pi))
        out += [-c1 * y, c1 * z, -c1 * x]
    if deg >= 2:
        c2 = 0.5 * math.sqrt(15.0 / pi)
        c20 = 0.25 * math.sqrt(5.0 / pi)
        c22 = 0.25 * math.sqrt(15.0 / pi)
        out += [c2 * x * y, -c2 * y * z, c20 * (2 * z * z - x * x - y * y), -c2 * x * z,
                c22 * (x * x - y * y)]
    if deg >= 3:
        c33 = 0.25 * math.sqrt(35.0 / (2.0 * pi))
        c32 = 0.5 * math.sqrt(105.0 / pi)
        c31 = 0.25 * math.sqrt(21.0 / (2.0 * pi))
        c30 = 0.25 * math.sqrt(7.0 / pi)
        c32b = 0.25 * math.sqrt(105.0 / pi)
        out += [-c33 * y * (3 * x * x - y * y), c32 * x * y * z,
                -c31 * y * (4 * z * z - x * x - y * y), c30 * z * (2 * z * z - 3 * x * x - 3 * y * y),
                -c31 * x * (4 * z * z - x * x - y * y), c32b * z * (x * x - y * y),
                -c33 * x * (x * x - 3 * y * y)]
    return torch.stack(out, -1)


def sh_color(sh, d, deg):
    """Colour = max(0, sum_k f_k Y_k(d) + 1/2) per channel (3DGS convention)."""
    Y = sh_basis(d, deg)                                  # (..., K)
    return torch.clamp((Y[..., :, None] * sh).sum(-2) + 0.5, min=0.0)


# ----------------------------------------------------------------------------
# camera helpers
# ----------------------------------------------------------------------------
def _t(a):
    return torch.as_tensor(np.asarray(a), dtype=DT)


def camera_tensors(cam):
    V = _t(cam.viewmat)
    Rv = V[:3, :3]
    tv = V[:3, 3]
    Kinv = torch.tensor([[1.0 / cam.fx, 0.0, -cam.cx / cam.fx],
                         [0.0, 1.0 / cam.fy, -cam.cy / cam.fy],
                         [0.0, 0.0, 1.0]], dtype=DT)
    eye_w = -Rv.T @ tv
    return Rv, tv, Kinv, eye_w


def pixel_rays(cam, px, py):
    """d_p = normalize(K^-1 (x + 1/2, y + 1/2, 1)) in camera space (Sec. 3.3)."""
    _, _, Kinv, _ = camera_tensors(cam)
    p = torch.stack([px.to(DT) + 0.5, py.to(DT) + 0.5, torch.ones_like(px, dtype=DT)], -1)
    d = p @ Kinv.T
    return d / torch.linalg.norm(d, dim=-1, keepdim=True)


# ----------------------------------------------------------------------------
# Eq. 4-6: ray-parameterised 1D Gaussian (App. A)
# ----------------------------------------------------------------------------
def gaussian_1d(o_g, d_g, w):
    """Given o_g = S^-1 R^T (o - mu), d_g = S^-1 R^T d (d unit), return
    (Sigma_i, mu_i, w-hat_i) with Sigma^2 = 1/(d_g.d_g), mu = -(o_g.d_g)/(d_g.d_g),
    w-hat = w e^K, K = -1/2 o_g.o_g + 1/2 (o_g.d_g)^2 / (d_g.d_g)  (Eq. 5-6)."""
    dd = (d_g * d_g).sum(-1)
    od = (o_g * d_g).sum(-1)
    oo = (o_g * o_g).sum(-1)
    Sigma = torch.sqrt(1.0 / dd)
    mu = -od / dd
    K = -0.5 * oo + 0.5 * od * od / dd
    return Sigma, mu, w * torch.exp(K)


# ----------------------------------------------------------------------------
# Eq. 10-12: analytic power moments of one Gaussian (App. C, t_f -> inf)
# ----------------------------------------------------------------------------
def gaussian_moments(mu, Sigma, w_hat, cfg: OracleConfig):
    """(m-hat_k)_i for k = 0..2n of one 1D Gaussian w-hat exp(-(t-mu)^2/(2 Sigma^2))
    on [t_n, inf), with g-hat linearised at mu: u_t = g(mu) + g'(mu)(t - mu).

    m0 = w Sigma sqrt(pi/2) (1 - erf(b_n)),  b_n = (t_n - mu)/(sqrt(2) Sigma)
    m1 = g m0 + g' w Sigma^2 e^{-b_n^2}
    mk = g m_{k-1} + g'^2 Sigma^2 (k-1) m_{k-2} + g' w Sigma^2 u_n^{k-1} e^{-b_n^2}
    (the boundary term enters with "+": it is -B_i(k) with B_i(k) negative,
    App. C; u_n = g(mu) + g'(mu)(t_n - mu) as in the derivation).
    g-hat is defined on [t_n, t_f] only: for a Gaussian whose mean lies before
    the near bound (mu < t_n) the linearisation point is t_n (reading), i.e.
    u_t = g(c) + g'(c)(t - c) with c = max(mu, t_n), written a + s (t - mu)."""
    tn = cfg.t_near
    c = torch.clamp(mu, min=tn)
    gc, dg = warp(c, cfg)
    g = gc + dg * (mu - c)
    bn = (tn - mu) / (math.sqrt(2.0) * Sigma)
    en = torch.exp(-bn * bn)
    un = g + dg * (tn - mu)
    S2 = Sigma * Sigma
    ms = [w_hat * Sigma * math.sqrt(math.pi / 2.0) * torch.special.erfc(bn)]
    ms.append(g * ms[0] + dg * w_hat * S2 * en)
    for k in range(2, 2 * cfg.n + 1):
        ms.append(g * ms[k - 1] + dg * dg * S2 * (k - 1) * ms[k - 2]
                  + dg * w_hat * S2 * un ** (k - 1) * en)
    return torch.stack(ms, -1)


# ----------------------------------------------------------------------------
# Sec. 3.2 / Eq. 8: moment bounds via the canonical representation
# ----------------------------------------------------------------------------
def biased_moments(m, cfg: OracleConfig):
    """Normalise by m0 and bias towards the moments of U[0,1]:
    b = (1 - alpha) m/m0 + alpha b*,  b*_k = 1/(k+1)  (reading)."""
    k = torch.arange(2 * cfg.n + 1, dtype=DT)
    bstar = 1.0 / (k + 1.0)
    return (1.0 - cfg.bias_alpha) * m / m[..., :1] + cfg.bias_alpha * bstar


def hankel(b, n):
    idx = torch.arange(n + 1)
    return b[..., idx[:, None] + idx[None, :]]


def _poly_eval(c, x):
    """sum_k c_k x^k and its derivative (c: (..., n+1), x: (..., r))."""
    n = c.shape[-1] - 1
    p = torch.zeros_like(x) + c[..., n:n + 1]
    dp = torch.zeros_like(x)
    for k in range(n - 1, -1, -1):
        dp = dp * x + p
        p = p * x + c[..., k:k + 1]
    return p, dp


def canonical_representation(b, eta, n):
    """Canonical representation of the moments b_0..b_2n with a support point
    at eta (Sec. 3.2): support x_1..x_n = roots of the kernel polynomial
    K(x) = v(x)^T H^-1 v(eta) (H_ij = b_{i+j}, v(x) = (1, x, .., x^n)), and
    weights w' from the Vandermonde system sum_i w'_i x_i^k = b_k, k = 0..n.
    Returns (x[..., n+1] with x_0 = eta, w'[..., n+1])."""
    H = hankel(b, n)
    powers = torch.arange(n + 1, dtype=DT)
    v_eta = eta[..., None] ** powers
    c = torch.linalg.solve(H, v_eta[..., None])[..., 0]      # kernel polynomial coefficients
    with torch.no_grad():
        cd = c.detach()
        comp = torch.zeros(cd.shape[:-1] + (n, n), dtype=DT)
        comp[..., 1:, :-1] = torch.eye(n - 1, dtype=DT)
        comp[..., :, -1] = -cd[..., :n] / cd[..., n:n + 1]
        r0 = torch.linalg.eigvals(comp).real
        for _ in range(3):                                    # Newton polish in FP64
            p, dp = _poly_eval(cd, r0)
            r0 = r0 - p / dp
        r0, _ = torch.sort(r0, dim=-1)
    # one Newton step with a live graph: exact implicit derivative of the roots
    p, dp = _poly_eval(c, r0)
    roots = r0 - p / dp.detach()
    x = torch.cat([eta[..., None], roots], -1)
    V = x[..., None, :] ** powers[:, None]                     # V[k, i] = x_i^k
    # Column equilibration of the Vandermonde system: column i is divided by
    # max(1, |x_i|)^n and the solution multiplied back. The solved system is
    # unchanged, but a root far outside [0, 1] (a kernel polynomial whose
    # leading coefficient passes through zero) no longer leaves the system
    # ill-conditioned and smearing rounding error over the other weights.
    s = torch.clamp(x.detach().abs(), min=1.0) ** n
    wts = torch.linalg.solve(V / s[..., None, :], b[..., :n + 1, None])[..., 0] / s
    return x, wts


def christoffel_weights(b, x, n):
    """1 / K(x, x) with K(x, y) = v(x)^T H^-1 v(y); equals the canonical weights."""
    H = hankel(b, n)
    powers = torch.arange(n + 1, dtype=DT)
    V = x[..., None] ** powers                                  # (..., r, n+1)
    sol = torch.linalg.solve(H[..., None, :, :], V[..., None])[..., 0]
    return 1.0 / (V * sol).sum(-1)


def moment_bounds(b, eta, n):
    """L(eta) = sum_{x_i < eta} w'_i,  U(eta) = sum_{x_i <= eta} w'_i  (Eq. 8)."""
    x, wts = canonical_representation(b, eta, n)
    lower = (x[..., 1:] < eta[..., None]).to(DT)
    upper = (x[..., 1:] <= eta[..., None]).to(DT)
    L = (wts[..., 1:] * lower).sum(-1)
    U = L + wts[..., 0] + (wts[..., 1:] * (upper - lower)).sum(-1)
    return L, U


def optical_depth(m, eta, cfg: OracleConfig):
    """tau(eta) = m0 ((1 - beta) L(eta) + beta U(eta)) on the normalised biased
    moments (Sec. 3.2); tau = 0 where m0 < m_min (empty pixel).
    m: (..., 2n+1) moments, eta: (..., Q) queries sharing the moment vector."""
    m0 = m[..., 0]
    empty = m0 < cfg.m_min
    safe = torch.where(empty[..., None], torch.ones_like(m), m)
    b = biased_moments(safe, cfg)
    Q = eta.shape[-1]
    bq = b[..., None, :].expand(eta.shape + (b.shape[-1],))
    L, U = moment_bounds(bq.reshape(-1, b.shape[-1]), eta.reshape(-1), cfg.n)
    frac = ((1.0 - cfg.beta) * L + cfg.beta * U).reshape(eta.shape)
    tau = m0[..., None] * frac
    return torch.where(empty[..., None].expand(eta.shape), torch.zeros_like(tau), tau)


# ----------------------------------------------------------------------------
# Eq. 13-14: trigonometric moments (App. C "Trigonometric Moments")
# ----------------------------------------------------------------------------
def erfc_first_order(a, b):
    """1 - erf(a + i b) with erf to first order in b around the real axis
    (App. C: erf(a + i b) ~ erf(a) + i b (2 / sqrt(pi)) e^{-a^2}); the real
    part is written erfc(a), which keeps its digits for large a."""
    return torch.complex(torch.special.erfc(a), -b * (2.0 / math.sqrt(math.pi)) * torch.exp(-a * a))


def trig_gaussian_moments(mu, Sigma, w_hat, cfg: OracleConfig, erfc_fn=None):
    """(m-tilde_k)_i, k = 0..n, of one 1D Gaussian on [t_n, inf): the integral
    of e^{i k (2 pi - theta) g-hat(t)} w-hat e^{-(t-mu)^2/(2 Sigma^2)} with g-hat
    linearised as u_t = a + s (t - mu) (Eq. 14, t_f -> inf):
      w-hat sqrt(pi/2) Sigma e^{i alpha a - Sigma^2 beta^2 / 2} (1 - erf(v_n)),
      alpha = k (2 pi - theta),  beta = alpha s,
      v_n = (t_n - mu)/(sqrt2 Sigma) - i Sigma beta / sqrt2,
    with erf of the complex argument to first order in its imaginary part
    (``erfc_fn(re, im)`` = 1 - erf(re + i im); default erfc_first_order, the
    method's).  As for the
    power moments, the warp is linearised at c = max(mu, t_n) (reading), and
    k = 0 is the exact total optical depth.  Returns complex (..., n+1)."""
    erfc_fn = erfc_fn or erfc_first_order
    tn = cfg.t_near
    c = torch.clamp(mu, min=tn)
    gc, dg = warp(c, cfg)
    a = gc + dg * (mu - c)
    k = torch.arange(cfg.n + 1, dtype=DT)
    alpha = k * (2.0 * math.pi - cfg.trig_theta)
    beta = alpha * dg[..., None]
    re = ((tn - mu) / (math.sqrt(2.0) * Sigma))[..., None].expand(beta.shape)
    im = -Sigma[..., None] * beta / math.sqrt(2.0)
    one_minus_erf = erfc_fn(re, im)
    mag = (w_hat * math.sqrt(math.pi / 2.0) * Sigma)[..., None] * torch.exp(-0.5 * (Sigma[..., None] * beta) ** 2)
    phase = alpha * a[..., None]
    return torch.complex(mag * torch.cos(phase), mag * torch.sin(phase)) * one_minus_erf


def trig_biased_moments(m, cfg: OracleConfig):
    """Normalise by m0 and bias towards the moments of the uniform distribution
    on the angles [0, 2 pi - theta] that the depths map to (reading):
    c = (1 - alpha) m/m0 + alpha c*,  c*_k = (e^{i k A} - 1)/(i k A), A = 2 pi - theta."""
    A = 2.0 * math.pi - cfg.trig_theta
    k = torch.arange(1, cfg.n + 1, dtype=DT)
    cstar = torch.cat([torch.ones(1, dtype=torch.complex128), (torch.exp(1j * k * A) - 1.0) / (1j * k * A)])
    return (1.0 - cfg.bias_alpha) * m / m[..., :1] + cfg.bias_alpha * cstar


def toeplitz_gram(c, n):
    """Gram matrix G_jl = <z^j, z^l> = int conj(z)^j z^l d(measure) = c_{l-j} of
    the monomials on the unit circle (c_{-k} = conj(c_k))."""
    idx = torch.arange(n + 1)
    d = idx[None, :] - idx[:, None]
    full = torch.cat([torch.conj(c[..., 1:].flip(-1)), c], -1)          # c_{-n} .. c_n
    return full[..., d + n]


def trig_canonical_representation(c, phi, n):
    """Canonical representation on the unit circle of the moments c_0..c_n
    with a node at z_0 = e^{i phi} (Gauss-Szego rule through z_0): the other
    nodes are the n roots of the kernel polynomial K(z, z_0) = v(z)^T G^-1
    conj(v(z_0)), which lie on the unit circle, and the weights are
    1 / K(z_i, z_i) (Christoffel function).  Returns (z[..., n+1], w[..., n+1])."""
    G = toeplitz_gram(c, n)
    powers = torch.arange(n + 1, dtype=DT)
    z0 = torch.polar(torch.ones_like(phi), phi)
    v0 = z0[..., None] ** powers
    a = torch.linalg.solve(G, torch.conj(v0)[..., None])[..., 0]      # K(z, z0) = sum_j a_j z^j

    def horner(coef, r):
        p = torch.zeros_like(r) + coef[..., n:n + 1]
        dp = torch.zeros_like(r)
        for k in range(n - 1, -1, -1):
            dp = dp * r + p
            p = p * r + coef[..., k:k + 1]
        return p, dp

    with torch.no_grad():
        ad = a.detach()
        comp = torch.zeros(ad.shape[:-1] + (n, n), dtype=ad.dtype)
        comp[..., 1:, :-1] = torch.eye(n - 1, dtype=ad.dtype)
        comp[..., :, -1] = -ad[..., :n] / ad[..., n:n + 1]
        r0 = torch.linalg.eigvals(comp)
        for _ in range(3):                                              # Newton polish in FP64
            p, dp = horner(ad, r0)
            r0 = r0 - p / dp
    # one Newton step with a live graph: exact implicit derivative of the roots
    p, dp = horner(a, r0)
    r = r0 - p / dp.detach()
    z = torch.cat([z0[..., None], r], -1)
    V = z[..., :, None] ** powers                                       # (..., n+1 nodes, n+1)
    sol = torch.linalg.solve(G[..., None, :, :], torch.conj(V)[..., None])[..., 0]
    K = (V * sol).sum(-1).real
    return z, 1.0 / K


def trig_moment_bounds(c, phi, cfg: OracleConfig):
    """Bounds of the normalised measure of the angles [cut, phi): with angles
    measured from the cut psi_c = 2 pi - theta/2 in the middle of the empty
    wrapping zone (reading), L = sum of the weights of the other nodes before
    phi, U = L + the weight of the node at phi."""
    z, w = trig_canonical_representation(c, phi, cfg.n)
    cut = 2.0 * math.pi - 0.5 * cfg.trig_theta
    ang = torch.remainder(torch.angle(z) - cut, 2.0 * math.pi)
    before = (ang[..., 1:] < ang[..., :1]).to(DT)
    L = (w[..., 1:] * before).sum(-1)
    return L, L + w[..., 0]


def trig_optical_depth(m, eta, cfg: OracleConfig):
    """tau(eta) = m0 ((1 - beta) L + beta U) from the trigonometric moments at
    the angle phi = (2 pi - theta) eta; tau = 0 where m0 < m_min.
    m: (..., n+1) complex moments, eta: (..., Q) warped depths."""
    m0 = m[..., 0].real
    empty = m0 < cfg.m_min
    safe = torch.where(empty[..., None], torch.ones_like(m), m)
    c = trig_biased_moments(safe, cfg)
    cq = c[..., None, :].expand(eta.shape + (c.shape[-1],))
    phi = (2.0 * math.pi - cfg.trig_theta) * eta
    L, U = trig_moment_bounds(cq.reshape(-1, c.shape[-1]), phi.reshape(-1), cfg)
    frac = ((1.0 - cfg.beta) * L + cfg.beta * U).reshape(eta.shape)
    tau = m0[..., None] * frac
    return torch.where(empty[..., None].expand(eta.shape), torch.zeros_like(tau), tau)


# ----------------------------------------------------------------------------
# Eq. 7 quadrature with the App. B sample spacing, penalty (App. D)
# ----------------------------------------------------------------------------
def sample_nodes(N):
    """Standard-normal nodes x_j = Phi^-1((j + 1/2)/(N + 1)), j = 0..N (App. B)."""
    u = (np.arange(N + 1) + 0.5) / (N + 1)
    return torch.as_tensor(ndtri(u), dtype=DT)


def sample_points(mu, Sigma, cfg: OracleConfig):
    """t_j = clamp(mu + kappa Sigma x_j, t_n, t_f)  (App. B)."""
    x = sample_nodes(cfg.n_intervals)
    t = mu[..., None] + cfg.kappa * Sigma[..., None] * x
    return torch.clamp(t, cfg.t_near, cfg.t_far)


def quadrature(mu, Sigma, w_hat, t, tau, cfg: OracleConfig):
    """Per-Gaussian opacity O_i and penalty P_i (Eq. 7 with (L_e)_i = 1, App. B;
    App. D penalty).  t, tau: (..., N+1) sample points and optical depths.

    O_i = sum_j (T_j - T_{j+1}) sigma_i(t_j) / sigma(t_j),
    sigma(t_j) = (tau_{j+1} - tau_j) / Delta_j  (density at the left edge).
    (T_j - T_{j+1}) is written T_j (1 - e^{-dtau}), identical since T = e^{-tau};
    the 0/0 limit dtau -> 0 gives T_j sigma_i(t_j) Delta_j."""
    T = torch.exp(-tau)
    Delta = t[..., 1:] - t[..., :-1]
    dtau = torch.clamp(tau[..., 1:] - tau[..., :-1], min=0.0)
    sig_i = w_hat[..., None] * torch.exp(-(t[..., :-1] - mu[..., None]) ** 2
                                         / (2.0 * Sigma[..., None] ** 2))
    small = dtau < 1e-12
    safe = torch.where(small, torch.ones_like(dtau), dtau)
    ratio = torch.where(small, torch.ones_like(dtau), -torch.expm1(-safe) / safe)
    wgt = T[..., :-1] * ratio * sig_i * Delta
    O = wgt.sum(-1)
    b = (t - mu[..., None]) / (math.sqrt(2.0) * Sigma[..., None])
    erfb = torch.special.erf(b)
    tau_ij = w_hat[..., None] * Sigma[..., None] * math.sqrt(math.pi / 2.0) * (erfb[..., 1:] - erfb[..., :-1])
    P = (torch.clamp(tau_ij - dtau, min=0.0) ** 2).sum(-1)
    return O, P


# ----------------------------------------------------------------------------
# culling and confidence-interval proxy (Sec. 3.3, Eq. 17-21, App. C)
# ----------------------------------------------------------------------------
@dataclass
class Preprocessed:
    mu_c: torch.Tensor        # (P,3) camera-space means
    Rg: torch.Tensor          # (P,3,3) Gaussian axes in camera space
    s: torch.Tensor           # (P,3) scales
    w: torch.Tensor           # (P,)  peak densities
    rgb: torch.Tensor         # (P,3) SH colours
    visible: torch.Tensor     # (P,) bool
    rect: torch.Tensor        # (P,4) int64 inclusive pixel ranges x0,y0,x1,y1 (empty if x0>x1)
    mu2d: torch.Tensor        # (P,2)
    half: torch.Tensor        # (P,2) rectangle half extents
    full: torch.Tensor        # (P,) bool: proxy fell back to the full image
    extra: dict = field(default_factory=dict)


def preprocess(scene, cam, cfg: OracleConfig, requires_grad=False, params=None):
    """Per-Gaussian camera-space quantities, culling, SH colour and proxy.
    ``params`` optionally supplies (means, scales, quats, weights, sh) tensors
    (for autograd); otherwise they are taken from ``scene``."""
    if params is None:
        params = tuple(_t(a) for a in (scene.means, scene.scales, scene.quats, scene.weights, scene.sh))
    means, scales, quats, weights, sh = params
    Rv, tv, Kinv, eye_w = camera_tensors(cam)
    mu_c = means @ Rv.T + tv
    Rg = Rv @ quat_to_rotmat(quats)
    dirs = means - eye_w
    dirs = dirs / torch.linalg.norm(dirs, dim=-1, keepdim=True)
    rgb = sh_color(sh, dirs, scene.sh_degree)

    with torch.no_grad():
        mu = mu_c.detach()
        s = scales.detach()
        w = weights.detach()
        R = Rg.detach()
        finite = torch.isfinite(mu).all(-1) & torch.isfinite(s).all(-1) & torch.isfinite(w) \
            & torch.isfinite(R).all(-1).all(-1) & (s > 0).all(-1) & (w > 0)
        # frustum culling with the bounding sphere r = r_mult * max diag(S) (Sec. 3.3)
        r = cfg.r_mult * s.max(-1).values
        W, Hh = cam.width, cam.height
        planes = torch.tensor([[cam.fx, 0.0, cam.cx], [-cam.fx, 0.0, W - cam.cx],
                               [0.0, cam.fy, cam.cy], [0.0, -cam.fy, Hh - cam.cy]], dtype=DT)
        planes = planes / torch.linalg.norm(planes, dim=-1, keepdim=True)
        outside = ((mu @ planes.T) < -r[:, None]).any(-1)
        near = torch.linalg.norm(mu, dim=-1) + r < cfg.t_near
        visible = finite & ~outside & ~near

        # proxy: Sigma^-1 = R S^-2 R^T (camera space, o = 0)
        A = R @ torch.diag_embed(1.0 / (s * s)) @ R.transpose(-1, -2)
        u = mu / torch.linalg.norm(mu, dim=-1, keepdim=True)
        uAu = torch.einsum("pi,pij,pj->p", u, A, u)
        C = (-math.log(1.0 - cfg.conf_c) * torch.sqrt(uAu)) / (math.sqrt(2.0 * math.pi)
                                                              * torch.linalg.norm(u, dim=-1))
        muAmu = torch.einsum("pi,pij,pj->p", mu, A, mu)
        kappa = 2.0 * (torch.log(C) - torch.log(w)) + muAmu
        mvec = torch.einsum("ji,pjk,pk->pi", Kinv, A, mu)          # K^-T A mu
        M = Kinv.T @ A @ Kinv
        Wc = mvec[:, :, None] * mvec[:, None, :] - kappa[:, None, None] * M
        W22 = Wc[:, :2, :2]
        w21 = Wc[:, :2, 2]
        w33 = Wc[:, 2, 2]
        det = W22[:, 0, 0] * W22[:, 1, 1] - W22[:, 0, 1] * W22[:, 1, 0]
        W22inv = torch.stack([W22[:, 1, 1], -W22[:, 0, 1], -W22[:, 1, 0], W22[:, 0, 0]], -1).reshape(-1, 2, 2) \
            / det[:, None, None]
        mu2d = -(W22inv @ w21[:, :, None])[:, :, 0]
        scale = torch.einsum("pi,pij,pj->p", mu2d, W22, mu2d) - w33
        Sig2d = scale[:, None, None] * W22inv
        negdef = (W22[:, 0, 0] < 0) & (det > 0)
        posdef = (Sig2d[:, 0, 0] > 0) & (Sig2d[:, 1, 1] > 0) & \
            (Sig2d[:, 0, 0] * Sig2d[:, 1, 1] - Sig2d[:, 0, 1] * Sig2d[:, 1, 0] > 0)
        weak = w <= C                                               # w-hat <= w <= C everywhere
        visible = visible & ~weak
        valid = (muAmu > kappa) & negdef & posdef & (mu[:, 2] > 0) & torch.isfinite(Sig2d).all(-1).all(-1)
        full = visible & ~valid
        hx = torch.sqrt(torch.clamp(Sig2d[:, 0, 0], min=0.0))
        hy = torch.sqrt(torch.clamp(Sig2d[:, 1, 1], min=0.0))
        # pixel (x, y) contributes iff its centre (x+1/2, y+1/2) lies in the closed rectangle
        x0 = torch.ceil(mu2d[:, 0] - hx - 0.5)
        x1 = torch.floor(mu2d[:, 0] + hx - 0.5)
        y0 = torch.ceil(mu2d[:, 1] - hy - 0.5)
        y1 = torch.floor(mu2d[:, 1] + hy - 0.5)
        big = 1e9
        x0 = torch.nan_to_num(x0, nan=big, posinf=big, neginf=-big).clamp(-big, big)
        x1 = torch.nan_to_num(x1, nan=-big, posinf=big, neginf=-big).clamp(-big, big)
        y0 = torch.nan_to_num(y0, nan=big, posinf=big, neginf=-big).clamp(-big, big)
        y1 = torch.nan_to_num(y1, nan=-big, posinf=big, neginf=-big).clamp(-big, big)
        rect = torch.stack([x0.clamp(min=0), y0.clamp(min=0), x1.clamp(max=W - 1), y1.clamp(max=Hh - 1)],
                           -1).to(torch.int64)
        fullrect = torch.tensor([0, 0, W - 1, Hh - 1], dtype=torch.int64)
        rect = torch.where(full[:, None], fullrect, rect)
        emptyrect = torch.tensor([1, 1, 0, 0], dtype=torch.int64)
        rect = torch.where(visible[:, None], rect, emptyrect)
    return Preprocessed(mu_c, Rg, scales, weights, rgb, visible, rect, mu2d, torch.stack([hx, hy], -1), full,
                        extra=dict(C=C, kappa=kappa, W=Wc, A=A))


def pairs_in_region(rect, x0, y0, w, h):
    """All (gaussian, px, py) with the pixel centre in the Gaussian's rectangle,
    restricted to the pixel region [x0, x0+w) x [y0, y0+h)."""
    gx0 = torch.clamp(rect[:, 0], min=x0)
    gy0 = torch.clamp(rect[:, 1], min=y0)
    gx1 = torch.clamp(rect[:, 2], max=x0 + w - 1)
    gy1 = torch.clamp(rect[:, 3], max=y0 + h - 1)
    nx = torch.clamp(gx1 - gx0 + 1, min=0)
    ny = torch.clamp(gy1 - gy0 + 1, min=0)
    cnt = nx * ny
    g = torch.repeat_interleave(torch.arange(rect.shape[0]), cnt)
    start = torch.cumsum(cnt, 0) - cnt
    local = torch.arange(int(cnt.sum())) - torch.repeat_interleave(start, cnt)
    px = gx0[g] + local % nx[g]
    py = gy0[g] + local // nx[g]
    return g, px, py


# ----------------------------------------------------------------------------
# full forward for one camera
# ----------------------------------------------------------------------------
def render(scene, cam, cfg: OracleConfig = None, region=None, params=None, probes=None,
           requires_grad=False, chunk=200_000, tau_fn=None, pre=None):
    """Render the pixel region (x0, y0, w, h) (default: the full image).

    Returns a dict with rgb (h,w,3), T (h,w) = e^{-m0}, P (h,w) penalty,
    m (h,w,2n+1) moments, O (h,w), S (h,w,3) = sum_i L_i, n_pairs, and
    tau_probe (h,w,Q) = tau(eta) at the probe depths (if ``probes`` given).
    ``tau_fn(pix_index, t)`` replaces the moment-based optical depth (used by
    the exact-tau quadrature pin).  ``pre`` reuses the result of
    ``preprocess(scene, cam, cfg)`` for the same inputs (no gradient)."""
    cfg = cfg or OracleConfig()
    if region is None:
        region = (0, 0, cam.width, cam.height)
    x0, y0, w, h = region
    if pre is None or params is not None:
        pre = preprocess(scene, cam, cfg, params=params)
    g, px, py = pairs_in_region(pre.rect, x0, y0, w, h)
    pix = (py - y0) * w + (px - x0)
    npix = w * h

    d = pixel_rays(cam, px, py)                                   # (n_pairs, 3) camera space
    Rg = pre.Rg[g]
    s = pre.s[g]
    o_g = -torch.einsum("pji,pj->pi", Rg, pre.mu_c[g]) / s          # S^-1 R^T (o - mu), o = 0
    d_g = torch.einsum("pji,pj->pi", Rg, d) / s
    Sigma, mu, w_hat = gaussian_1d(o_g, d_g, pre.w[g])

    trig = cfg.basis == "trig"
    if trig:
        mk = trig_gaussian_moments(mu, Sigma, w_hat, cfg)           # (n_pairs, n+1) complex
        m = torch.zeros(npix, cfg.n + 1, dtype=torch.complex128).index_add(0, pix, mk)
        depth = trig_optical_depth
    else:
        mk = gaussian_moments(mu, Sigma, w_hat, cfg)               # (n_pairs, 2n+1)
        m = torch.zeros(npix, 2 * cfg.n + 1, dtype=DT).index_add(0, pix, mk)
        depth = optical_depth

    t = sample_points(mu, Sigma, cfg)                              # (n_pairs, N+1)
    if tau_fn is None:
        eta, _ = warp(t, cfg)
        taus = []
        for a in range(0, t.shape[0], chunk):
            taus.append(depth(m[pix[a:a + chunk]], eta[a:a + chunk], cfg))
        tau = torch.cat(taus, 0) if taus else torch.zeros_like(t)
    else:
        tau = tau_fn(pix, t)
    O_i, P_i = quadrature(mu, Sigma, w_hat, t, tau, cfg)
    L_i = pre.rgb[g] * O_i[:, None]

    O = torch.zeros(npix, dtype=DT).index_add(0, pix, O_i)
    S = torch.zeros(npix, 3, dtype=DT).index_add(0, pix, L_i)
    P = torch.zeros(npix, dtype=DT).index_add(0, pix, P_i)
    m0 = m[:, 0].real
    Tf = torch.exp(-m0)
    bg = torch.tensor(cfg.bg, dtype=DT)
    rgb = ((1.0 - Tf) / torch.clamp(O, min=cfg.eps))[:, None] * S + Tf[:, None] * bg   # Eq. 15
    out = dict(rgb=rgb.reshape(h, w, 3), T=Tf.reshape(h, w), P=P.reshape(h, w),
               m=m.reshape(h, w, -1), O=O.reshape(h, w), S=S.reshape(h, w, 3),
               n_pairs=int(g.shape[0]), pre=pre)
    if probes is not None:
        q = torch.as_tensor(probes, dtype=DT)
        out["tau_probe"] = depth(m, q.expand(npix, -1), cfg).reshape(h, w, -1)
    out["pairs"] = (g, px, py)
    return out


# ----------------------------------------------------------------------------
# tile binning (by tile key only, no depth sort)
# ----------------------------------------------------------------------------
def bin_tiles(rect, width, height, tile_w=16, tile_h=16):
    """Tile lists of the pixel rectangles: for every tile (row-major) the
    ascending ids of the Gaussians whose rectangle overlaps it.  Returns
    (ids int64, ranges (T,2) int64)."""
    tx = (width + tile_w - 1) // tile_w
    ty = (height + tile_h - 1) // tile_h
    nonempty = (rect[:, 0] <= rect[:, 2]) & (rect[:, 1] <= rect[:, 3])
    gid = torch.nonzero(nonempty)[:, 0]
    r = rect[gid]
    a0 = r[:, 0] // tile_w
    a1 = r[:, 2] // tile_w
    b0 = r[:, 1] // tile_h
    b1 = r[:, 3] // tile_h
    nx = a1 - a0 + 1
    ny = b1 - b0 + 1
    cnt = nx * ny
    g = torch.repeat_interleave(gid, cnt)
    start = torch.cumsum(cnt, 0) - cnt
    local = torch.arange(int(cnt.sum())) - torch.repeat_interleave(start, cnt)
    gi = torch.repeat_interleave(torch.arange(gid.shape[0]), cnt)
    tile = (b0[gi] + local // nx[gi]) * tx + (a0[gi] + local % nx[gi])
    key = tile * (rect.shape[0] + 1) + g
    order = torch.argsort(key)
    ids = g[order]
    counts = torch.bincount(tile, minlength=tx * ty)
    ends = torch.cumsum(counts, 0)
    ranges = torch.stack([ends - counts, ends], -1)
    return ids, ranges


# ----------------------------------------------------------------------------
# references used only by the pins
# ----------------------------------------------------------------------------
def exact_optical_depth(mu, Sigma, w_hat, t, cfg: OracleConfig):
    """Exact tau(t) = sum_i int_{t_n}^{t} sigma_i (erf closed form) for Gaussians
    (..., G) on one ray evaluated at t (..., Q)."""
    s2 = math.sqrt(2.0) * Sigma[..., None, :]
    a = (t[..., :, None] - mu[..., None, :]) / s2
    b = (cfg.t_near - mu[..., None, :]) / s2
    term = w_hat[..., None, :] * Sigma[..., None, :] * math.sqrt(math.pi / 2.0) * (torch.special.erf(a) - torch.special.erf(b))
    return term.sum(-1)


# ----------------------------------------------------------------------------
# oracle gradient: autograd through render (roots differentiated implicitly)
# ----------------------------------------------------------------------------
def render_grad(scene, cam, cfg: OracleConfig = None, dL_drgb=None, dL_dP=None, region=None, dL_dT=None):
    """Gradient of sum(dL_drgb * rgb) + sum(dL_dP * P) + sum(dL_dT * T) over
    the region with respect to (means, scales, quats, weights, sh); proxy
    rectangles and culling are constants (computed without gradient)."""
    cfg = cfg or OracleConfig()
    params = [torch.tensor(np.asarray(a, dtype=np.float64), requires_grad=True)
              for a in (scene.means, scene.scales, scene.quats, scene.weights, scene.sh)]
    out = render(scene, cam, cfg, region=region, params=tuple(params))
    loss = (out["rgb"] * torch.as_tensor(np.asarray(dL_drgb), dtype=DT)).sum()
    if dL_dP is not None:
        loss = loss + (out["P"] * torch.as_tensor(np.asarray(dL_dP), dtype=DT)).sum()
    if dL_dT is not None:
        loss = loss + (out["T"] * torch.as_tensor(np.asarray(dL_dT), dtype=DT)).sum()
    grads = torch.autograd.grad(loss, params, allow_unused=True)
    names = ["means", "scales", "quats", "weights", "sh"]
    res = {n: (g.detach().numpy() if g is not None else np.zeros(p.shape)) for n, g, p in zip(names, grads, params)}
    res["loss"] = float(loss.detach())
    res["out"] = out
    return res


def render_loss(scene, cam, cfg, dL_drgb, dL_dP=None, region=None):
    """The scalar loss of render_grad without gradient (for finite differences)."""
    with torch.no_grad():
        out = render(scene, cam, cfg, region=region)
        loss = (out["rgb"] * torch.as_tensor(np.asarray(dL_drgb), dtype=DT)).sum()
        if dL_dP is not None:
            loss = loss + (out["P"] * torch.as_tensor(np.asarray(dL_dP), dtype=DT)).sum()
    return float(loss), out["pre"].rect
