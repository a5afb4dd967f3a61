// Adjoint of the trigonometric-moment path (Sec. 3.2, Eq. 13-14; App. C
// "Trigonometric Moments"; the adjoint passes of Sec. 3.3).
//
// Pass 1 differentiates each bound query with respect to the pixel's
// Verblunsky coefficients alpha_k (and m0) and sums the result per pixel in
// nine floats: dL/dm0 at fixed alpha, then dL/dRe alpha_k and dL/dIm alpha_k.
// Once per pixel, reverse-mode Levinson-Durbin (FP64, the forward's
// precision) takes that to the biased normalised moments c_k and through the
// normalisation to the raw moments {m0, Re m_k, Im m_k}.  Pass 2 pushes the
// raw-moment adjoint through the moments of each Gaussian (Eq. 14).
//
// Query derivative.  tau = m0 F with F = c_w lam(psi_w) + [right] + s sum_k
// lam(psi_k): s = +1 and c_w = beta when the nodes below psi_w are summed
// (left), s = -1 and c_w = beta - 1 when the nodes above are (right), and lam
// the Christoffel weight 1/K_4(z, z).  The nodes satisfy Theta(psi_k) =
// Theta(psi_w) -/+ 2 pi k, so with Theta' > 0
//   dpsi_k = (dTheta(psi_w) - dTheta(psi_k)) / Theta'(psi_k)      (moments)
//   dpsi_k / dpsi_w = Theta'(psi_w) / Theta'(psi_k),
// and dF = c_w dlam(psi_w) + s sum_k [dlam(psi_k) + lam'(psi_k) dpsi_k], where
// dlam and dTheta at a fixed angle come from one reverse sweep of the Szego
// recursion (szego_adjoint) and lam' = d lam / d psi from a forward-mode
// sweep (szego_trace).
#pragma once
#include "common.cuh"

namespace mb {

constexpr int NTRIG_ADJ = NMOM;   // per-pixel adjoint floats of the trigonometric bounds

// The Szego recursion at z = e^{i psi} with its psi-derivative and the
// states the reverse sweep needs.
struct SzegoTrace {
    float cs, sn;
    float pr[5], pi[5], sr[5], si[5];   // Phi_k(z) and Phi_k^*(z), k = 0..4
    float iE[5];                        // 1 / E_k
    float Q[5];                         // |Phi_k|^2 / E_k, k = 1..4
    float K, dK;                        // K_4(z, z) and dK / dpsi
    float dth;                          // Theta'(psi) = K / (|Phi_4|^2 / E_4)
};

MB_HD void szego_trace(const TrigRecon& T, float psi, SzegoTrace& t) {
    sincosf(psi, &t.sn, &t.cs);
    const float cs = t.cs, sn = t.sn;
    float pr = 1.0f, pi = 0.0f, sr = 1.0f, si = 0.0f;
    float dpr = 0.0f, dpi = 0.0f, dsr = 0.0f, dsi = 0.0f;
    float E = 1.0f, K = 1.0f, dK = 0.0f;
    t.pr[0] = 1.0f; t.pi[0] = 0.0f; t.sr[0] = 1.0f; t.si[0] = 0.0f;
    t.iE[0] = 1.0f; t.Q[0] = 0.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float zr = cs * pr - sn * pi, zi = fmaf(cs, pi, sn * pr);             // z Phi_k
        const float dzr = fmaf(cs, dpr, -sn * dpi) - zi, dzi = fmaf(cs, dpi, sn * dpr) + zr;   // i z Phi_k + z Phi_k'
        const float ar = T.ar[k], ai = T.ai[k];
        const float npr = zr - fmaf(ar, sr, ai * si), npi = zi - fmaf(ar, si, -ai * sr);
        const float nsr = sr - fmaf(ar, zr, -ai * zi), nsi = si - fmaf(ar, zi, ai * zr);
        const float ndpr = dzr - fmaf(ar, dsr, ai * dsi), ndpi = dzi - fmaf(ar, dsi, -ai * dsr);
        const float ndsr = dsr - fmaf(ar, dzr, -ai * dzi), ndsi = dsi - fmaf(ar, dzi, ai * dzr);
        pr = npr; pi = npi; sr = nsr; si = nsi;
        dpr = ndpr; dpi = ndpi; dsr = ndsr; dsi = ndsi;
        E *= T.rho2[k];
        const float iE = fdiv_(1.0f, E);
        t.pr[k + 1] = pr; t.pi[k + 1] = pi; t.sr[k + 1] = sr; t.si[k + 1] = si;
        t.iE[k + 1] = iE;
        // |Phi_k|^2 / E_k scaled before squaring: |Phi_k| can be ~1e-24 next to
        // an atom of a concentrated measure, where its square underflows
        const float rs = sqrtf(iE), qr = pr * rs, qi = pi * rs;
        t.Q[k + 1] = fmaf(qr, qr, qi * qi);
        K += t.Q[k + 1];
        dK = fmaf(2.0f * fmaf(pr, dpr, pi * dpi), iE, dK);
    }
    t.K = K;
    t.dK = dK;
    t.dth = fdiv_(K, t.Q[4]);
}

// Reverse sweep of the recursion for the seeds gK = dL/dK_4(z, z) and gTh =
// dL/dTheta(psi) at a fixed angle: adds dL/dRe alpha_k to A[1 + k] and
// dL/dIm alpha_k to A[5 + k] (rho_k = 1 - |alpha_k|^2 included).  Complex
// adjoints are carried as x-hat = dL/dRe x + i dL/dIm x.
MB_HD void szego_adjoint(const TrigRecon& T, const SzegoTrace& t, float gK, float gTh, float A[NTRIG_ADJ]) {
    // Theta = 5 psi - 2 arg Phi_4^*: S-hat_4 = -2 gTh i S_4 / |S_4|^2, formed
    // from S_4 / max(|Re|, |Im|) (|S_4|^2 itself can underflow)
    float Shr = 0.0f, Shi = 0.0f;
    const float sm = fmaxf(fabsf(t.sr[4]), fabsf(t.si[4]));
    if (gTh != 0.0f && sm > 0.0f) {
        const float ism = 1.0f / sm, ur = t.sr[4] * ism, ui = t.si[4] * ism;
        const float f = 2.0f * gTh * ism / fmaf(ur, ur, ui * ui);
        Shr = f * ui;
        Shi = -f * ur;
    }
    float Phr = 0.0f, Phi = 0.0f;
    float qsum = 0.0f;   // sum_{m > k} |Phi_m|^2 / E_m
#pragma unroll
    for (int k = 3; k >= 0; --k) {
        // K = 1 + sum_m |Phi_m|^2 / E_m
        Phr = fmaf(2.0f * gK * t.iE[k + 1], t.pr[k + 1], Phr);
        Phi = fmaf(2.0f * gK * t.iE[k + 1], t.pi[k + 1], Phi);
        qsum += t.Q[k + 1];
        const float ar = T.ar[k], ai = T.ai[k];
        // E_m (m > k) holds rho_k: rho-hat_k = -gK qsum / rho_k, rho = 1 - |alpha|^2
        const float rh = -gK * fdiv_(qsum, T.rho2[k]);
        float ahr = -2.0f * rh * ar, ahi = -2.0f * rh * ai;
        const float zr = t.cs * t.pr[k] - t.sn * t.pi[k], zi = fmaf(t.cs, t.pi[k], t.sn * t.pr[k]);
        // Phi_{k+1} = z Phi_k - conj(alpha) Phi_k^*,  Phi_{k+1}^* = Phi_k^* - alpha z Phi_k
        const float zhr = Phr - fmaf(ar, Shr, ai * Shi), zhi = Phi - fmaf(ar, Shi, -ai * Shr);
        const float nShr = Shr - fmaf(ar, Phr, -ai * Phi), nShi = Shi - fmaf(ar, Phi, ai * Phr);
        ahr -= fmaf(Phr, t.sr[k], Phi * t.si[k]) + fmaf(zr, Shr, zi * Shi);
        ahi -= fmaf(Phr, t.si[k], -Phi * t.sr[k]) + fmaf(zr, Shi, -zi * Shr);
        A[1 + k] += ahr;
        A[5 + k] += ahi;
        Phr = fmaf(t.cs, zhr, t.sn * zhi);
        Phi = fmaf(t.cs, zhi, -t.sn * zhr);
        Shr = nShr;
        Shi = nShi;
    }
}

// Adjoint of one trigonometric bound query with dL/dtau = gq: adds to the
// pixel's A (dL/dm0 at fixed alpha in A[0], the alpha adjoints after it) and
// dL/d(warped depth) to *geta.
// A query whose derivative is not finite in FP32 (z_w or a node on top of an
// atom of a nearly discrete measure, where Theta' overflows) contributes
// nothing.
MB_HD void trig_query_adjoint(const Params& p, const TrigRecon& T, const TrigQueryRec& q, float gq, float* geta,
                              float Apix[NTRIG_ADJ]) {
    if (T.m0 <= 0.0f || gq == 0.0f) return;
    float A[NTRIG_ADJ];
#pragma unroll
    for (int k = 0; k < NTRIG_ADJ; ++k) A[k] = 0.0f;
    const bool left = q.j <= 2;
    const float s = left ? 1.0f : -1.0f;
    const float cw = left ? p.beta : p.beta - 1.0f;
    const float gm = gq * T.m0;
    float F = left ? 0.0f : 1.0f;
    float ratio = 0.0f;   // sum_k lam'(psi_k) / Theta'(psi_k)
    float ge = 0.0f;
    // the solved nodes first (their seeds need only their own angle), z_w
    // last (its Theta seed sums the nodes' ratios); one copy of the sweeps
#pragma unroll 1
    for (int r = 0; r <= q.ns; ++r) {
        const bool w = r == q.ns;
        SzegoTrace t;
        szego_trace(T, w ? q.psi : (r == 0 ? q.x[0] : q.x[1]), t);
        const float lam = fdiv_(1.0f, t.K);
        const float dlam = -t.dK * lam * lam;
        float gK, gTh;
        if (w) {
            F = fmaf(cw, lam, F);
            gK = -gm * cw * lam * lam;
            gTh = gm * s * ratio;
            if (q.inside) {
                const float nodes = ratio != 0.0f ? s * ratio * t.dth : 0.0f;
                ge = gm * p.trig_A * fmaf(cw, dlam, nodes);
            }
        } else {
            const float rk = fdiv_(dlam, t.dth);
            F = fmaf(s, lam, F);
            ratio += rk;
            gK = -gm * s * lam * lam;
            gTh = -gm * s * rk;
        }
        szego_adjoint(T, t, gK, gTh, A);
    }
    A[0] = gq * F;
    bool ok = isfinite(ge);
#pragma unroll
    for (int k = 0; k < NTRIG_ADJ; ++k) ok = ok && isfinite(A[k]);
    if (!ok) return;
#pragma unroll
    for (int k = 0; k < NTRIG_ADJ; ++k) Apix[k] += A[k];
    *geta += ge;
}

// Per-pixel moment adjoint: from the alpha adjoints (A) through reverse-mode
// Levinson-Durbin to the biased normalised moments c_k, then through c_k =
// (1 - a) m_k / m0 + a c*_k to the raw moments.  psi = {dL/dm0, dL/dRe m_k,
// dL/dIm m_k}, with gm0 the derivative through the rescaling (Eq. 15) and the
// final transmittance.
MB_HD void trig_finish_adjoint(const Params& p, const float I[NMOM], const float A[NTRIG_ADJ], float gm0,
                               float psi[NMOM]) {
    typedef MB_RECON_T real;
#pragma unroll
    for (int k = 0; k < NMOM; ++k) psi[k] = 0.0f;
    psi[0] = gm0;
    if (!(I[0] >= p.m_min) || !isfinite(I[0])) return;
    real vr[4], vi[4];
    LevTrace<real> t;
    const real bias = trig_verblunsky<real>(p, I, vr, vi, &t);
    real ghr[4], ghi[4];   // g_k = conj(alpha_k): g-hat = conj(alpha-hat)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        ghr[k] = (real)A[1 + k];
        ghi[k] = -(real)A[5 + k];
    }
    real Phr[5] = {0, 0, 0, 0, 0}, Phi[5] = {0, 0, 0, 0, 0};   // adjoint of Phi_{k+1}
    real Eh = 0;                                                // adjoint of E_{k+1}
    real chr[5] = {0, 0, 0, 0, 0}, chi[5] = {0, 0, 0, 0, 0};
#pragma unroll
    for (int k = 3; k >= 0; --k) {
        const real gr = t.gr[k], gi = t.gi[k], Ek = t.E[k];
        // E_{k+1} = E_k (1 - |g_k|^2)
        ghr[k] += Eh * Ek * (-2 * gr);
        ghi[k] += Eh * Ek * (-2 * gi);
        real Ehk = Eh * (1 - (gr * gr + gi * gi));
        // Phi_{k+1}[j] = Phi_k[j-1] - g_k conj(Phi_k[k-j])
        real Qhr[5] = {0, 0, 0, 0, 0}, Qhi[5] = {0, 0, 0, 0, 0};   // adjoint of Phi_k
#pragma unroll
        for (int jj = 0; jj <= 4; ++jj) {
            if (jj > k + 1) break;
            const real hr = Phr[jj], hi = Phi[jj];
            if (jj >= 1) { Qhr[jj - 1] += hr; Qhi[jj - 1] += hi; }
            if (jj <= k) {
                const real ur = t.Pr[k][k - jj], ui = t.Pi[k][k - jj];
                ghr[k] -= ur * hr - ui * hi;
                ghi[k] -= ur * hi + ui * hr;
                Qhr[k - jj] -= gr * hr + gi * hi;
                Qhi[k - jj] -= gi * hr - gr * hi;
            }
        }
        // g_k = n_k / E_k
        const real nhr = ghr[k] / Ek, nhi = ghi[k] / Ek;
        Ehk -= (ghr[k] * t.nr[k] + ghi[k] * t.ni[k]) / (Ek * Ek);
        // n_k = sum_j Phi_k[j] c_{j+1}
#pragma unroll
        for (int jj = 0; jj <= 3; ++jj) {
            if (jj > k) break;
            const real cr = t.cr[jj + 1], ci = t.ci[jj + 1];
            Qhr[jj] += cr * nhr + ci * nhi;
            Qhi[jj] += cr * nhi - ci * nhr;
            const real pr = t.Pr[k][jj], pi = t.Pi[k][jj];
            chr[jj + 1] += pr * nhr + pi * nhi;
            chi[jj + 1] += pr * nhi - pi * nhr;
        }
#pragma unroll
        for (int jj = 0; jj <= 4; ++jj) { Phr[jj] = Qhr[jj]; Phi[jj] = Qhi[jj]; }
        Eh = Ehk;
    }
    const real inv0 = real(1) / (real)I[0];
    const real sc = (1 - bias) * inv0;
    real g0 = (real)A[0];
#pragma unroll
    for (int k = 1; k <= 4; ++k) {
        psi[2 * k - 1] = (float)(sc * chr[k]);
        psi[2 * k] = (float)(sc * chi[k]);
        g0 -= sc * inv0 * (chr[k] * (real)I[2 * k - 1] + chi[k] * (real)I[2 * k]);
    }
    psi[0] += (float)g0;
}

// g-hat''(t) of the warp (power transform): G3 (1 + 2t/a)^(lambda-2) =
// g-hat'(t) G3 / (G2 (1 + 2t/a)).
MB_HD float warp_dd(const Params& p, float t, float dg) {
    const float z = fmaf(p.two_over_a, t, 1.0f);
    return p.G3 * fdiv_(dg, p.G2 * z);
}

// int psi d(d mu_i) for the trigonometric moments of one Gaussian: the reverse
// of trig_moments with psi = {dL/dm0, dL/dRe m_k, dL/dIm m_k}; adds to the
// derivatives with respect to (mu, Sigma, w-hat).
MB_HD void trig_moment_adjoint(const Params& p, const Gauss1D& g, const float psi[NMOM], float* g_mu, float* g_Sig,
                               float* g_what) {
    const float cpt = fmaxf(g.mu, p.t_near);
    float a, s;
    warp_g(p, cpt, a, s);
    a = fmaf(s, g.mu - cpt, a);
    const float iSg = 1.0f / g.Sig;
    const float bn = (p.t_near - g.mu) * (0.70710678118654752f * iSg);
    const float ec = erfcf(bn);
    const float en = expf(-bn * bn);
    const float base = g.what * g.Sig * 1.25331413731550025f;
    const float q = g.Sig * s * p.trig_A;
    const float d1 = expf(-0.5f * q * q);
    const float d2 = d1 * d1, d4 = d2 * d2, d8 = d4 * d4;
    const float damp[4] = {d1, d4, d8 * d1, d8 * d8};
    const float im1 = q * 0.79788456080286536f * en;
    float sn, cs;
    sincosf(p.trig_A * a, &sn, &cs);
    float zr = cs, zi = sn;
    float ech = psi[0] * base;        // dL/d erfc(b_n)
    float baseh = psi[0] * ec;        // dL/d base
    float imh = 0.0f, ah = 0.0f, qh = 0.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float kk = (float)(k + 1);
        const float ei = kk * im1;
        const float pr = psi[2 * k + 1], pim = psi[2 * k + 2];
        const float Xr = zr * ec - zi * ei, Xi = fmaf(zr, ei, zi * ec);   // m_k / (base damp_k)
        const float sc = base * damp[k];
        const float R = fmaf(pr, Xr, pim * Xi);                            // Re(conj(psi_k) X)
        baseh = fmaf(damp[k], R, baseh);
        qh = fmaf(base * R, -kk * kk * q * damp[k], qh);                   // d damp_k / dq = -k^2 q damp_k
        ech = fmaf(sc, fmaf(pr, zr, pim * zi), ech);
        imh = fmaf(sc * kk, fmaf(-pr, zi, pim * zr), imh);
        ah = fmaf(sc * kk * p.trig_A, fmaf(pim, Xr, -pr * Xi), ah);       // dm_k / da = i k A m_k
        const float nr = zr * cs - zi * sn;
        zi = fmaf(zr, sn, zi * cs);
        zr = nr;
    }
    // im1 = q sqrt(2/pi) e_n
    qh = fmaf(imh, 0.79788456080286536f * en, qh);
    const float enh = imh * q * 0.79788456080286536f;
    // erfc(b_n) and e_n = exp(-b_n^2)
    const float bnh = -1.12837916709551257f * en * ech - 2.0f * bn * en * enh;
    // q = Sigma s A, base = w-hat Sigma sqrt(pi/2), b_n = (t_n - mu) / (sqrt2 Sigma)
    const float sh = qh * g.Sig * p.trig_A;
    float mu_h = ah * s - bnh * (0.70710678118654752f * iSg);
    if (g.mu > p.t_near) mu_h = fmaf(sh, warp_dd(p, cpt, s), mu_h);   // s = g-hat'(mu) when mu > t_n
    *g_mu += mu_h;
    *g_Sig += baseh * g.what * 1.25331413731550025f + qh * s * p.trig_A - bnh * bn * iSg;
    *g_what += baseh * g.Sig * 1.25331413731550025f;
}

}  // namespace mb
