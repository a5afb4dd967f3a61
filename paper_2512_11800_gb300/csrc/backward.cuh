// Adjoint of the moment rasterizer (Sec. 3.3 "Adjoint Rendering", Eq. 22).
//
// Pass 1 (adjoint moments): per pixel, the derivative of the loss with respect
// to the pixel's moment measure, represented as a polynomial Psi(t) of degree
// 2n in standardised warped depth t = (y - c)/s, so that dL = int Psi d(dmu)
// for any perturbation dmu of the raw (unnormalised, unbiased) measure.
// Pass 2 (gradients): per (pixel, Gaussian) pair, the direct derivatives of
// the quadrature, the penalty and the bound queries with respect to the 1D
// Gaussian (mu, Sigma, w-hat), plus int Psi d(d mu_i) through the reverse
// sweep of the moment recurrence, chained to the record coefficients.
//
// Derivative of a bound F = sum_i c_i w_i of the canonical representation:
// with K(s, t) = sum_k h_k pi_k(s) pi_k(t) the kernel of the biased measure,
// x_i the roots of K(., y), w_i = 1/K(x_i, x_i) and w_0 = 1/K(y, y):
//   dw_0 / dmu  = w_0^2 K(., y)^2,
//   dw_i / dmu  = w_i^2 K(., x_i) [K(., x_i) - 2 rho_i K(., y)],
//                 rho_i = d1K(x_i, x_i) / d1K(x_i, y),
//   dw_0 / dy   = -2 w_0^2 d1K(y, y),  dw_i / dy = 2 w_i^2 rho_i d1K(y, x_i)
// (implicit differentiation of K(x_i, y) = 0 and of the Christoffel function),
// where "d/dmu = Phi" means dF = int Phi d(dmu_b) for the biased normalised
// measure mu_b.  For tau = m0 F with mu_b = (1-alpha) mu/m0 + alpha U:
//   dtau = int [(1-alpha) Phi + alpha int Phi dU] d(dmu)   (dmu: raw measure).
#pragma once
#include "common.cuh"
#include "trig_adjoint.cuh"

namespace mb {

constexpr int NPOLY = NMOM;   // coefficients of a degree-2n polynomial

// monomial coefficients (standardised t) of the monic orthogonal polynomials;
// row k (k+1 entries) starts at k(k+1)/2
MB_HD void pi_monomials(const Recon& R, float C[15]) {
    C[0] = 1.0f;
    C[1] = -R.al[0];
    C[2] = 1.0f;
    // pi_{k+1} = (t - al_k) pi_k - be_k pi_{k-1}
#pragma unroll
    for (int k = 1; k < 4; ++k) {
        const int o0 = (k - 1) * k / 2, o1 = k * (k + 1) / 2, o2 = (k + 1) * (k + 2) / 2;
        const float a = R.al[k], b = R.be[k - 1];
#pragma unroll
        for (int jj = 0; jj <= k + 1; ++jj) {
            float v = 0.0f;
            if (jj >= 1) v += C[o1 + jj - 1];
            if (jj <= k) v -= a * C[o1 + jj];
            if (jj <= k - 1) v -= b * C[o0 + jj];
            C[o2 + jj] = v;
        }
    }
}

// pi_k(x) and pi_k'(x), k = 0..4
MB_HD void pis_d(const Recon& R, float x, float P[5], float D[5]) {
    P[0] = 1.0f; D[0] = 0.0f;
    P[1] = x - R.al[0]; D[1] = 1.0f;
#pragma unroll
    for (int k = 1; k < 4; ++k) {
        const float xa = x - R.al[k], b = R.be[k - 1];
        P[k + 1] = fmaf(xa, P[k], -b * P[k - 1]);
        D[k + 1] = fmaf(xa, D[k], fmaf(-b, D[k - 1], P[k]));
    }
}

// The bound derivative Phi(t) is a sum of products K(t, x) K(t, x') of kernel
// polynomials, K(t, x) = sum_k e_k(x) pi_k(t) with e_k(x) = h_k pi_k(x)
// (h_0 = 1).  It is accumulated per pixel as Phi = sum_{k<=l} B_kl pi_k pi_l,
// 15 coefficients; B_kl sits at bidx(k, l).
constexpr int NB = 15;
MB_HD constexpr int bidx(int k, int l) { return k * 5 - k * (k - 1) / 2 + (l - k); }

MB_HD void kernel_coeffs(const Recon& R, const float P[5], float e[5]) {
    e[0] = P[0];
#pragma unroll
    for (int k = 1; k < 5; ++k) e[k] = R.h[k - 1] * P[k];
}

// B += s sym(u v^T), i.e. Phi += s K_u K_v for K_u = sum_k u_k pi_k
MB_HD void sym_update(float B[NB], float s, const float u[5], const float v[5]) {
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const float su = s * u[k], sv = s * v[k];
        B[bidx(k, k)] = fmaf(su, v[k], B[bidx(k, k)]);
#pragma unroll
        for (int l = k + 1; l < 5; ++l) B[bidx(k, l)] = fmaf(su, v[l], fmaf(sv, u[l], B[bidx(k, l)]));
    }
}

// B += s u u^T, i.e. Phi += s K_u^2
MB_HD void sym_update_sq(float B[NB], float s, const float u[5]) {
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const float su = s * u[k];
        B[bidx(k, k)] = fmaf(su, u[k], B[bidx(k, k)]);
        const float su2 = 2.0f * su;
#pragma unroll
        for (int l = k + 1; l < 5; ++l) B[bidx(k, l)] = fmaf(su2, u[l], B[bidx(k, l)]);
    }
}

// sum_k a_k b_k: with a = pi(t) and b = e(x) = (h_k pi_k(x)) it is K(t, x)
MB_HD float dot5(const float a[5], const float b[5]) {
    return fmaf(a[4], b[4], fmaf(a[3], b[3], fmaf(a[2], b[2], fmaf(a[1], b[1], a[0] * b[0]))));
}

// Adjoint of one bound query.  Adds gq * m0 * dF/dy (standardised y) to *gy
// and gq * Phi_F to B.  Both (1 - alpha) Phi and int Phi dU are linear in Phi,
// so the bias is applied once per pixel to the summed polynomial
// (finish_moment_adjoint).
MB_HD void query_adjoint(const Params& p, const Recon& R, const QueryRec& q, float gq, float* gy, float B[NB]) {
    if (R.m0 <= 0.0f || gq == 0.0f) return;
    float Py[5], Dy[5], ey[5];
    pis_d(R, q.y, Py, Dy);
    kernel_coeffs(R, Py, ey);                   // K(t, y) = sum_k ey_k pi_k(t)
    const float Kyy = dot5(Py, ey);
    const float w0 = fdiv_(1.0f, Kyy);          // Kyy >= 1
    const float K1yy = dot5(Dy, ey);
    const float dw0 = -2.0f * w0 * w0 * K1yy;
    const bool left = q.j <= 2;
    const float sgn = left ? 1.0f : -1.0f;      // sign of the root weights in F
    const float c0 = left ? p.beta : -(1.0f - p.beta);
    float dF = c0 * dw0;
    sym_update_sq(B, gq * c0 * w0 * w0, ey);
    if (!left) B[0] += gq;      // the constant 1 of F = 1 - ...
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        if (r >= q.nroot) break;
        const float x = q.x[r];
        float Px[5], Dx[5], ex[5];
        pis_d(R, x, Px, Dx);
        kernel_coeffs(R, Px, ex);
        const float w = fdiv_(1.0f, dot5(Px, ex));
        if (!isfinite(w) || w == 0.0f) continue;
        const float K1xx = dot5(Dx, ex);
        const float K1xy = dot5(Dx, ey);
        const float K1yx = dot5(Dy, ex);
        const float rho = K1xy != 0.0f ? fdiv_(K1xx, K1xy) : 0.0f;
        dF = fmaf(sgn, 2.0f * w * w * rho * K1yx, dF);
        // Phi += s (K_x^2 - 2 rho K_x K_y) = s sym(e_x (e_x - 2 rho e_y)^T)
        float v[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) v[k] = fmaf(-2.0f * rho, ey[k], ex[k]);
        sym_update(B, gq * sgn * w * w, ex, v);
    }
    *gy = fmaf(gq * R.m0, dF, *gy);
}

// Phi = sum_{k<=l} B_kl pi_k pi_l in standardised monomials (once per pixel).
MB_HD void phi_monomials(const Recon& R, const float B[NB], float phi[NPOLY]) {
    float C[15];
    pi_monomials(R, C);
#pragma unroll
    for (int k = 0; k < NPOLY; ++k) phi[k] = 0.0f;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        float q[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};   // q_k = sum_{l>=k} B_kl pi_l
#pragma unroll
        for (int l = k; l < 5; ++l)
#pragma unroll
            for (int jj = 0; jj <= l; ++jj) q[jj] = fmaf(B[bidx(k, l)], C[l * (l + 1) / 2 + jj], q[jj]);
#pragma unroll
        for (int i = 0; i <= k; ++i)
#pragma unroll
            for (int jj = 0; jj < 5; ++jj) phi[i + jj] = fmaf(C[k * (k + 1) / 2 + i], q[jj], phi[i + jj]);
    }
}

// Moment adjoint of the pixel from the summed bound derivative Phi:
// psi = (1 - alpha) Phi + (alpha int Phi dU + dL/dm0 through the rescaling) e_0,
// int Phi dU by the 5-point Gauss-Legendre rule (exact for degree 2n = 8).
MB_HD void finish_moment_adjoint(const Params& p, const Recon& R, float gm0, float psi[NPOLY]) {
    float lam0 = 0.0f;
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        const float t = (p.gl_y[m] - R.c) * R.inv_s;
        float v = psi[NPOLY - 1];
#pragma unroll
        for (int k = NPOLY - 2; k >= 0; --k) v = fmaf(v, t, psi[k]);
        lam0 = fmaf(p.gl_w[m], v, lam0);
    }
#pragma unroll
    for (int k = 0; k < NPOLY; ++k) psi[k] *= 1.0f - p.bias_alpha;
    psi[0] += p.bias_alpha * lam0 + gm0;
}

struct PairOut {
    float O;                  // O_i
    float g_mu, g_Sig, g_what; // dL/d(mu, Sigma, w-hat) of this pair (direct part)
};

// Recomputes the pair's quadrature (Eq. 7, App. B, App. D) and back-propagates
// L_i = a O_i + gP P_i: accumulates the bound derivative Phi of the pixel into
// B and returns the direct derivatives with respect to (mu, Sigma, w-hat).
// With SAVED the bound queries come from the quadrature pass (qin, N+1 float4)
// instead of being solved again.
// The query record and the per-pixel adjoint size of a bound representation:
// power moments (Phi coefficients B) or trigonometric moments (m0 and the
// Verblunsky-coefficient adjoints).
template <class RecT>
struct BoundAdj;
template <>
struct BoundAdj<Recon> {
    typedef QueryRec Query;
    static constexpr int NACC = NB;
};
template <>
struct BoundAdj<TrigRecon> {
    typedef TrigQueryRec Query;
    static constexpr int NACC = NTRIG_ADJ;
};

// One sample t_j of a pair with its bound query and running adjoints.
template <class QR>
struct Sample {
    float t, tau, dg, b, erf, gau;   // sample, optical depth, warp slope, b = (t - mu)/(sqrt2 Sigma), erf(b), e^{-b^2}
    bool clamped;               // t_j clamped to [t_n, t_f] (no derivative to mu, Sigma)
    QR q;
    float gt, gtau;             // dL/dt_j, dL/dtau_j
};

// Optical depth of a sample at warped depth gj with its query record: read
// from the kept query (SAVED, power moments only; QB = 8: the compact form,
// its roots restored by two Laguerre steps) or solved again.
template <bool SAVED, int QB>
MB_HD float sample_query(const Params& p, const Recon& R, float gj, float4 qv, QueryRec& q) {
    if (SAVED) {
        const float y = (fmaf(2.0f, gj, -1.0f) - R.c) * R.inv_s;
        if (QB == 8) return unpack_query_compact(R, make_float2(qv.x, qv.y), y, q);
        return unpack_query(qv, y, q);
    }
    return bound_query<true>(R, p.beta, fmaf(2.0f, gj, -1.0f), &q);
}
template <bool SAVED, int QB>
MB_HD float sample_query(const Params& p, const TrigRecon& T, float gj, float4 qv, TrigQueryRec& q) {
    if (SAVED) return unpack_trig_query(p, qv, gj, q);
    return trig_bound_query<true>(p, T, gj, &q);
}

// Kept query j of a pair (QB bytes each) as a float4 ({tau, bits} in x, y
// for the compact form).
template <int QB>
MB_HD float4 load_kept_query(const char* __restrict__ q, int j) {
    if (QB == 8) {
        const float2 v = reinterpret_cast<const float2*>(q)[j];
        return make_float4(v.x, v.y, 0.0f, 0.0f);
    }
    return reinterpret_cast<const float4*>(q)[j];
}

// Adjoint of a sample's bound query for dL/dtau = gq: adds to the pixel's
// accumulators and returns dL/d(warped depth).
MB_HD float sample_query_adjoint(const Params& p, const Recon& R, const QueryRec& q, float gq, float B[NB]) {
    float gy = 0.0f;
    query_adjoint(p, R, q, gq, &gy, B);
    return gy * 2.0f * R.inv_s;   // y' = (2 g-hat - 1 - c) / s
}
MB_HD float sample_query_adjoint(const Params& p, const TrigRecon& T, const TrigQueryRec& q, float gq,
                                 float A[NTRIG_ADJ]) {
    float ge = 0.0f;
    trig_query_adjoint(p, T, q, gq, &ge, A);
    return ge;
}

template <bool SAVED, int QB, class RecT, class QR>
MB_HD void load_sample(const Params& p, const RecT& R, const Gauss1D& g, float isq, int j, float4 qv, Sample<QR>& s) {
    const float raw = fmaf(p.kappa * g.Sig, p.x_nodes[j], g.mu);
    s.t = fminf(fmaxf(raw, p.t_near), p.t_far);
    s.clamped = s.t != raw;
    float gj;
    warp_g(p, s.t, gj, s.dg);
    s.tau = sample_query<SAVED, QB>(p, R, gj, qv, s.q);
    s.b = (s.t - g.mu) * isq;
    s.erf = p.x_erf[j];
    s.gau = p.x_gau[j];
    if (s.clamped) {
        s.erf = erff(s.b);
        s.gau = expf(-s.b * s.b);
    }
    s.gt = 0.0f;
    s.gtau = 0.0f;
}

// Recomputes the pair's quadrature (Eq. 7, App. B, App. D) and back-propagates
// L_i = a O_i + gP P_i: accumulates the bound derivative Phi of the pixel into
// B and returns the direct derivatives with respect to (mu, Sigma, w-hat).
// With SAVED the bound queries come from the quadrature pass (qin, N+1 of QB
// bytes) instead of being solved again.  Streamed over the samples: interval j is
// processed once samples j and j+1 are loaded, after which sample j's
// adjoints are final and go through its bound query (one copy of the query
// code, no per-sample arrays).  Saved queries are read one sample ahead of
// their use, so each load overlaps a whole interval's arithmetic.
template <int NI, bool SAVED = false, class RecT = Recon, int QB = 16>
MB_HD PairOut pair_backward(const Params& p, const RecT& R, const Gauss1D& g, float a, float gP, float B[],
                            const char* __restrict__ qin = nullptr) {
    const int N = NI > 0 ? NI : p.n_intervals;
    PairOut o;
    o.O = 0.0f;
    o.g_mu = 0.0f;
    o.g_Sig = 0.0f;
    o.g_what = 0.0f;
    const float iSig = 1.0f / g.Sig;
    const float iSig2 = iSig * iSig;
    const float isq = 0.70710678118654752f * iSig;
    const float escale = g.Sig * 1.25331413731550025f;             // d tau_ij / d w-hat per erf difference
    const float tscale = g.what * escale;
    const float dscale = g.what * g.Sig * 1.41421356237309505f;   // d tau_ij / d b = dscale e^{-b^2}
    Sample<typename BoundAdj<RecT>::Query> c, n;
    // T_j = e^{-tau_j}, carried: T_{j+1} = T_j e^{-dtau_j} (e^{-dtau} = 1 - dtau ph)
    float Tc = 0.0f, Tn = 0.0f;
    // interval j between samples c = j and n = j + 1: term = T_j ph(dtau)
    // sig_j Delta_j and the penalty v^2
    auto interval = [&]() {
        const float Delta = n.t - c.t;
        const float dtr = n.tau - c.tau;
        const bool pos = dtr > 0.0f;
        const float dtau = pos ? dtr : 0.0f;
        const float Tj = Tc;
        const float d0 = c.t - g.mu;
        const float e0 = c.gau;
        const float sig = g.what * e0;
        // ph(x) = (1 - e^-x)/x and ph'(x) = (e^-x - ph(x))/x: Taylor series
        // below x = 0.05 (truncation < 5e-10), where e^-x - ph cancels
        float ph, dph;
        if (dtau < 0.05f) {
            ph = fmaf(dtau, fmaf(dtau, fmaf(dtau, fmaf(dtau, 1.0f / 120.0f, -1.0f / 24.0f), 1.0f / 6.0f), -0.5f),
                      1.0f);
            dph = fmaf(dtau, fmaf(dtau, fmaf(dtau, fmaf(dtau, -1.0f / 144.0f, 1.0f / 30.0f), -0.125f), 1.0f / 3.0f),
                       -0.5f);
        } else {
            // dtau >= 0.05: 1 - e^-x keeps its digits with the fast exponential
            const float em = exp_(-dtau);
            const float idt = fdiv_(1.0f, dtau);
            ph = (1.0f - em) * idt;
            dph = (em - ph) * idt;
        }
        Tn = Tj * fmaf(-dtau, ph, 1.0f);
        const float term = Tj * ph * sig * Delta;
        o.O += term;
        const float tij = tscale * (n.erf - c.erf);
        const float v = fmaxf(tij - dtau, 0.0f);
        c.gtau -= a * term;
        const float gdt = a * Tj * dph * sig * Delta - 2.0f * gP * v;
        if (pos) {
            n.gtau += gdt;
            c.gtau -= gdt;
        }
        const float gsig = a * Tj * ph * Delta;
        const float gD = a * Tj * ph * sig;
        n.gt += gD;
        c.gt -= gD;
        const float sd = gsig * sig * d0 * iSig2;
        c.gt -= sd;
        o.g_mu += sd;
        o.g_Sig += sd * d0 * iSig;
        o.g_what += gsig * e0;
        const float gtij = 2.0f * gP * v;
        if (gtij != 0.0f) {
            o.g_what += gtij * escale * (n.erf - c.erf);
            o.g_Sig += gtij * tij * iSig;
            const float c1 = gtij * dscale * n.gau;
            const float c0 = -gtij * dscale * c.gau;
            n.gt += c1 * isq;
            c.gt += c0 * isq;
            o.g_mu -= (c1 + c0) * isq;
            o.g_Sig -= (c1 * n.b + c0 * c.b) * iSig;
        }
    };
    // sample j (c) is final: through its bound query to y_j and the moments
    auto sample_final = [&](int j) {
        c.gt = fmaf(sample_query_adjoint(p, R, c.q, c.gtau, B), c.dg, c.gt);
        if (!c.clamped) {
            o.g_mu += c.gt;
            o.g_Sig = fmaf(c.gt, p.kappa * p.x_nodes[j], o.g_Sig);
        }
    };
    if (SAVED) {
        // kept queries: read one sample ahead of their use
        float4 qa = load_kept_query<QB>(qin, 0), qb = load_kept_query<QB>(qin, 1);
        load_sample<SAVED, QB>(p, R, g, isq, 0, qa, c);
        Tc = exp_(-c.tau);
        Tn = Tc;
#pragma unroll 1
        for (int j = 0; j <= N; ++j) {
            if (j < N) {
                load_sample<SAVED, QB>(p, R, g, isq, j + 1, qb, n);
                if (j + 2 <= N) qb = load_kept_query<QB>(qin, j + 2);
                interval();
            }
            sample_final(j);
            c = n;
            Tc = Tn;
        }
    } else {
        // queries solved here: iteration i loads sample i (i <= N), then
        // handles interval i - 1 and sample i - 1 (i >= 1), so that the large
        // solver code has one copy
        const float4 none = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll 1
        for (int i = 0; i <= N + 1; ++i) {
            if (i <= N) {
                load_sample<SAVED, QB>(p, R, g, isq, i, none, n);
                if (i == 0) {
                    Tc = exp_(-n.tau);
                    Tn = Tc;
                    c = n;
                    continue;
                }
                interval();
            }
            sample_final(i - 1);
            c = n;
            Tc = Tn;
        }
    }
    return o;
}

// int Psi d(d mu_i): reverse sweep of the moment recurrence (Eq. 10-12, App. C)
// written for the standardised linearised warp t = A + S (t_ray - mu).
MB_HD void moment_adjoint(const Params& p, const Recon& R, const Gauss1D& g, const float psi[NPOLY], float* g_mu,
                          float* g_Sig, float* g_what) {
    // linearisation point c = max(mu, t_n): a = g(c) + g'(c)(mu - c), s = g'(c);
    // da/dmu = s in both cases, ds/dmu = g''(mu) only when c = mu
    const float cpt = fmaxf(g.mu, p.t_near);
    float gm, dgm, ddgm;
    warp_g(p, cpt, gm, dgm);
    gm = fmaf(dgm, g.mu - cpt, gm);
    if (g.mu > p.t_near) {
        const float z = fmaf(p.two_over_a, cpt, 1.0f);
        ddgm = p.G3 * fdiv_(dgm, p.G2 * z);   // g'' = G3 z^(lambda-2)
    } else {
        ddgm = 0.0f;
    }
    const float A = (fmaf(2.0f, gm, -1.0f) - R.c) * R.inv_s;
    const float S = 2.0f * dgm * R.inv_s;
    const float dS = 2.0f * ddgm * R.inv_s;
    const float dn = p.t_near - g.mu;
    const float iSg = 1.0f / g.Sig;
    const float bn = dn * (0.70710678118654752f * iSg);
    const float en = expf(-bn * bn);
    const float un = fmaf(S, dn, A);
    const float w = g.what, Sg = g.Sig, S2 = g.Sig2;
    float M[NPOLY], up[NPOLY];
    up[0] = 1.0f;
#pragma unroll
    for (int k = 1; k < NPOLY; ++k) up[k] = up[k - 1] * un;
    M[0] = w * Sg * 1.25331413731550025f * erfcf(bn);
    M[1] = fmaf(A, M[0], S * w * S2 * en);
#pragma unroll
    for (int k = 2; k < NPOLY; ++k)
        M[k] = fmaf(A, M[k - 1], fmaf(S * S * S2 * (float)(k - 1), M[k - 2], S * w * S2 * up[k - 1] * en));
    float Mb[NPOLY];
#pragma unroll
    for (int k = 0; k < NPOLY; ++k) Mb[k] = psi[k];
    float Ab = 0.0f, Sb = 0.0f, Sgb = 0.0f, wb = 0.0f, unb = 0.0f, enb = 0.0f, bnb = 0.0f, mub = 0.0f;
#pragma unroll
    for (int k = NPOLY - 1; k >= 2; --k) {
        const float c = Mb[k];
        const float km1 = (float)(k - 1);
        Mb[k - 1] = fmaf(A, c, Mb[k - 1]);
        Mb[k - 2] = fmaf(S * S * S2 * km1, c, Mb[k - 2]);
        Ab = fmaf(M[k - 1], c, Ab);
        const float bt = w * S2 * up[k - 1] * en;    // boundary term / S
        Sb = fmaf(2.0f * S * S2 * km1 * M[k - 2] + bt, c, Sb);
        Sgb = fmaf(2.0f * S * S * Sg * km1 * M[k - 2] + 2.0f * S * w * Sg * up[k - 1] * en, c, Sgb);
        wb = fmaf(S * S2 * up[k - 1] * en, c, wb);
        unb = fmaf(S * w * S2 * km1 * up[k - 2] * en, c, unb);
        enb = fmaf(S * w * S2 * up[k - 1], c, enb);
    }
    {
        const float c = Mb[1];
        Ab = fmaf(M[0], c, Ab);
        Mb[0] = fmaf(A, c, Mb[0]);
        Sb = fmaf(w * S2 * en, c, Sb);
        wb = fmaf(S * S2 * en, c, wb);
        Sgb = fmaf(2.0f * S * w * Sg * en, c, Sgb);
        enb = fmaf(S * w * S2, c, enb);
    }
    {
        const float c = Mb[0];
        wb = fmaf(Sg * 1.25331413731550025f * erfcf(bn), c, wb);
        Sgb = fmaf(M[0] * iSg, c, Sgb);
        bnb = fmaf(-w * Sg * 1.41421356237309505f * en, c, bnb);
    }
    bnb = fmaf(-2.0f * bn * en, enb, bnb);
    Ab += unb;
    Sb = fmaf(dn, unb, Sb);
    mub = fmaf(-S, unb, mub);
    mub = fmaf(-(0.70710678118654752f * iSg), bnb, mub);
    Sgb = fmaf(-bn * iSg, bnb, Sgb);
    mub = fmaf(S, Ab, mub);
    mub = fmaf(dS, Sb, mub);
    *g_mu += mub;
    *g_Sig += Sgb;
    *g_what += wb;
}

// record-coefficient gradient layout (floats)
enum GradField { G_C0 = 0, G_CX = 3, G_CY = 6, G_GA = 9, G_MX = 12, G_MY = 15, G_O = 18, G_LNW = 21, G_RGB = 22, NGRAD = 25 };

// (mu, Sigma, w-hat) of a pair -> record coefficients (inverse of pair_gaussian)
MB_HD void geometry_adjoint(const float* __restrict__ r, float dx, float dy, float rlen, float r2, const Gauss1D& g,
                            float g_mu, float g_Sig, float g_what, float out[NGRAD]) {
    const float vx = fmaf(dy, r[R_CY + 0], fmaf(dx, r[R_CX + 0], r[R_C0 + 0]));
    const float vy = fmaf(dy, r[R_CY + 1], fmaf(dx, r[R_CX + 1], r[R_C0 + 1]));
    const float vz = fmaf(dy, r[R_CY + 2], fmaf(dx, r[R_CX + 2], r[R_C0 + 2]));
    const float cross2 = fmaf(vx, vx, fmaf(vy, vy, vz * vz));
    const float gx = fmaf(dy, r[R_MY + 0], fmaf(dx, r[R_MX + 0], r[R_GA + 0]));
    const float gy = fmaf(dy, r[R_MY + 1], fmaf(dx, r[R_MX + 1], r[R_GA + 1]));
    const float gz = fmaf(dy, r[R_MY + 2], fmaf(dx, r[R_MX + 2], r[R_GA + 2]));
    const float dd = fmaf(gx, gx, fmaf(gy, gy, gz * gz));
    const float inv = 1.0f / dd;
    const float g_dd = inv * (-0.5f * g.Sig * g_Sig - g.mu * g_mu + 0.5f * g.what * cross2 * inv * g_what);
    const float g_od = -rlen * inv * g_mu;
    const float g_c2 = -0.5f * g.what * inv * g_what;
    const float dg[3] = {gx, gy, gz};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float gd = 2.0f * dg[k] * g_dd;
        out[G_GA + k] += gd;
        out[G_MX + k] += gd * dx;
        out[G_MY + k] += gd * dy;
    }
    out[G_O + 0] += g_od;
    out[G_O + 1] += g_od * dx;
    out[G_O + 2] += g_od * dy;
    const float v[3] = {vx, vy, vz};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float gv = 2.0f * v[k] * g_c2;
        out[G_C0 + k] += gv;
        out[G_CX + k] += gv * dx;
        out[G_CY + k] += gv * dy;
    }
    out[G_LNW] += g.what * g_what;
}

// Compact form of the geometry adjoint.  With g = g_a + dx m_x + dy m_y and
// v = c0 + dx cx + dy cy, the 22 record-coefficient derivatives of a pair are
// 2 g_k g_dd {1, dx, dy}, 2 v_k g_c2 {1, dx, dy}, g_od {1, dx, dy} and
// w-hat g_what; summed over a record's pixels they only need the 16 pixel
// moments g_dd {1, dx, dy, dx^2, dx dy, dy^2}, g_c2 {same}, g_od {1, dx, dy}
// and w-hat g_what, expanded once per record with its vectors
// (expand_geometry).  Pass 1 adds the 3 colour fields.
enum CompactField { K_DD = 0, K_C2 = 6, K_OD = 12, K_LNW = 15, K_RGB = 16, NK_MOM = 16, NK_QUAD = 19 };

MB_HD void geometry_adjoint_compact(const float* __restrict__ r, float dx, float dy, float rlen, const Gauss1D& g,
                                    float g_mu, float g_Sig, float g_what, float out[]) {
    const float vx = fmaf(dy, r[R_CY + 0], fmaf(dx, r[R_CX + 0], r[R_C0 + 0]));
    const float vy = fmaf(dy, r[R_CY + 1], fmaf(dx, r[R_CX + 1], r[R_C0 + 1]));
    const float vz = fmaf(dy, r[R_CY + 2], fmaf(dx, r[R_CX + 2], r[R_C0 + 2]));
    const float cross2 = fmaf(vx, vx, fmaf(vy, vy, vz * vz));
    const float gx = fmaf(dy, r[R_MY + 0], fmaf(dx, r[R_MX + 0], r[R_GA + 0]));
    const float gy = fmaf(dy, r[R_MY + 1], fmaf(dx, r[R_MX + 1], r[R_GA + 1]));
    const float gz = fmaf(dy, r[R_MY + 2], fmaf(dx, r[R_MX + 2], r[R_GA + 2]));
    const float dd = fmaf(gx, gx, fmaf(gy, gy, gz * gz));
    const float inv = 1.0f / dd;
    const float g_dd = inv * (-0.5f * g.Sig * g_Sig - g.mu * g_mu + 0.5f * g.what * cross2 * inv * g_what);
    const float g_od = -rlen * inv * g_mu;
    const float g_c2 = -0.5f * g.what * inv * g_what;
    const float m[6] = {1.0f, dx, dy, dx * dx, dx * dy, dy * dy};
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        out[K_DD + i] = fmaf(g_dd, m[i], out[K_DD + i]);
        out[K_C2 + i] = fmaf(g_c2, m[i], out[K_C2 + i]);
    }
    out[K_OD + 0] += g_od;
    out[K_OD + 1] = fmaf(g_od, dx, out[K_OD + 1]);
    out[K_OD + 2] = fmaf(g_od, dy, out[K_OD + 2]);
    out[K_LNW] = fmaf(g.what, g_what, out[K_LNW]);
}

// Record-coefficient derivative f (GradField) from the compact sums s of one record.
MB_HD float expand_geometry(const float* __restrict__ r, const float* __restrict__ s, int f) {
    if (f >= G_RGB) return s[K_RGB + f - G_RGB];
    if (f >= G_LNW) return s[K_LNW];
    if (f >= G_O) return s[K_OD + f - G_O];
    // f in [G_C0, G_O): block b (0: c0/g_a, 1: cx/m_x, 2: cy/m_y), component k
    const bool geo = f >= G_GA;
    const int b = ((f - (geo ? G_GA : G_C0)) / 3), k = (f - (geo ? G_GA : G_C0)) % 3;
    const float* S = s + (geo ? K_DD : K_C2);
    const float a0 = r[(geo ? R_GA : R_C0) + k], a1 = r[(geo ? R_MX : R_CX) + k], a2 = r[(geo ? R_MY : R_CY) + k];
    // moments for {1, dx, dy} x {1, dx, dy}: row b of [[S0,S1,S2],[S1,S3,S4],[S2,S4,S5]]
    const float s0 = b == 0 ? S[0] : (b == 1 ? S[1] : S[2]);
    const float s1 = b == 0 ? S[1] : (b == 1 ? S[3] : S[4]);
    const float s2 = b == 0 ? S[2] : (b == 1 ? S[4] : S[5]);
    return 2.0f * fmaf(a0, s0, fmaf(a1, s1, a2 * s2));
}

#ifdef __CUDACC__
// Warp reduce-scatter of M <= 32 per-lane values.  Each of 5 butterfly levels
// halves the slots a lane holds (n -> ceil(n/2); the upper lane of a pair
// keeps the upper part), so M = 19 takes 10 + 5 + 3 + 2 + 1 = 21 shuffles.
// Lane L returns the warp sum of v[rs_index<M>(L)] (0 where that is -1).  All
// 32 lanes must call it.
template <int N, int O>
struct ReduceScatterLevel {
    static __device__ __forceinline__ void run(float* v, int lane) {
        constexpr int H = (N + 1) / 2;
        const bool up = (lane & O) != 0;
#pragma unroll
        for (int i = 0; i < H; ++i) {
            const float hv = (H + i < N) ? v[H + i] : 0.0f;
            const float send = up ? v[i] : hv;
            const float keep = up ? hv : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, O);
        }
        ReduceScatterLevel<H, O / 2>::run(v, lane);
    }
};
template <int N>
struct ReduceScatterLevel<N, 0> {
    static __device__ __forceinline__ void run(float*, int) {}
};

template <int M>
__device__ __forceinline__ float reduce_scatter(float v[M]) {
    ReduceScatterLevel<M, 16>::run(v, threadIdx.x & 31);
    return v[0];
}

// The value index a lane returns from reduce_scatter<M>, or -1.
template <int M>
MB_HD int rs_index(int lane) {
    int n = M, base = 0, cnt = M;
    for (int o = 16; o >= 1; o >>= 1) {
        const int h = (n + 1) / 2;
        if (lane & o) {
            base += h;
            cnt -= h;
        } else {
            cnt = cnt < h ? cnt : h;
        }
        n = h;
    }
    return cnt >= 1 ? base : -1;
}

// Warp reduction of 16 per-lane values: lanes f and f + 16 return the warp
// sum of v[f] (16 shuffles).  All 32 lanes must call it.
__device__ __forceinline__ float reduce_scatter16(float v[16]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 8; o >= 1; o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < o; ++i) {
            const float send = up ? v[i] : v[i + o];
            const float keep = up ? v[i + o] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 16);
}
#endif

// Per-pixel backward context from the forward outputs (Eq. 15 adjoint).
struct PixelAdj {
    float gS[3];   // dL/d(sum L_i)
    float gO;      // dL/dO
    float gm0;     // dL/dm0 through the rescaling
    float gP;      // dL/dP
};

MB_HD PixelAdj pixel_adjoint(const Params& p, float m0, const float S[3], float O, const float g[3], float gP) {
    PixelAdj a;
    const float Tf = expf(-m0);
    const float op = -expm1f(-m0);
    const float den = fmaxf(p.eps, O);
    const float r = op / den;
    const float gs = g[0] * S[0] + g[1] * S[1] + g[2] * S[2];
    for (int c = 0; c < 3; ++c) a.gS[c] = r * g[c];
    a.gO = O > p.eps ? -op * gs / (O * O) : 0.0f;
    a.gm0 = Tf * gs / den - Tf * (g[0] * p.bg[0] + g[1] * p.bg[1] + g[2] * p.bg[2]);
    a.gP = gP;
    return a;
}

}  // namespace mb
