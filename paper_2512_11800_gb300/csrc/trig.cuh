// Trigonometric (Fourier) moments of the moment-based rasterizer (Sec. 3.2,
// Eq. 13-14; App. C "Trigonometric Moments") and their transmittance bounds.
// Included by common.cuh after the power-moment reconstruction.
//
// Warped depth g-hat in [0, 1] maps to the angle phi = A g-hat on the unit
// circle, A = 2 pi - theta, leaving an empty wrapping zone of angle theta.
// Per pixel: m0 and the complex moments m_k = sum_i int e^{i k phi(t)}
// sigma_i(t) dt, k = 1..4 (9 floats, the storage of the power moments).
//
// Bounds.  The canonical representation of the (normalised, biased) moments
// through the query z_w = e^{i psi_w} is the Gauss-Szego rule through z_w: its
// nodes are the zeros of the para-orthogonal polynomial z Phi_4(z) - t Phi_4^*(z)
// (|t| = 1) built from the monic Szego polynomials Phi_k, and its weights are
// the Christoffel function 1/K_4(z, z).  The nodes are where the phase
//   Theta(psi) = 5 psi - 2 arg Phi_4^*(e^{i psi})
// takes the values Theta(psi_w) + 2 pi k: Theta is continuous and strictly
// increasing (by 10 pi per turn), so each node is a monotone 1D root, and
// Theta'(psi) = K_4(z, z) / |phi_4(z)|^2 (phi_4 = Phi_4 / |Phi_4|) gives both
// the Newton step and the weight.  arg Phi^* is continuous because it is a
// sum of args of factors 1 - alpha_k z Phi_k / Phi_k^* with positive real part
// (|alpha_k| < 1, |z Phi_k / Phi_k^*| = 1 on the circle); two factors at a
// time keep each atan2 on its principal branch.  The lower bound L sums the
// weights of the nodes between the cut psi_lo = -theta/2 (middle of the
// wrapping zone) and psi_w; U = L + the weight of z_w; tau = m0 ((1 - beta) L
// + beta U), as for the power moments (Eq. 8).
#pragma once

namespace mb {

constexpr float TWO_PI_F = 6.28318530717958648f;

// Per-pixel state of the trigonometric bounds (kept in the RECON floats).
struct TrigRecon {
    float m0;
    float ar[4], ai[4];   // Verblunsky (reflection) coefficients alpha_0..alpha_3
    float rho2[4];        // 1 - |alpha_k|^2, formed in FP64 (it cancels for nearly atomic measures)
    float th_lo;          // Theta at the cut psi_lo
};

// Moments of one Gaussian (Eq. 14): m_k = w-hat sqrt(pi/2) Sigma
// e^{i k A a - (k A s Sigma)^2 / 2} (1 - erf(v_n)), with the warp linearised as
// a + s (t - mu) at c = max(mu, t_n) and 1 - erf(v_n) to first order in the
// imaginary part of v_n = b_n - i k A s Sigma / sqrt2 (App. C):
// erfc(b_n) + i k A s Sigma sqrt(2/pi) e^{-b_n^2}.  acc = {m0, Re m1, Im m1, ..}.
MB_HD void trig_moments(const Params& p, const Gauss1D& g, float acc[NMOM]) {
    const float cpt = fmaxf(g.mu, p.t_near);
    float a, s;
    warp_g(p, cpt, a, s);
    a = fmaf(s, g.mu - cpt, a);
    const float bn = (p.t_near - g.mu) * (0.70710678118654752f / g.Sig);
    const float ec = erfcf(bn);
    const float en = expf(-bn * bn);
    const float base = g.what * g.Sig * 1.25331413731550025f;
    acc[0] = fmaf(base, ec, acc[0]);
    const float q = g.Sig * s * p.trig_A;                    // k A s Sigma / k
    const float d1 = expf(-0.5f * q * q);                    // damping of k = 1; k-th: d1^(k^2)
    const float d2 = d1 * d1, d4 = d2 * d2, d8 = d4 * d4;
    const float damp[4] = {d1, d4, d8 * d1, d8 * d8};
    const float im1 = q * 0.79788456080286536f * en;         // imaginary part of 1 - erf for k = 1
    float sn, cs;
    sincosf(p.trig_A * a, &sn, &cs);
    float zr = cs, zi = sn;                                  // e^{i k A a}
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float ei = (float)(k + 1) * im1;
        const float sc = base * damp[k];
        acc[2 * k + 1] = fmaf(sc, zr * ec - zi * ei, acc[2 * k + 1]);
        acc[2 * k + 2] = fmaf(sc, zr * ei + zi * ec, acc[2 * k + 2]);
        const float nr = zr * cs - zi * sn;
        zi = fmaf(zr, sn, zi * cs);
        zr = nr;
    }
}

struct TrigEval {
    float th;    // Theta(psi)
    float dth;   // Theta'(psi)
    float lam;   // Christoffel weight 1 / K_4(z, z)
};

// Theta, Theta' and the Christoffel weight at z = e^{i psi} from the Szego
// recursion Phi_{k+1} = z Phi_k - conj(alpha_k) Phi_k^*,
// Phi_{k+1}^* = Phi_k^* - alpha_k z Phi_k, |Phi_k|^2 norms E_{k+1} = E_k (1 - |alpha_k|^2).
MB_HD TrigEval trig_eval(const TrigRecon& T, float psi) {
    float sn, cs;
    sincosf(psi, &sn, &cs);
    float pr = 1.0f, pi = 0.0f, sr = 1.0f, si = 0.0f, E = 1.0f, K = 1.0f;
    float s2r = 1.0f, s2i = 0.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float zr = cs * pr - sn * pi, zi = fmaf(cs, pi, sn * pr);
        const float ar = T.ar[k], ai = T.ai[k];
        const float npr = zr - fmaf(ar, sr, ai * si), npi = zi - fmaf(ar, si, -ai * sr);
        const float nsr = sr - fmaf(ar, zr, -ai * zi), nsi = si - fmaf(ar, zi, ai * zr);
        E *= T.rho2[k];
        pr = npr; pi = npi; sr = nsr; si = nsi;
        K += fdiv_(fmaf(pr, pr, pi * pi), E);
        if (k == 1) { s2r = sr; s2i = si; }
    }
    const float t1 = atan2f(s2i, s2r);
    const float t2 = atan2f(fmaf(si, s2r, -sr * s2i), fmaf(sr, s2r, si * s2i));
    TrigEval r;
    r.th = fmaf(5.0f, psi, -2.0f * (t1 + t2));
    const float pn2 = fdiv_(fmaf(pr, pr, pi * pi), E);
    r.dth = fdiv_(K, pn2);
    r.lam = fdiv_(1.0f, K);
    return r;
}

// The node psi in (a, b) with Theta(psi) = target, given Theta(a) = ta and
// Theta(b) = tb (ta < target < tb).  Newton on Theta, kept inside the
// bracket and replaced by bisection whenever it would leave the bracket or
// not halve the previous step (for nearly atomic measures Theta is close to
// a staircase, where plain Newton can cycle).  It stops once the node is
// within 2e-7 (relative) of the current point, and returns the Christoffel
// weight evaluated there.
// One evaluation site in the loop (the code is large: a single copy keeps
// the adjoint kernel's hot loop in the instruction cache).
MB_HD float trig_node_weight(const TrigRecon& T, float target, float a, float ta, float b, float tb, float* node) {
    float x = a + (b - a) * fminf(fmaxf(fdiv_(target - ta, tb - ta), 0.0f), 1.0f);
    float dx_old = b - a, dx = dx_old;
    const float h_floor = 5e-7f * (1.0f + fabsf(target));   // FP32 resolution of Theta
    TrigEval e;
    e.lam = 0.0f;
    bool last = false;   // the step just taken was below the tolerance: this evaluation is the final one
#pragma unroll 1
    for (int it = 0; it < 33; ++it) {
        e = trig_eval(T, x);
        const float h = e.th - target;
        const float tol = 2e-7f * (1.0f + fabsf(x));
        if (last || it == 32 || fabsf(h) <= fmaxf(tol * e.dth, h_floor)) break;
        if (h > 0.0f) b = x;
        else a = x;
        const float xn = x - fdiv_(h, e.dth);
        dx_old = dx;
        if (!(xn > a && xn < b) || fabsf(2.0f * h) > fabsf(dx_old * e.dth)) {
            dx = 0.5f * (b - a);
            x = a + dx;
        } else {
            dx = xn - x;
            x = xn;
        }
        last = fabsf(dx) < tol;
    }
    *node = x;
    return isfinite(e.lam) ? e.lam : 0.0f;
}

// A solved trigonometric bound query, kept for the adjoint.
struct TrigQueryRec {
    float psi;      // psi_w = A clamp(gq, 0, 1)
    int j;          // band of Theta(psi_w) above the cut, 0..4 (left side when j <= 2)
    int ns;         // nodes solved (0..2), nearest to z_w first
    float x[2];     // their angles
    bool inside;    // gq in (0, 1): psi_w moves with the warped depth
};

// tau at warped depth gq in [0, 1] (angle psi = A gq).  REC keeps the nodes.
template <bool REC>
MB_HD float trig_bound_query(const Params& p, const TrigRecon& T, float gq, TrigQueryRec* rec) {
    if (REC) { rec->psi = 0.0f; rec->j = 0; rec->ns = 0; rec->x[0] = 0.0f; rec->x[1] = 0.0f; rec->inside = false; }
    if (T.m0 <= 0.0f) return 0.0f;
    const float psi_w = p.trig_A * fminf(fmaxf(gq, 0.0f), 1.0f);
    const TrigEval w = trig_eval(T, psi_w);
    const float lo = p.trig_lo, hi = p.trig_lo + TWO_PI_F;
    const float th_lo = T.th_lo, th_hi = T.th_lo + 5.0f * TWO_PI_F;
    int j = (int)floorf((w.th - th_lo) * (1.0f / TWO_PI_F));
    j = j < 0 ? 0 : (j > 4 ? 4 : j);
    float acc = 0.0f;
    const bool left = j <= 2;
    const int ns = left ? j : 4 - j;
    if (REC) { rec->psi = psi_w; rec->j = j; rec->ns = ns; rec->inside = gq > 0.0f && gq < 1.0f; }
    // nodes nearest to z_w first: each bounds the next one's bracket
    float edge = psi_w, th_edge = w.th;
#pragma unroll 1
    for (int k = 1; k <= ns; ++k) {
        float node;
        if (left) {
            const float target = w.th - TWO_PI_F * (float)k;
            acc += trig_node_weight(T, target, lo, th_lo, edge, th_edge, &node);
            edge = node;
            th_edge = target;
        } else {
            const float target = w.th + TWO_PI_F * (float)k;
            acc += trig_node_weight(T, target, edge, th_edge, hi, th_hi, &node);
            edge = node;
            th_edge = target;
        }
        if (REC) {   // static indices keep the record in registers
            if (k == 1) rec->x[0] = node;
            else rec->x[1] = node;
        }
    }
    const float w0 = w.lam;
    float L = left ? acc : 1.0f - w0 - acc;
    L = fminf(fmaxf(L, 0.0f), fmaxf(1.0f - w0, 0.0f));
    return T.m0 * fmaf(p.beta, w0, L);
}

MB_HD float trig_optical_depth(const Params& p, const TrigRecon& T, float gq) {
    return trig_bound_query<false>(p, T, gq, nullptr);
}

// A trigonometric bound query kept for the adjoint (16 bytes):
// {tau, x_0, x_1, j | ns << 4}; psi_w and `inside` follow from the warped
// depth, which the adjoint forms with the same operations.
MB_HD float4 pack_trig_query(float tau, const TrigQueryRec& q) {
    return make_float4(tau, q.x[0], q.x[1], int_bits_as_float(q.j | (q.ns << 4)));
}
MB_HD float unpack_trig_query(const Params& p, float4 v, float gq, TrigQueryRec& q) {
    const int m = float_bits_as_int(v.w);
    q.psi = p.trig_A * fminf(fmaxf(gq, 0.0f), 1.0f);
    q.inside = gq > 0.0f && gq < 1.0f;
    q.j = m & 15;
    q.ns = m >> 4;
    q.x[0] = v.y;
    q.x[1] = v.z;
    return v.x;
}

// Levinson-Durbin recursion of one attempt, with the states the adjoint
// re-traces: the monic Szego polynomials Phi_k (coefficients P[k][0..k]),
// their norms E_k, the numerators n_k = <1, z Phi_k> and g_k = n_k / E_k =
// conj(alpha_k).
template <typename real>
struct LevTrace {
    real cr[5], ci[5];          // biased normalised moments c_0..c_4
    real Pr[4][5], Pi[4][5];    // Phi_k, k = 0..3
    real E[5];                  // E_0..E_4
    real nr[4], ni[4];          // n_k
    real gr[4], gi[4];          // g_k = conj(alpha_k)
};

// Normalise and bias the moments, c_k = (1 - alpha) m_k / m0 + alpha c*_k,
// and run Levinson-Durbin for the Verblunsky coefficients; the bias is raised
// x4 per attempt (to at most 0.5) while some |alpha_k| reaches 1 (Toeplitz
// matrix not positive definite).  Returns the bias used; tr (if given) holds
// the final attempt.
template <typename real>
MB_HD real trig_verblunsky(const Params& p, const float I[NMOM], real vr[4], real vi[4], LevTrace<real>* tr) {
    const real inv0 = real(1) / (real)I[0];
    real alpha = (real)p.bias_alpha;
    LevTrace<real> t;
#pragma unroll 1
    for (int attempt = 0; attempt < 8; ++attempt) {
        t.cr[0] = 1;
        t.ci[0] = 0;
#pragma unroll
        for (int k = 1; k <= 4; ++k) {
            t.cr[k] = (real(1) - alpha) * (real)I[2 * k - 1] * inv0 + alpha * (real)p.cstar_re[k - 1];
            t.ci[k] = (real(1) - alpha) * (real)I[2 * k] * inv0 + alpha * (real)p.cstar_im[k - 1];
        }
        real Pr[5] = {1, 0, 0, 0, 0}, Pi[5] = {0, 0, 0, 0, 0};
        real E = 1;
        bool ok = true;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
#pragma unroll
            for (int jj = 0; jj < 5; ++jj) { t.Pr[k][jj] = Pr[jj]; t.Pi[k][jj] = Pi[jj]; }
            t.E[k] = E;
            // conj(alpha_k) = <1, z Phi_k> / E_k = sum_j P_j c_{j+1} / E_k
            real nr = 0, ni = 0;
#pragma unroll
            for (int jj = 0; jj <= 3; ++jj) {
                if (jj <= k) {
                    nr += Pr[jj] * t.cr[jj + 1] - Pi[jj] * t.ci[jj + 1];
                    ni += Pr[jj] * t.ci[jj + 1] + Pi[jj] * t.cr[jj + 1];
                }
            }
            const real gr = nr / E, gi = ni / E;     // conj(alpha_k)
            t.nr[k] = nr; t.ni[k] = ni; t.gr[k] = gr; t.gi[k] = gi;
            // Phi_{k+1}[j] = Phi_k[j-1] - conj(alpha_k) conj(Phi_k[k-j])
            real Qr[5], Qi[5];
#pragma unroll
            for (int jj = 0; jj <= 4; ++jj) {
                real ur = 0, ui = 0;
                if (jj >= 1 && jj - 1 <= k) { ur = Pr[jj - 1]; ui = Pi[jj - 1]; }
                if (jj <= k) {
                    const real sr = Pr[k - jj], si = -Pi[k - jj];
                    ur -= gr * sr - gi * si;
                    ui -= gr * si + gi * sr;
                }
                Qr[jj] = ur;
                Qi[jj] = ui;
            }
#pragma unroll
            for (int jj = 0; jj <= 4; ++jj) { Pr[jj] = Qr[jj]; Pi[jj] = Qi[jj]; }
            vr[k] = gr;
            vi[k] = -gi;                               // alpha_k
            const real r2 = gr * gr + gi * gi;
            if (!(r2 < real(1) - real(1e-9))) ok = false;
            E *= real(1) - r2;
        }
        t.E[4] = E;
        if (ok || alpha >= real(0.5)) break;
        alpha = alpha * 4 < real(0.5) ? alpha * 4 : real(0.5);
    }
    if (tr) *tr = t;
    return alpha;
}

// Per-pixel reconstruction: normalise and bias the moments towards those of
// the uniform distribution on the angles [0, A] and run Levinson-Durbin for
// the Verblunsky coefficients (FP64, trig_verblunsky), then Theta at the cut
// (FP32, the same evaluation the queries use).
MB_HD void reconstruct_trig(const Params& p, const float I[NMOM], TrigRecon& T) {
    typedef MB_RECON_T real;
    T.m0 = I[0];
    T.th_lo = 0.0f;
    if (!(I[0] >= p.m_min) || !isfinite(I[0])) {
        T.m0 = 0.0f;
#pragma unroll
        for (int k = 0; k < 4; ++k) { T.ar[k] = 0.0f; T.ai[k] = 0.0f; T.rho2[k] = 1.0f; }
        return;
    }
    real vr[4] = {0, 0, 0, 0}, vi[4] = {0, 0, 0, 0};
    trig_verblunsky<real>(p, I, vr, vi, (LevTrace<real>*)nullptr);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        real r = sqrt(vr[k] * vr[k] + vi[k] * vi[k]);
        const real lim = real(1) - real(1e-6);
        const real sc = r > lim ? lim / r : real(1);
        T.ar[k] = (float)(vr[k] * sc);
        T.ai[k] = (float)(vi[k] * sc);
        T.rho2[k] = (float)(real(1) - r * r * sc * sc);
    }
    T.th_lo = trig_eval(T, p.trig_lo).th;
}

MB_HD TrigRecon load_trig_recon(const float* __restrict__ rc, int64_t npix, int64_t pix) {
    TrigRecon T;
    T.m0 = rc[0 * npix + pix];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        T.ar[k] = rc[(1 + k) * npix + pix];
        T.ai[k] = rc[(5 + k) * npix + pix];
        T.rho2[k] = rc[(9 + k) * npix + pix];
    }
    T.th_lo = rc[13 * npix + pix];
    return T;
}

MB_HD void store_trig_recon(const TrigRecon& T, float* __restrict__ rc, int64_t npix, int64_t pix) {
    rc[0 * npix + pix] = T.m0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        rc[(1 + k) * npix + pix] = T.ar[k];
        rc[(5 + k) * npix + pix] = T.ai[k];
        rc[(9 + k) * npix + pix] = T.rho2[k];
    }
    rc[13 * npix + pix] = T.th_lo;
}

}  // namespace mb
