// Shared device code of the GB300 moment-based Gaussian rasterizer.
//
// Everything here runs in FP32 except the per-Gaussian preprocessing
// (preprocess.cu, FP64).  Notation follows "Moment-Based 3D Gaussian
// Splatting" (MB3DGS): mu, Sigma, w-hat of the ray-parameterised Gaussian
// (Eq. 4-6), warped depth g-hat (Sec. 3.2), moments (Eq. 10-12), moment
// bounds L, U (Eq. 8), quadrature (Eq. 7), rescaling (Eq. 15).
#pragma once
#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

#include "../../include/mb3dgs.h"

namespace mb {

constexpr int TPB = 256;              // threads per raster block: one per pixel of a 256-pixel tile
constexpr int NMOM = 9;               // 2n+1 moments, n = 4
constexpr int NQ = 4;                 // n: roots of the kernel polynomial
constexpr int REC = 32;               // floats per (view, Gaussian) record
constexpr int RECON = 20;             // floats per pixel of reconstruction state
constexpr int MAX_NODES = 9;          // N+1 <= 9 sample points
constexpr int LAG_ITERS = 4;          // Laguerre iterations per root
constexpr int SCHED_BYTES = 512;      // tile-queue counters and order buckets
constexpr double OUTER_SPAN = 8.0;   // outer-root search span beyond the Gauss nodes (y units)
constexpr int TAB_SEGS = 5;           // segments of the tabulated transmittance (between Gauss nodes)

// record field offsets (floats)
enum RecField {
    R_C0 = 0,    // o_g x g_a (3)
    R_CX = 3,    // o_g x m_x (3)
    R_CY = 6,    // o_g x m_y (3)
    R_GA = 9,    // g_a = S^-1 R^T K^-1 (anchor, 1) (3)
    R_MX = 12,   // m_x = S^-1 R^T e_x / f_x (3)
    R_MY = 15,   // m_y = S^-1 R^T e_y / f_y (3)
    R_O0 = 18,   // o_g.g_a
    R_OX = 19,   // o_g.m_x
    R_OY = 20,   // o_g.m_y
    R_LNW = 21,  // ln w
    R_RGB = 22,  // SH colour (3)
    R_AX = 25,   // anchor pixel-centre x (half-integer)
    R_AY = 26,
    R_RECT = 27, // int x0, y0, x1, y1 (inclusive pixel range; x0 > x1 = empty)
    R_FLAGS = 31 // int: bit0 visible, bit1 full-image proxy
};

struct ViewDesc {
    float R[9];        // world->camera rotation, row-major
    float t[3];
    float fx, fy, cx, cy;
    int width, height;
    int tiles_x, tiles_y;
    int tile_w, tile_h;  // pixels per tile (tile_w * tile_h = TPB)
    int tile_base;     // first global tile index of this view
    int64_t pixel_base;  // first global pixel index of this view
};

struct ViewTable {
    int n_views;
    ViewDesc v[MB3DGS_MAX_VIEWS];
};

// Method constants passed by value to every kernel.
struct Params {
    int n_intervals;
    int batch;        // Gaussian records staged in shared memory at a time (<= TPB)
    int schedule;     // MB3DGS_SCHEDULE_*
    float kappa, beta, conf_c, t_near, t_far, eps, bias_alpha, m_min, r_mult;
    float bg[3];
    float warp_lambda;
    // g-hat(t) = G0 + G1 (1 + 2t/a)^lambda, g-hat'(t) = G2 (1 + 2t/a)^(lambda-1), a = |lambda-1|
    float G0, G1, G2, G3, two_over_a;   // g-hat''(t) = G3 (1 + 2t/a)^(lambda-2)
    float gl_y[5], gl_w[5];   // 5-point Gauss-Legendre rule for U[-1,1] (probability weights)
    int lam_is_m15;        // lambda == -1.5: powers via rsqrt
    float x_nodes[MAX_NODES];    // standard-normal sample nodes (App. B)
    // A sample that is not clamped to [t_n, t_f] sits at mu + kappa Sigma x_j,
    // so b_j = (t_j - mu) / (sqrt2 Sigma) = kappa x_j / sqrt2 is a constant of
    // the node: erf(b_j) and e^{-b_j^2}, evaluated on the host in double.
    float x_erf[MAX_NODES], x_gau[MAX_NODES];
    float sh_c[16];        // real SH normalisation constants
    float leg_to_pow[NMOM * NMOM]; // m-hat_k = sum_l leg_to_pow[k*9+l] I_l
    int strict;
    int moment_dtype;
    int basis;             // MB3DGS_BASIS_POWER | MB3DGS_BASIS_TRIG
    float trig_A;          // angle range 2 pi - theta of the trigonometric moments
    float trig_lo;         // cut -theta/2 (middle of the wrapping zone)
    float cstar_re[4], cstar_im[4];   // moments of the uniform distribution on [0, A] (bias target)
    int tab_m;             // knots per segment of the tabulated transmittance (0: off)
    int qbytes;            // bytes of a kept bound query: 16, or 8 with compact queries
};

// Workspace layout (byte offsets), computed on the host.
// Device status word at the start of every workspace (64 bytes).
struct StatusWords {
    int status;                     // MB3DGS_* code (atomicMin of errors)
    int pad;
    long long n_total;              // (tile, Gaussian) pairs of the frame
    long long n_valid;              // pairs written (0 when over capacity)
    unsigned long long nonfinite;   // Gaussians with non-finite parameters
    unsigned long long n_pixpairs;  // (pixel, Gaussian) pairs: pixel centre in the proxy rectangle
};
static_assert(sizeof(StatusWords) <= 64, "status region");

struct Layout {
    size_t status;      // int32 status; int32 pad; int64 n_pairs_total; int64 n_pairs_valid; int64 n_nonfinite
    size_t rec;         // float [VP][REC]
    size_t counts;      // int32 [VP]
    size_t offsets;     // int32 [VP]
    size_t scan_tmp;    // int32 scratch for the scans
    size_t keys[2];     // uint32 [cap] ping-pong
    size_t vals[2];     // int32  [cap]
    size_t hist;        // uint32 [256][nb_sort]
    size_t ranges;      // int32 [T][2]
    size_t moments;     // F32: float [9][NPIX]; 16-bit: float [NPIX], then 16-B aligned uint4 [NPIX] (8 halves a pixel)
    size_t recon;       // float [RECON][NPIX]
    size_t saved;       // float [4][NPIX]: sum L (3), O
    size_t dm;          // float [9][NPIX] adjoint moments (backward)
    size_t grec;        // float [VP][28] per-record gradients (backward)
    size_t order;       // int32 [T] tiles in work order (longest list first)
    size_t sched;       // SCHED_BYTES: per-launch tile queues, bucket counts and cursors
    size_t npp;         // int32 [NPIX] (pixel, Gaussian) pairs per pixel
    size_t pq_off;      // int64 [NPIX] exclusive scan of npp
    size_t pq;          // [qcap][N+1] saved bound queries: float4 {tau, x0, x1, j | nroot << 4}, or 8-byte compact
    size_t tab_e;       // float [4][NPIX] segment edges of the tabulated transmittance
    size_t tab;         // float2 [5 (M+1)][NPIX] tabulated (tau, dtau/deta)
    int tab_m;          // knots per segment M (0: no table)
    size_t total;
    int64_t VP, P, npix, cap;
    int64_t qcap;       // query slots (0: queries are recomputed by the backward); a pixel keeps
                        // its queries iff all of its pairs fit (pq_off + npp <= qcap)
    int64_t n_tiles;
    int nb_sort, sort_passes, final_buf;
    int n_views;
    size_t scan_tmp_elems;
};

__host__ __device__ inline int64_t ceil_div64(int64_t a, int64_t b) { return (a + b - 1) / b; }

#define MB_HD __host__ __device__ __forceinline__

// approximate division (2 ulp) where the quotient feeds an iteration or a weight
MB_HD float fdiv_(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fdividef(a, b);
#else
    return a / b;
#endif
}

// approximate exponential (2 ulp + the rounding of x log2 e) where a relative
// error of ~1e-6 is far below the parity bar: per-pair weights, carried T
MB_HD float exp_(float x) {
#ifdef __CUDA_ARCH__
    return __expf(x);
#else
    return expf(x);
#endif
}

MB_HD float rsqrt_(float x) {
#ifdef __CUDA_ARCH__
    return rsqrtf(x);
#else
    return 1.0f / sqrtf(x);
#endif
}

// ----------------------------------------------------------------------------
// warp g-hat and its derivative (Sec. 3.2; power transform with lambda)
// ----------------------------------------------------------------------------
MB_HD void warp_g(const Params& p, float t, float& g, float& dg) {
    float z = fmaf(p.two_over_a, t, 1.0f);
    float zl, zl1;
    if (p.lam_is_m15) {
        float r = rsqrt_(z);
        zl = r * r * r;          // z^-1.5
        zl1 = zl * (r * r);      // z^-2.5
    } else {
        zl = powf(z, p.warp_lambda);
        zl1 = zl / z;
    }
    g = fmaf(p.G1, zl, p.G0);
    dg = p.G2 * zl1;
}

MB_HD float warp_only(const Params& p, float t) {
    float z = fmaf(p.two_over_a, t, 1.0f);
    float zl;
    if (p.lam_is_m15) {
        float r = rsqrt_(z);
        zl = r * r * r;
    } else {
        zl = powf(z, p.warp_lambda);
    }
    return fmaf(p.G1, zl, p.G0);
}

// ----------------------------------------------------------------------------
// Ray-parameterised 1D Gaussian of one (pixel, Gaussian) pair (Eq. 4-6).
// The record holds o_g x d_g, |d_g|^2 and o_g.d_g as polynomials in the pixel
// offset (dx, dy) from an anchor pixel centre, so the only per-pair rounding is
// in small, well-conditioned quantities.
// ----------------------------------------------------------------------------
struct Gauss1D {
    float mu, Sig, Sig2, what;
};

MB_HD Gauss1D pair_gaussian(const float* __restrict__ r, float dx, float dy, float rlen,
                                                 float r2) {
    float vx = fmaf(dy, r[R_CY + 0], fmaf(dx, r[R_CX + 0], r[R_C0 + 0]));
    float vy = fmaf(dy, r[R_CY + 1], fmaf(dx, r[R_CX + 1], r[R_C0 + 1]));
    float vz = fmaf(dy, r[R_CY + 2], fmaf(dx, r[R_CX + 2], r[R_C0 + 2]));
    float cross2 = fmaf(vx, vx, fmaf(vy, vy, vz * vz));
    // d_g = g_a + dx m_x + dy m_y as a vector: |d_g|^2 >= 0 and no squared cancellation
    const float gx = fmaf(dy, r[R_MY + 0], fmaf(dx, r[R_MX + 0], r[R_GA + 0]));
    const float gy = fmaf(dy, r[R_MY + 1], fmaf(dx, r[R_MX + 1], r[R_GA + 1]));
    const float gz = fmaf(dy, r[R_MY + 2], fmaf(dx, r[R_MX + 2], r[R_GA + 2]));
    float dd = fmaf(gx, gx, fmaf(gy, gy, gz * gz));
    float od = fmaf(dy, r[R_OY], fmaf(dx, r[R_OX], r[R_O0]));
    float inv = fdiv_(1.0f, dd);
    Gauss1D g;
    g.Sig2 = r2 * inv;
    g.Sig = g.Sig2 * rsqrt_(g.Sig2);      // Sigma^2 > 0: |d_g|^2 of a finite record is positive
    g.mu = -od * rlen * inv;
    g.what = exp_(fmaf(-0.5f * cross2, inv, r[R_LNW]));
    return g;
}

MB_HD bool rect_contains(const float* __restrict__ r, int px, int py) {
    const int* ri = reinterpret_cast<const int*>(r + R_RECT);
    return px >= ri[0] && px <= ri[2] && py >= ri[1] && py <= ri[3];
}

// ----------------------------------------------------------------------------
// Moments of one Gaussian in the Legendre basis of y = 2 g-hat - 1 (App. C
// recurrence, rewritten for P_k): with y_t = A + S (t - mu) the linearised
// warp, I_k = int_{t_n}^inf P_k(y_t) w-hat e^{-(t-mu)^2/(2 Sigma^2)} dt obeys
// (k+1) I_{k+1} + k I_{k-1} = (2k+1) [A I_k + S Sigma^2 (P_k(y_n) G_n + S D_k)],
// D_k = int P_k'(y_t) G dt = sum_{j = k-1, k-3, ..} (2j+1) I_j,
// and I_0 = m-hat_0 (Eq. 10).  Same moment space as the power moments.  The
// warp is linearised at max(mu, t_n) (it is defined on [t_n, t_f] only).
// ----------------------------------------------------------------------------
MB_HD void legendre_moments(const Params& p, const Gauss1D& g, float acc[NMOM]) {
    // g-hat lives on [t_n, t_f]: linearise at c = max(mu, t_n), u = a + s (t - mu)
    const float cpt = fmaxf(g.mu, p.t_near);
    float a, s;
    warp_g(p, cpt, a, s);
    a = fmaf(s, g.mu - cpt, a);
    const float A = fmaf(2.0f, a, -1.0f);
    const float S = 2.0f * s;
    const float bn = (p.t_near - g.mu) * (0.70710678118654752f / g.Sig);
    const float I0 = g.what * g.Sig * 1.25331413731550025f * erfcf(bn);
    const float Gn = g.what * expf(-bn * bn);
    const float yn = fmaf(S, p.t_near - g.mu, A);
    const float SS2 = S * g.Sig2;
    float Ikm1 = 0.0f, Ik = I0, Pkm1 = 0.0f, Pk = 1.0f, Dkm1 = 0.0f, Dk = 0.0f;
    acc[0] += I0;
#pragma unroll
    for (int k = 0; k < NMOM - 1; ++k) {
        const float c2k1 = (float)(2 * k + 1);
        const float inv = 1.0f / (float)(k + 1);
        float t = fmaf(A, Ik, SS2 * fmaf(Pk, Gn, S * Dk));
        float In = (c2k1 * t - (float)k * Ikm1) * inv;
        acc[k + 1] += In;
        float Pn = (c2k1 * yn * Pk - (float)k * Pkm1) * inv;
        float Dn = fmaf(c2k1, Ik, Dkm1);
        Ikm1 = Ik; Ik = In;
        Pkm1 = Pk; Pk = Pn;
        Dkm1 = Dk; Dk = Dn;
    }
}

// ----------------------------------------------------------------------------
// Per-pixel reconstruction state (Sec. 3.2).  The biased, normalised measure's
// monic orthogonal polynomials pi_k obey pi_{k+1} = (y - al_k) pi_k - be_k
// pi_{k-1}; the modified Chebyshev algorithm (Gautschi) gets al, be from the
// Legendre moments.  The canonical representation through eta is the
// Gauss-Radau rule with a node at eta; its other nodes are the roots of the
// kernel polynomial K(x, eta) = sum_k h_k pi_k(x) pi_k(eta), h_k =
// 1/(be_1..be_k), and they interlace with the Gauss nodes z (roots of pi_4).
// Weights are 1/K(x, x) (Christoffel).
// ----------------------------------------------------------------------------
struct Recon {
    float m0;
    float c, inv_s;   // standardisation y' = (y - c) / s, c = al_0, s = sqrt(be_1) (mean / std of the measure)
    float span;       // outer-root search span (8 y-units) in standardised units
    float al[4];      // standardised recurrence coefficients (al[0] = 0)
    float be[4];      // be_1..be_4 (be[0] = 1)
    float h[4];       // h_1..h_4
    float z[4];       // Gauss nodes, ascending
};

MB_HD void pis(const Recon& R, float x, float P[5]) {
    P[0] = 1.0f;
    P[1] = x - R.al[0];
    P[2] = fmaf(x - R.al[1], P[1], -R.be[0] * P[0]);
    P[3] = fmaf(x - R.al[2], P[2], -R.be[1] * P[1]);
    P[4] = fmaf(x - R.al[3], P[3], -R.be[2] * P[2]);
}

MB_HD float kernel_poly(const Recon& R, const float e[5], float x) {
    float P[5];
    pis(R, x, P);
    return e[0] * P[0] + e[1] * P[1] + e[2] * P[2] + e[3] * P[3] + e[4] * P[4];
}

MB_HD float christoffel_weight(const Recon& R, float x) {
    float P[5];
    pis(R, x, P);
    float K = 1.0f + R.h[0] * P[1] * P[1] + R.h[1] * P[2] * P[2] + R.h[2] * P[3] * P[3] + R.h[3] * P[4] * P[4];
    float w = fdiv_(1.0f, K);
    return isfinite(w) ? w : 0.0f;
}

// Monomial coefficients c of K(., y) = sum_k e_k pi_k (standardised x), from
// Clenshaw's recurrence carried out on polynomials: r_4 = e_4,
// r_k = e_k + (x - al_k) r_{k+1} - be_k r_{k+2} (be indexed as in pis), K = r_0.
MB_HD void kernel_monomials(const Recon& R, const float e[5], float c[5]) {
    const float r3_0 = fmaf(-R.al[3], e[4], e[3]);
    const float r2_0 = fmaf(-R.al[2], r3_0, fmaf(-R.be[2], e[4], e[2]));
    const float r2_1 = fmaf(-R.al[2], e[4], r3_0);
    const float r1_0 = fmaf(-R.al[1], r2_0, fmaf(-R.be[1], r3_0, e[1]));
    const float r1_1 = fmaf(-R.al[1], r2_1, fmaf(-R.be[1], e[4], r2_0));
    const float r1_2 = fmaf(-R.al[1], e[4], r2_1);
    c[0] = fmaf(-R.al[0], r1_0, fmaf(-R.be[0], r2_0, e[0]));
    c[1] = fmaf(-R.al[0], r1_1, fmaf(-R.be[0], r2_1, r1_0));
    c[2] = fmaf(-R.al[0], r1_2, fmaf(-R.be[0], e[4], r1_1));
    c[3] = fmaf(-R.al[0], e[4], r1_2);
    c[4] = e[4];
}

// One Laguerre step for a degree-4 polynomial with value f, f' and f''.
// The square root is approximate (it sets the step; the residual f of the
// next evaluation sets the root).  den = f' - q or f' + q signed with f, the
// denominator towards the neighbouring root on the chosen side.  The clamp to
// [lo, hi] also maps a non-finite step (den = 0) into the bracket.
MB_HD float laguerre_step(float x, float f, float fp, float fpp, float lo, float hi, bool right) {
    const float v = fmaxf(3.0f * fmaf(3.0f * fp, fp, -4.0f * f * fpp), 1e-30f);
    const float q = v * rsqrt_(v);
    const float den = fp + copysignf(q, right ? -f : f);
    const float xn = x - (f != 0.0f ? fdiv_(4.0f * f, den) : 0.0f);
    return fminf(fmaxf(xn, lo), hi);
}

// K(x) = sum_k e_k pi_k(x) and its first two derivatives through the
// three-term recurrence (the accurate form near a root).
MB_HD void kernel_poly_d2(const Recon& R, const float e[5], float x, float& f, float& fp, float& fpp) {
    float p0 = 1.0f, p1 = x - R.al[0];
    float d0 = 0.0f, d1 = 1.0f;
    float s0 = 0.0f, s1 = 0.0f;
    f = e[0] + e[1] * p1;
    fp = e[1];
    fpp = 0.0f;
#pragma unroll
    for (int k = 1; k < 4; ++k) {
        const float xa = x - R.al[k];
        const float b = R.be[k - 1];
        float p2 = fmaf(xa, p1, -b * p0);
        float d2 = fmaf(xa, d1, fmaf(-b, d0, p1));
        float s2 = fmaf(xa, s1, fmaf(-b, s0, 2.0f * d1));
        f = fmaf(e[k + 1], p2, f);
        fp = fmaf(e[k + 1], d2, fp);
        fpp = fmaf(e[k + 1], s2, fpp);
        p0 = p1; p1 = p2; d0 = d1; d1 = d2; s0 = s1; s1 = s2;
    }
}

// Laguerre iteration towards the neighbouring root on one side.  For a
// real-rooted polynomial the iterates move monotonically to the adjacent root
// in the chosen direction, cubically near it.  All but the last step evaluate
// the kernel polynomial by Horner's rule on its monomial coefficients c; the
// last step evaluates it through the three-term recurrence (coefficients e),
// which sets the accuracy of the root.
MB_HD float laguerre(const Recon& R, const float e[5], const float c[5], float x, float lo, float hi,
                     bool right) {
#pragma unroll
    for (int it = 0; it < LAG_ITERS - 1; ++it) {
        float f = c[4], d1 = 0.0f, d2 = 0.0f;
#pragma unroll
        for (int k = 3; k >= 0; --k) {
            d2 = fmaf(d2, x, d1);
            d1 = fmaf(d1, x, f);
            f = fmaf(f, x, c[k]);
        }
        x = laguerre_step(x, f, d1, 2.0f * d2, lo, hi, right);
    }
    float f, fp, fpp;
    kernel_poly_d2(R, e, x, f, fp, fpp);
    return laguerre_step(x, f, fp, fpp, lo, hi, right);
}

// Roots of one bound query, kept by the backward pass (standardised units).
struct QueryRec {
    float y;        // standardised query
    int j;          // number of Gauss nodes below y
    int nroot;      // roots used (0..2)
    float x[2];     // their positions
    float F;        // (1 - beta) L + beta U
};

// Bracket of root sv of a query with j Gauss nodes below it (1 <= j <= 3),
// as bound_query solves them (the same expressions, written inline there):
// the interior root in (z_1, z_2) first when j == 2, then the outer root
// beyond z_1 (j <= 2) or z_4 (j == 3).
MB_HD void root_bracket(const Recon& R, int j, int sv, float& lo, float& hi) {
    const bool left = j <= 2;
    const float zb = left ? R.z[0] : R.z[3];
    const float far = left ? zb - R.span : zb + R.span;
    const bool in = j == 2 && sv == 0;
    lo = in ? R.z[0] : (left ? far : zb);
    hi = in ? R.z[1] : (left ? zb : far);
}

// tau(eta) = m0 ((1 - beta) L + beta U) = m0 (L + beta w0) at warped depth
// y = 2 eta - 1 (Sec. 3.2, Eq. 8).  REC keeps the roots for the adjoint.
template <bool REC>
MB_HD float bound_query(const Recon& R, float beta, float y_raw, QueryRec* rec) {
    if (REC) { rec->nroot = 0; rec->j = 0; rec->F = 0.0f; rec->y = 0.0f; rec->x[0] = 0.0f; rec->x[1] = 0.0f; }
    if (R.m0 <= 0.0f) return 0.0f;
    const float y = (y_raw - R.c) * R.inv_s;
    float P[5];
    pis(R, y, P);
    float e[5];
    e[0] = 1.0f;
    e[1] = R.h[0] * P[1];
    e[2] = R.h[1] * P[2];
    e[3] = R.h[2] * P[3];
    e[4] = R.h[3] * P[4];
    const float K = 1.0f + e[1] * P[1] + e[2] * P[2] + e[3] * P[3] + e[4] * P[4];
    const float w0 = fdiv_(1.0f, K);
    const int j = (R.z[0] < y) + (R.z[1] < y) + (R.z[2] < y) + (R.z[3] < y);
    if (REC) { rec->y = y; rec->j = j; }
    // scale the kernel coefficients (roots are scale invariant) to keep f^2 finite
    const float sc = fdiv_(1.0f, fabsf(e[0]) + fabsf(e[1]) + fabsf(e[2]) + fabsf(e[3]) + fabsf(e[4]));
#pragma unroll
    for (int k = 0; k < 5; ++k) e[k] *= sc;
    float L;
    if (j == 0) {
        L = 0.0f;
    } else if (j == NQ) {
        L = 1.0f - w0;
    } else {
        const bool left = (j <= 2);
        const float zb = left ? R.z[0] : R.z[3];
        const float far = left ? zb - R.span : zb + R.span;
        const bool inner = j == 2;
        // The nodes of the representation through y interlace with the Gauss
        // nodes, and K(., y) > 0 on the root-free interval around y.  Between
        // `far` and y lie: the outer root (if any) and, for j == 2, exactly one
        // interior root.  So the outer root exists iff K(far) < 0 (j = 1, 3) or
        // K(far) > 0 (j = 2).  Testing the sign at the outer Gauss node instead
        // fails when a root sits within rounding of that node (y next to the
        // neighbouring node).
        const float ff = kernel_poly(R, e, far);
        const bool outer = (ff < 0.0f) != inner;
        const int ns = (int)outer + (int)inner;
        float c[5];
        kernel_monomials(R, e, c);
        float acc = 0.0f;
        // At most two root solves, through one copy of the solver so that
        // lanes needing one root of either kind iterate together: first the
        // interior root in (z_1, z_2) approached from z_2 (next to eta's
        // interval) when j == 2, then the outer root left of z_1 (j <= 2) or
        // right of z_4 (j == 3) when K changes sign beyond the nodes.
        // (root_bracket restates these brackets for the compact kept queries;
        // here they stay inline, where the loop-invariant parts are hoisted)
#pragma unroll 1
        for (int sv = 0; sv < ns; ++sv) {
            const bool in = inner && sv == 0;
            const float x0 = in ? R.z[1] : far;
            const float lo = in ? R.z[0] : (left ? far : zb);
            const float hi = in ? R.z[1] : (left ? zb : far);
            const float x = laguerre(R, e, c, x0, lo, hi, !in && left);
            acc += christoffel_weight(R, x);
            if (REC) {   // static indices keep the record in registers
                if (sv == 0) rec->x[0] = x;
                else rec->x[1] = x;
            }
        }
        if (REC) rec->nroot = ns;
        L = left ? acc : 1.0f - w0 - acc;
    }
    L = fminf(fmaxf(L, 0.0f), 1.0f - w0);
    const float F = fmaf(beta, w0, L);
    if (REC) rec->F = F;
    return R.m0 * F;
}

MB_HD float optical_depth(const Recon& R, float beta, float y_raw) {
    return bound_query<false>(R, beta, y_raw, nullptr);
}

// A bound query kept by the quadrature pass for the adjoint (one float4):
// {tau, x_0, x_1, j | nroot << 4}; the standardised y is recomputed.
MB_HD float int_bits_as_float(int i) {
#ifdef __CUDA_ARCH__
    return __int_as_float(i);
#else
    float f;
    memcpy(&f, &i, 4);
    return f;
#endif
}
MB_HD int float_bits_as_int(float f) {
#ifdef __CUDA_ARCH__
    return __float_as_int(f);
#else
    int i;
    memcpy(&i, &f, 4);
    return i;
#endif
}
MB_HD float4 pack_query(float tau, const QueryRec& q) {
    return make_float4(tau, q.x[0], q.x[1], int_bits_as_float(q.j | (q.nroot << 4)));
}
MB_HD float unpack_query(const float4 v, float y, QueryRec& q) {
    const int m = float_bits_as_int(v.w);
    q.y = y;
    q.j = m & 15;
    q.nroot = m >> 4;
    q.x[0] = v.y;
    q.x[1] = v.z;
    q.F = 0.0f;
    return v.x;
}

// Compact kept query (8 bytes): {tau, bits}, bits = u_0 | u_1 << 16 with u_r
// the 16-bit position of root r in its bracket (QPOS_NONE: no outer root).
// The number j of Gauss nodes below y is not stored: the adjoint recomputes
// y with the same operations, so the same j; the interior root (j == 2) is
// root 0 and always present.
constexpr unsigned QPOS_NONE = 0xFFFFu;
constexpr float QPOS_SCALE = 65535.0f;
#ifndef MB_QPOS_POLISH
#define MB_QPOS_POLISH 1
#endif
MB_HD float2 pack_query_compact(const Recon& R, float tau, const QueryRec& q) {
    unsigned code[2] = {QPOS_NONE, QPOS_NONE};
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        if (r < q.nroot) {
            float lo, hi;
            root_bracket(R, q.j, r, lo, hi);
            const float u = (q.x[r] - lo) / (hi - lo);
            code[r] = (unsigned)fminf(fmaxf(u * QPOS_SCALE + 0.5f, 0.0f), QPOS_SCALE - 1.0f);
        }
    }
    return make_float2(tau, int_bits_as_float((int)(code[0] | (code[1] << 16))));
}

// One Laguerre step towards the nearest root (the larger denominator), for
// polishing a root known to a few 1e-6 of its bracket.
MB_HD float laguerre_nearest_step(float x, float f, float fp, float fpp, float lo, float hi) {
    const float v = fmaxf(3.0f * fmaf(3.0f * fp, fp, -4.0f * f * fpp), 1e-30f);
    const float q = v * rsqrt_(v);
    const float xn = x - (f != 0.0f ? fdiv_(4.0f * f, fp + copysignf(q, fp)) : 0.0f);
    return fminf(fmaxf(xn, lo), hi);
}

// Decodes a compact kept query at standardised y: j from y, each root from
// its 16-bit position (within 8e-6 of its bracket), polished by MB_QPOS_POLISH
// Laguerre steps of the kernel polynomial through the three-term recurrence.
MB_HD float unpack_query_compact(const Recon& R, float2 v, float y, QueryRec& q) {
    const unsigned bits = (unsigned)float_bits_as_int(v.y);
    q.y = y;
    q.j = (R.z[0] < y) + (R.z[1] < y) + (R.z[2] < y) + (R.z[3] < y);
    q.F = 0.0f;
    q.x[0] = 0.0f;
    q.x[1] = 0.0f;
    const unsigned c0 = bits & 0xFFFFu, c1 = bits >> 16;
    // slot 0: the interior root (j == 2, always) or the outer one (j = 1, 3)
    q.nroot = (q.j >= 1 && q.j <= 3 && c0 != QPOS_NONE) ? 1 + (q.j == 2 && c1 != QPOS_NONE) : 0;
    if (R.m0 <= 0.0f) q.nroot = 0;
#if MB_QPOS_POLISH > 0
    float e[5];
    if (q.nroot > 0) {
        float P[5];
        pis(R, y, P);
        e[0] = 1.0f;
#pragma unroll
        for (int k = 1; k < 5; ++k) e[k] = R.h[k - 1] * P[k];
        // the same scaling as the solve (roots are scale invariant)
        const float sc = fdiv_(1.0f, fabsf(e[0]) + fabsf(e[1]) + fabsf(e[2]) + fabsf(e[3]) + fabsf(e[4]));
#pragma unroll
        for (int k = 0; k < 5; ++k) e[k] *= sc;
    }
#endif
#pragma unroll 1
    for (int r = 0; r < q.nroot; ++r) {
        float lo, hi;
        root_bracket(R, q.j, r, lo, hi);
        float x = fmaf(hi - lo, (float)(r == 0 ? c0 : c1) * (1.0f / QPOS_SCALE), lo);
#if MB_QPOS_POLISH > 0
#pragma unroll
        for (int it = 0; it < MB_QPOS_POLISH; ++it) {
            float f, fp, fpp;
            kernel_poly_d2(R, e, x, f, fp, fpp);
            x = laguerre_nearest_step(x, f, fp, fpp, lo, hi);
        }
#endif
        if (r == 0) q.x[0] = x;
        else q.x[1] = x;
    }
    return v.x;
}

#ifndef MB_RECON_T
#define MB_RECON_T double
#endif
MB_HD void reconstruct_pixel(const Params& p, const float I[NMOM], Recon& R) {
    typedef MB_RECON_T real;
    R.m0 = I[0];
    if (!(I[0] >= p.m_min) || !isfinite(I[0])) {
        R.m0 = 0.0f;
        R.c = 0.0f; R.inv_s = 1.0f; R.span = 1.0f;
#pragma unroll
        for (int k = 0; k < 4; ++k) { R.al[k] = 0.0f; R.be[k] = 0.25f; R.h[k] = 1.0f; R.z[k] = 0.0f; }
        return;
    }
    // monic-Legendre modified moments of the normalised measure, biased towards U[-1,1]
    const real cl[NMOM] = {1.0, 1.0, 2.0 / 3.0, 2.0 / 5.0, 8.0 / 35.0, 8.0 / 63.0, 16.0 / 231.0, 16.0 / 429.0,
                           128.0 / 6435.0};
    const real inv0 = real(1) / (real)I[0];
    real alr[4], ber[5];
    // Moments rounded to 16-bit storage can leave the feasible set (a
    // non-positive be_k); the bias towards U[-1,1] is then raised for this
    // pixel (x4 per attempt) until the recurrence is positive definite.  With
    // FP32 storage and the default bias the first attempt always succeeds.
    real alpha = (real)p.bias_alpha;
#pragma unroll 1
    for (int attempt = 0; attempt < 8; ++attempt) {
        const real oma = real(1) - alpha;
        real sg0[NMOM + 1], sg1[NMOM + 1], sg2[NMOM + 1];
#pragma unroll
        for (int l = 0; l < NMOM; ++l) {
            sg1[l] = cl[l] * (real)I[l] * inv0 * oma;
            sg0[l] = 0;
        }
        sg1[0] = 1;
        sg1[NMOM] = 0;
        sg0[NMOM] = 0;
        ber[0] = 1;
        alr[0] = sg1[1];
        bool ok = true;
#pragma unroll
        for (int k = 1; k <= 4; ++k) {
#pragma unroll
            for (int l = 0; l <= NMOM; ++l) sg2[l] = 0;
#pragma unroll
            for (int l = 1; l < NMOM; ++l) {
                if (l >= k && l <= 8 - k) {
                    const real bl = (real)(l * l) / (real)(4 * l * l - 1);
                    sg2[l] = sg1[l + 1] - alr[k - 1] * sg1[l] - ber[k - 1] * sg0[l] + bl * sg1[l - 1];
                }
            }
            ber[k] = sg2[k] / sg1[k - 1];
            if (!(ber[k] > real(1e-12)) || !(ber[k] < real(1e12))) ok = false;
            if (k < 4) alr[k] = sg2[k + 1] / sg2[k] - sg1[k] / sg1[k - 1];
#pragma unroll
            for (int l = 0; l <= NMOM; ++l) { sg0[l] = sg1[l]; sg1[l] = sg2[l]; }
        }
        if (ok || alpha >= real(0.5)) break;
        alpha = alpha * 4 < real(0.5) ? alpha * 4 : real(0.5);
    }
#pragma unroll
    for (int k = 1; k <= 4; ++k)
        if (!(ber[k] > real(1e-12))) ber[k] = real(1e-12);
    // standardise: y' = (y - al_0) / sqrt(be_1); al' = (al - al_0)/s, be' = be / s^2, h' = 1/prod be'
    const real sd = sqrt(ber[1]);
    const real isd = real(1) / sd;
    R.c = (float)alr[0];
    R.inv_s = (float)isd;
    const real span_max = OUTER_SPAN * isd;
    float al[4], be[5];
    be[0] = 1.0f;
    real hk = 1;
#pragma unroll
    for (int k = 0; k < 4; ++k) al[k] = (float)((alr[k] - alr[0]) * isd);
#pragma unroll
    for (int k = 1; k < 5; ++k) {
        const real bs = ber[k] * isd * isd;
        be[k] = (float)bs;
        hk = hk / bs;
        R.h[k - 1] = (float)hk;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) { R.al[k] = al[k]; R.be[k] = be[k + 1]; }
    // Beyond distance d of the outermost Gauss node a root's Christoffel weight is
    // below 1/(h_4 d^8) (K(x,x) >= h_4 pi_4(x)^2 >= h_4 d^8): search only up to
    // the d where that bound reaches 1e-7, at most 8 warped-depth units.
    {
        real d = pow((real)R.h[3] * real(1e-7), real(-0.125));
        d = d < real(1) ? real(1) : d;
        R.span = (float)(d < span_max ? d : span_max);
    }
    // Gauss nodes: eigenvalues of the 4x4 Jacobi matrix by Sturm-count bisection
    float sb[4];
    sb[0] = 0.0f;
    sb[1] = sqrtf(be[1]); sb[2] = sqrtf(be[2]); sb[3] = sqrtf(be[3]);
    float lo = 1e30f, hi = -1e30f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float rad = (k > 0 ? sb[k] : 0.0f) + (k < 3 ? sb[k + 1] : 0.0f);
        lo = fminf(lo, al[k] - rad);
        hi = fmaxf(hi, al[k] + rad);
    }
    lo -= 1e-6f * (fabsf(lo) + 1.0f);
    hi += 1e-6f * (fabsf(hi) + 1.0f);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        float a = lo, b = hi;
#pragma unroll 1
        for (int it = 0; it < 40; ++it) {
            const float x = 0.5f * (a + b);
            int cnt = 0;
            float d = al[0] - x;
            cnt += d < 0.0f;
#pragma unroll
            for (int k = 1; k < 4; ++k) {
                if (fabsf(d) < 1e-30f) d = -1e-30f;
                d = (al[k] - x) - be[k] / d;
                cnt += d < 0.0f;
            }
            if (cnt > e) b = x; else a = x;
        }
        R.z[e] = 0.5f * (a + b);
    }
}

MB_HD Recon load_recon(const float* __restrict__ rc, int64_t npix, int64_t pix) {
    Recon R;
    R.m0 = rc[0 * npix + pix];
    R.c = rc[1 * npix + pix];
    R.inv_s = rc[2 * npix + pix];
    R.span = rc[3 * npix + pix];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        R.al[k] = rc[(4 + k) * npix + pix];
        R.be[k] = rc[(8 + k) * npix + pix];
        R.h[k] = rc[(12 + k) * npix + pix];
        R.z[k] = rc[(16 + k) * npix + pix];
    }
    return R;
}

MB_HD void store_recon(const Recon& R, float* __restrict__ rc, int64_t npix, int64_t pix) {
    rc[0 * npix + pix] = R.m0;
    rc[1 * npix + pix] = R.c;
    rc[2 * npix + pix] = R.inv_s;
    rc[3 * npix + pix] = R.span;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        rc[(4 + k) * npix + pix] = R.al[k];
        rc[(8 + k) * npix + pix] = R.be[k];
        rc[(12 + k) * npix + pix] = R.h[k];
        rc[(16 + k) * npix + pix] = R.z[k];
    }
}

}  // namespace mb
#include "trig.cuh"
namespace mb {

// ----------------------------------------------------------------------------
// Per-pair quadrature (Eq. 7 with App. B samples) and penalty (App. D).
// NI > 0: compile-time number of intervals; NI == 0: runtime p.n_intervals.
// Returns O_i; adds P_i to *pen.
// ----------------------------------------------------------------------------
// Optical depth at warped depth gq of one sample: power-moment bounds (with
// the query kept for the adjoint when qout != nullptr) or trigonometric ones.
template <bool SAVE, int QB = 16>
MB_HD float sample_depth(const Params& p, const Recon& R, float gq, char* qout) {
    const float y = fmaf(2.0f, gq, -1.0f);
    if (SAVE && qout) {
        QueryRec q;
        const float tau = bound_query<true>(R, p.beta, y, &q);
        if (QB == 8) *reinterpret_cast<float2*>(qout) = pack_query_compact(R, tau, q);
        else *reinterpret_cast<float4*>(qout) = pack_query(tau, q);
        return tau;
    }
    return optical_depth(R, p.beta, y);
}
template <bool SAVE, int QB = 16>
MB_HD float sample_depth(const Params& p, const TrigRecon& T, float gq, char* qout) {
    if (SAVE && qout) {
        TrigQueryRec q;
        const float tau = trig_bound_query<true>(p, T, gq, &q);
        *reinterpret_cast<float4*>(qout) = pack_trig_query(tau, q);
        return tau;
    }
    return trig_optical_depth(p, T, gq);
}

template <int NI, bool SAVE = false, class RecT = Recon, int QB = 16>
MB_HD float pair_quadrature(const Params& p, const RecT& R, const Gauss1D& g, float* pen,
                            char* __restrict__ qout = nullptr) {
    // streamed over the samples (one copy of the bound-query code): interval
    // j-1 is accumulated once sample j is known
    const int N = NI > 0 ? NI : p.n_intervals;
    const float ks = p.kappa * g.Sig;
    const float isq = 0.70710678118654752f / g.Sig;
    const float tscale = g.what * g.Sig * 1.25331413731550025f;
    float O = 0.0f, P = 0.0f;
    float t_prev = 0.0f, tau_prev = 0.0f, erf_prev = 0.0f;
    float gau_prev = 0.0f;
    float T_prev = 0.0f;   // e^{-tau_prev}, carried: T_{j+1} = T_j e^{-dtau_j}
#pragma unroll 1
    for (int j = 0; j <= N; ++j) {
        const float raw = fmaf(ks, p.x_nodes[j], g.mu);
        const float tj = fminf(fmaxf(raw, p.t_near), p.t_far);
        const float tau = sample_depth<SAVE, QB>(p, R, warp_only(p, tj), qout ? qout + j * QB : nullptr);
        float erf_j = p.x_erf[j], gau_j = p.x_gau[j];
        if (tj != raw) {
            const float b = (tj - g.mu) * isq;
            erf_j = erff(b);
            gau_j = expf(-b * b);
        }
        if (j > 0) {
            const float Delta = tj - t_prev;
            const float dtau = fmaxf(tau - tau_prev, 0.0f);
            const float Tj = T_prev;
            const float sig = g.what * gau_prev;
            // (1 - e^{-dtau}) / dtau and e^{-dtau}: Taylor series to dtau^4 below
            // 0.05 (truncation < 5e-10), where 1 - e^{-dtau} cancels
            float ratio, em;
            if (dtau < 0.05f) {
                ratio = fmaf(dtau, fmaf(dtau, fmaf(dtau, fmaf(dtau, 1.0f / 120.0f, -1.0f / 24.0f), 1.0f / 6.0f), -0.5f),
                             1.0f);
                em = fmaf(-dtau, ratio, 1.0f);
            } else {
                em = exp_(-dtau);
                ratio = fdiv_(1.0f - em, dtau);
            }
            O = fmaf(Tj * ratio, sig * Delta, O);
            T_prev = Tj * em;
            const float tij = tscale * (erf_j - erf_prev);
            const float v = fmaxf(tij - dtau, 0.0f);
            P = fmaf(v, v, P);
        }
        if (j == 0) T_prev = exp_(-tau);
        t_prev = tj;
        tau_prev = tau;
        erf_prev = erf_j;
        gau_prev = gau_j;
    }
    *pen += P;
    return O;
}

// Pixel of a thread in a tile: each warp covers an 8 x 4 block (fewer
// partially covered warps than 32 x 1 rows for rectangle-shaped footprints),
// warps laid out row-major over the tile.
MB_HD void tile_pixel(const ViewDesc& V, int tx, int ty, int lane, int warp, int& px, int& py) {
    const int wpr = V.tile_w >> 3;
    px = tx * V.tile_w + (warp % wpr) * 8 + (lane & 7);
    py = ty * V.tile_h + (warp / wpr) * 4 + (lane >> 3);
}

MB_HD int find_view(const ViewTable& vt, int64_t tile) {
    int v = 0;
    for (int k = 1; k < vt.n_views; ++k)
        if (tile >= vt.v[k].tile_base) v = k;
    return v;
}

__device__ __forceinline__ void set_status(int* status, int code) { atomicMin(status, code); }

// host-side count of kernel launches issued by the library (for reporting)
void count_launch(int n = 1);

}  // namespace mb
