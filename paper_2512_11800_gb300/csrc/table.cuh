// Tabulated transmittance: a per-pixel table of the bound optical depth
// tau(eta) (Eq. 8) for the quadrature pass, in place of one bound query (a
// root solve of the kernel polynomial) per sample.
//
// tau is smooth in the warped depth eta between the Gauss nodes of the
// pixel's moment measure and has a kink at each node (the set of canonical
// nodes on the lower side changes there).  So [0, 1] is cut at the nodes
// that fall inside it into at most five segments, each sampled at M + 1
// knots with tau and dtau/deta (the same implicit derivative of the bound as
// the adjoint uses), and a query is the cubic Hermite interpolant of its
// segment.  The knots are Chebyshev-Lobatto spaced, u_i = (1 - cos(pi i / M))
// / 2 of the segment: tau changes fastest next to the nodes (the atoms of a
// concentrated measure sit there), where this spacing puts its knots (host
// study: a few times smaller error than equal spacing at the same M).  The
// table replaces only the forward queries: the adjoint needs the roots
// themselves, so with a table it solves them again and differentiates the
// solved bounds that the table approximates.
#pragma once
#include "backward.cuh"

namespace mb {

// Position of knot i of M in a segment, (1 - cos(pi i / M)) / 2.  The table
// build and the queries evaluate the same expression, so they agree on the
// knots whatever the rounding of the approximate cosine.
MB_HD float tab_knot_u(int i, int M) {
    const float x = 3.14159265358979324f * (float)i / (float)M;
#ifdef __CUDA_ARCH__
    return 0.5f * (1.0f - __cosf(x));
#else
    return 0.5f * (1.0f - cosf(x));
#endif
}

// dF/dy (standardised y) of the bound F = L + beta w0 at a solved query
// (Eq. 8): dw0/dy = -2 w0^2 d1K(y, y) and dw_i/dy = 2 w_i^2 rho_i d1K(y, x_i),
// rho_i = d1K(x_i, x_i) / d1K(x_i, y) (implicit differentiation of K(x_i, y)
// = 0 and of the Christoffel function).
MB_HD float bound_dF_dy(const Params& p, const Recon& R, const QueryRec& q) {
    if (R.m0 <= 0.0f) return 0.0f;
    float Py[5], Dy[5], ey[5];
    pis_d(R, q.y, Py, Dy);
    kernel_coeffs(R, Py, ey);
    const float w0 = fdiv_(1.0f, dot5(Py, ey));
    const float dw0 = -2.0f * w0 * w0 * dot5(Dy, ey);
    const bool left = q.j <= 2;
    float dF = (left ? p.beta : -(1.0f - p.beta)) * dw0;
    for (int r = 0; r < 2; ++r) {
        if (r >= q.nroot) break;
        float Px[5], Dx[5], ex[5];
        pis_d(R, q.x[r], Px, Dx);
        kernel_coeffs(R, Px, ex);
        const float w = fdiv_(1.0f, dot5(Px, ex));
        const float K1xy = dot5(Dx, ey);
        if (!isfinite(w) || w == 0.0f || K1xy == 0.0f) continue;
        const float rho = fdiv_(dot5(Dx, ex), K1xy);
        dF = fmaf(left ? 2.0f : -2.0f, w * w * rho * dot5(Dy, ex), dF);
    }
    return dF;
}

// Segment edges in eta: the Gauss nodes mapped from standardised y' to
// eta = (y + 1) / 2, y = c + y' / inv_s, clipped to [0, 1] (ascending).
MB_HD void table_edges(const Recon& R, float e[4]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float y = R.c + fdiv_(R.z[k], R.inv_s);
        e[k] = fminf(fmaxf(0.5f * (y + 1.0f), 0.0f), 1.0f);
    }
}

// Knot i of segment s of a pixel: (tau, dtau/deta).  The segment's end knots
// are evaluated a few ulps inside it, so that their derivative is the one of
// the segment's side of a node.
MB_HD float2 table_knot(const Params& p, const Recon& R, const float e[4], int s, int i, int M) {
    if (R.m0 <= 0.0f) return make_float2(0.0f, 0.0f);
    const float a = s > 0 ? e[s - 1] : 0.0f, b = s < 4 ? e[s] : 1.0f;
    float eta = fmaf(b - a, tab_knot_u(i, M), a);
    const float nudge = 4e-7f;
    if (i == 0) eta = fminf(eta + nudge, b);
    if (i == M) eta = fmaxf(eta - nudge, a);
    QueryRec q;
    const float tau = bound_query<true>(R, p.beta, fmaf(2.0f, eta, -1.0f), &q);
    const float d = bound_dF_dy(p, R, q) * R.m0 * R.inv_s * 2.0f;   // dy'/deta = 2 inv_s
    return make_float2(tau, isfinite(d) ? d : 0.0f);
}

// A pixel's table as seen by the quadrature pass: knots [s][i] at
// tab[(s (M+1) + i) npix + pix] (planar over pixels, so that the lanes of a
// warp, which query neighbouring pixels at similar depths, read neighbouring
// entries).
struct TabPixel {
    float m0;
    float e[4];
    const float2* __restrict__ tab;
    int64_t pix, npix;
    int M;
};

MB_HD float table_depth(const TabPixel& T, float gq) {
    if (T.m0 <= 0.0f) return 0.0f;
    const float eta = fminf(fmaxf(gq, 0.0f), 1.0f);
    const int s = (eta > T.e[0]) + (eta > T.e[1]) + (eta > T.e[2]) + (eta > T.e[3]);
    const float a = s > 0 ? T.e[s - 1] : 0.0f, b = s < 4 ? T.e[s] : 1.0f;
    const float w = b - a;
    if (!(w > 0.0f)) return T.tab[(size_t)(s * (T.M + 1)) * T.npix + T.pix].x;
    // knot interval of the segment coordinate v: i = floor(M acos(1 - 2v) / pi),
    // corrected by one where rounding put v outside [u_i, u_{i+1})
    const float v = fminf(fmaxf(fdiv_(eta - a, w), 0.0f), 1.0f);
    int i = (int)(acosf(fmaf(-2.0f, v, 1.0f)) * ((float)T.M * 0.318309886183790672f));
    i = i < 0 ? 0 : (i > T.M - 1 ? T.M - 1 : i);
    float u0 = tab_knot_u(i, T.M), u1 = tab_knot_u(i + 1, T.M);
    if (i > 0 && v < u0) {
        --i;
        u1 = u0;
        u0 = tab_knot_u(i, T.M);
    } else if (i < T.M - 1 && v >= u1) {
        ++i;
        u0 = u1;
        u1 = tab_knot_u(i + 1, T.M);
    }
    const float hu = u1 - u0;
    const float t = fdiv_(v - u0, hu), h = w * hu;
    const float2 k0 = T.tab[(size_t)(s * (T.M + 1) + i) * T.npix + T.pix];
    const float2 k1 = T.tab[(size_t)(s * (T.M + 1) + i + 1) * T.npix + T.pix];
    const float t2 = t * t, omt = 1.0f - t;
    const float h00 = (1.0f + 2.0f * t) * omt * omt, h10 = t * omt * omt;
    const float h01 = t2 * (3.0f - 2.0f * t), h11 = t2 * (t - 1.0f);
    return fmaf(h00, k0.x, fmaf(h10 * h, k0.y, fmaf(h01, k1.x, h11 * h * k1.y)));
}

template <bool SAVE, int QB = 16>
MB_HD float sample_depth(const Params& p, const TabPixel& T, float gq, char*) {
    return table_depth(T, gq);
}

}  // namespace mb
