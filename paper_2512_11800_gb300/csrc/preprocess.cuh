// Per-(view, Gaussian) preprocessing arithmetic (FP64), shared by the
// preprocess kernel; see preprocess.cu for the method description.
// MB_PRE_T selects the arithmetic type; only the host-emulation stability
// test builds it with float (to measure what FP32 would lose).
#pragma once
#include "common.cuh"

#ifndef MB_PRE_T
#define MB_PRE_T double
#endif

namespace mb {

typedef MB_PRE_T pre_t;


MB_HD void cross3(const pre_t a[3], const pre_t b[3], pre_t c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
MB_HD pre_t dot3(const pre_t a[3], const pre_t b[3]) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// SH colour in FP32 (no cancellation to guard against; FP64 is slow on GB300).
MB_HD float sh_color_channel(const Params& p, const float* __restrict__ sh, int K, int c, float x, float y, float z) {
    const float* f = sh + c;  // stride 3
    float acc = p.sh_c[0] * f[0];
    if (K > 1) {
        acc += p.sh_c[1] * (-y) * f[3 * 1] + p.sh_c[2] * z * f[3 * 2] + p.sh_c[3] * (-x) * f[3 * 3];
    }
    if (K > 4) {
        const float xx = x * x, yy = y * y, zz = z * z;
        acc += p.sh_c[4] * (x * y) * f[3 * 4] + p.sh_c[5] * (-y * z) * f[3 * 5] +
               p.sh_c[6] * (2 * zz - xx - yy) * f[3 * 6] + p.sh_c[7] * (-x * z) * f[3 * 7] +
               p.sh_c[8] * (xx - yy) * f[3 * 8];
        if (K > 9) {
            acc += p.sh_c[9] * (-y * (3 * xx - yy)) * f[3 * 9] + p.sh_c[10] * (x * y * z) * f[3 * 10] +
                   p.sh_c[11] * (-y * (4 * zz - xx - yy)) * f[3 * 11] +
                   p.sh_c[12] * (z * (2 * zz - 3 * xx - 3 * yy)) * f[3 * 12] +
                   p.sh_c[13] * (-x * (4 * zz - xx - yy)) * f[3 * 13] + p.sh_c[14] * (z * (xx - yy)) * f[3 * 14] +
                   p.sh_c[15] * (-x * (xx - 3 * yy)) * f[3 * 15];
        }
    }
    acc += 0.5f;
    return acc > 0.0f ? acc : 0.0f;
}

MB_HD void preprocess_one(const Params& p, const ViewDesc& V, const float* __restrict__ means,
                          const float* __restrict__ scales, const float* __restrict__ quats,
                          const float* __restrict__ weights, const float* __restrict__ sh, int64_t i, int sh_deg,
                          float* __restrict__ r, int* count, bool* bad_input) {
    int* ri = reinterpret_cast<int*>(r);
    *bad_input = false;

    pre_t mu[3], s[3], q[4], w;
    bool finite = true;
    for (int k = 0; k < 3; ++k) {
        mu[k] = means[3 * i + k];
        s[k] = scales[3 * i + k];
        finite &= isfinite(mu[k]) && isfinite(s[k]) && s[k] > 0.0;
    }
    for (int k = 0; k < 4; ++k) {
        q[k] = quats[4 * i + k];
        finite &= isfinite(q[k]);
    }
    w = weights[i];
    finite &= isfinite(w) && w > 0.0;
    const pre_t qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    finite &= qn > 0.0;

    bool visible = finite;
    bool full = false;
    int x0 = 1, y0 = 1, x1 = 0, y1 = 0;
    pre_t Rg[3][3], muc[3], A[3][3];
    if (!finite && !(w == 0.0)) *bad_input = true;
    if (visible) {
        const pre_t qw = q[0] / qn, qx = q[1] / qn, qy = q[2] / qn, qz = q[3] / qn;
        const pre_t Rq[3][3] = {{1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy)},
                                 {2 * (qx * qy + qw * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx)},
                                 {2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), 1 - 2 * (qx * qx + qy * qy)}};
        for (int a = 0; a < 3; ++a) {
            muc[a] = (pre_t)V.R[3 * a] * mu[0] + (pre_t)V.R[3 * a + 1] * mu[1] + (pre_t)V.R[3 * a + 2] * mu[2] +
                     (pre_t)V.t[a];
            for (int b = 0; b < 3; ++b)
                Rg[a][b] = (pre_t)V.R[3 * a] * Rq[0][b] + (pre_t)V.R[3 * a + 1] * Rq[1][b] +
                           (pre_t)V.R[3 * a + 2] * Rq[2][b];
        }
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                A[a][b] = Rg[a][0] * Rg[b][0] / (s[0] * s[0]) + Rg[a][1] * Rg[b][1] / (s[1] * s[1]) +
                          Rg[a][2] * Rg[b][2] / (s[2] * s[2]);
        // frustum culling with the bounding sphere (Sec. 3.3)
        const pre_t rad = (pre_t)p.r_mult * fmax(s[0], fmax(s[1], s[2]));
        const pre_t W = V.width, H = V.height;
        const pre_t pl[4][3] = {{V.fx, 0.0, V.cx}, {-V.fx, 0.0, W - V.cx}, {0.0, V.fy, V.cy}, {0.0, -V.fy, H - V.cy}};
        for (int k = 0; k < 4; ++k) {
            const pre_t nrm = sqrt(pl[k][0] * pl[k][0] + pl[k][1] * pl[k][1] + pl[k][2] * pl[k][2]);
            if ((pl[k][0] * muc[0] + pl[k][1] * muc[1] + pl[k][2] * muc[2]) / nrm < -rad) visible = false;
        }
        const pre_t dist = sqrt(dot3(muc, muc));
        if (dist + rad < (pre_t)p.t_near) visible = false;
    }
    if (visible) {
        // confidence-interval proxy (Eq. 17-21): camera at the origin
        pre_t u[3] = {muc[0], muc[1], muc[2]};
        const pre_t un = sqrt(dot3(u, u));
        for (int k = 0; k < 3; ++k) u[k] /= un;
        pre_t Au[3], Amu[3];
        for (int a = 0; a < 3; ++a) {
            Au[a] = A[a][0] * u[0] + A[a][1] * u[1] + A[a][2] * u[2];
            Amu[a] = A[a][0] * muc[0] + A[a][1] * muc[1] + A[a][2] * muc[2];
        }
        const pre_t uAu = dot3(u, Au);
        const pre_t muAmu = dot3(muc, Amu);
        const pre_t C = (-log1p(-(pre_t)p.conf_c) * sqrt(uAu)) / sqrt(2.0 * 3.14159265358979323846);
        if (w <= C) {
            visible = false;  // w-hat <= w <= C everywhere: below the confidence level
        } else {
            const pre_t kap = 2.0 * (log(C) - log(w)) + muAmu;
            const pre_t fxd = V.fx, fyd = V.fy, cxd = V.cx, cyd = V.cy;
            const pre_t Ki[3][3] = {{1.0 / fxd, 0.0, -cxd / fxd}, {0.0, 1.0 / fyd, -cyd / fyd}, {0.0, 0.0, 1.0}};
            pre_t mvec[3], M3[3][3], AK[3][3];
            for (int a = 0; a < 3; ++a) mvec[a] = Ki[0][a] * Amu[0] + Ki[1][a] * Amu[1] + Ki[2][a] * Amu[2];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) AK[a][b] = A[a][0] * Ki[0][b] + A[a][1] * Ki[1][b] + A[a][2] * Ki[2][b];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) M3[a][b] = Ki[0][a] * AK[0][b] + Ki[1][a] * AK[1][b] + Ki[2][a] * AK[2][b];
            pre_t Wc[3][3];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) Wc[a][b] = mvec[a] * mvec[b] - kap * M3[a][b];
            const pre_t det = Wc[0][0] * Wc[1][1] - Wc[0][1] * Wc[1][0];
            const pre_t i00 = Wc[1][1] / det, i01 = -Wc[0][1] / det, i10 = -Wc[1][0] / det, i11 = Wc[0][0] / det;
            const pre_t m2x = -(i00 * Wc[0][2] + i01 * Wc[1][2]);
            const pre_t m2y = -(i10 * Wc[0][2] + i11 * Wc[1][2]);
            const pre_t scl = m2x * (Wc[0][0] * m2x + Wc[0][1] * m2y) + m2y * (Wc[1][0] * m2x + Wc[1][1] * m2y) -
                               Wc[2][2];
            const pre_t s00 = scl * i00, s11 = scl * i11, s01 = scl * i01, s10 = scl * i10;
            const bool negdef = Wc[0][0] < 0.0 && det > 0.0;
            const bool posdef = s00 > 0.0 && s11 > 0.0 && s00 * s11 - s01 * s10 > 0.0;
            const bool valid = muAmu > kap && negdef && posdef && muc[2] > 0.0 && isfinite(s00) && isfinite(s11) &&
                               isfinite(m2x) && isfinite(m2y);
            if (valid) {
                const pre_t hx = sqrt(s00), hy = sqrt(s11);
                const pre_t big = 1e9;
                pre_t fx0 = ceil(m2x - hx - 0.5), fx1 = floor(m2x + hx - 0.5);
                pre_t fy0 = ceil(m2y - hy - 0.5), fy1 = floor(m2y + hy - 0.5);
                fx0 = fmin(fmax(fx0, -big), big); fx1 = fmin(fmax(fx1, -big), big);
                fy0 = fmin(fmax(fy0, -big), big); fy1 = fmin(fmax(fy1, -big), big);
                x0 = (int)fmax(fx0, 0.0); y0 = (int)fmax(fy0, 0.0);
                x1 = (int)fmin(fx1, (pre_t)(V.width - 1)); y1 = (int)fmin(fy1, (pre_t)(V.height - 1));
            } else {
                full = true;
                x0 = 0; y0 = 0; x1 = V.width - 1; y1 = V.height - 1;
            }
        }
    }
    if (visible && (x0 > x1 || y0 > y1)) visible = false;
    if (!visible) {
        x0 = 1; y0 = 1; x1 = 0; y1 = 0;
        for (int k = 0; k < REC; ++k) r[k] = 0.0f;
        ri[R_RECT + 0] = x0; ri[R_RECT + 1] = y0; ri[R_RECT + 2] = x1; ri[R_RECT + 3] = y1;
        ri[R_FLAGS] = 0;
        *count = 0;
        return;
    }
    // anchor: pixel centre nearest to the projected mean, inside the rectangle
    pre_t ax, ay;
    if (!full && muc[2] > 0.0) {
        ax = floor(V.fx * muc[0] / muc[2] + V.cx) + 0.5;
        ay = floor(V.fy * muc[1] / muc[2] + V.cy) + 0.5;
        ax = fmin(fmax(ax, x0 + 0.5), x1 + 0.5);
        ay = fmin(fmax(ay, y0 + 0.5), y1 + 0.5);
    } else {
        ax = floor(0.5 * (x0 + x1)) + 0.5;
        ay = floor(0.5 * (y0 + y1)) + 0.5;
    }
    // M = S^-1 Rg^T: camera space -> normalised Gaussian frame
    pre_t M[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) M[a][b] = Rg[b][a] / s[a];
    const pre_t da[3] = {(ax - V.cx) / V.fx, (ay - V.cy) / V.fy, 1.0};
    pre_t ga[3], mx[3], my[3], og[3];
    for (int a = 0; a < 3; ++a) {
        ga[a] = M[a][0] * da[0] + M[a][1] * da[1] + M[a][2];
        mx[a] = M[a][0] / V.fx;
        my[a] = M[a][1] / V.fy;
        og[a] = -(M[a][0] * muc[0] + M[a][1] * muc[1] + M[a][2] * muc[2]);
    }
    pre_t c0[3], cx[3], cy[3];
    cross3(og, ga, c0);
    cross3(og, mx, cx);
    cross3(og, my, cy);
    for (int k = 0; k < 3; ++k) {
        r[R_C0 + k] = (float)c0[k];
        r[R_CX + k] = (float)cx[k];
        r[R_CY + k] = (float)cy[k];
    }
    for (int k = 0; k < 3; ++k) {
        r[R_GA + k] = (float)ga[k];
        r[R_MX + k] = (float)mx[k];
        r[R_MY + k] = (float)my[k];
    }
    r[R_O0] = (float)dot3(og, ga);
    r[R_OX] = (float)dot3(og, mx);
    r[R_OY] = (float)dot3(og, my);
    r[R_LNW] = (float)log(w);
    // SH colour at the world-space direction from the camera centre to the mean
    pre_t eye[3];
    for (int a = 0; a < 3; ++a) eye[a] = -((pre_t)V.R[a] * V.t[0] + (pre_t)V.R[3 + a] * V.t[1] + (pre_t)V.R[6 + a] * V.t[2]);
    pre_t dx = mu[0] - eye[0], dy = mu[1] - eye[1], dz = mu[2] - eye[2];
    const pre_t dn = sqrt(dx * dx + dy * dy + dz * dz);
    dx /= dn; dy /= dn; dz /= dn;
    const int K = (sh_deg + 1) * (sh_deg + 1);
    for (int c = 0; c < 3; ++c) r[R_RGB + c] = sh_color_channel(p, sh + i * 3 * K, K, c, (float)dx, (float)dy, (float)dz);
    r[R_AX] = (float)ax;
    r[R_AY] = (float)ay;
    ri[R_RECT + 0] = x0; ri[R_RECT + 1] = y0; ri[R_RECT + 2] = x1; ri[R_RECT + 3] = y1;
    ri[R_FLAGS] = 1 | (full ? 2 : 0);
    const int tx0 = x0 / V.tile_w, tx1 = x1 / V.tile_w, ty0 = y0 / V.tile_h, ty1 = y1 / V.tile_h;
    *count = (tx1 - tx0 + 1) * (ty1 - ty0 + 1);
}

}  // namespace mb
