// Backward kernels: quadrature/bound adjoint pass, moment adjoint pass,
// preprocessing adjoint.  The rescaling derivative (Eq. 15) is folded into
// the passes as in the paper's two-pass adjoint (Sec. 3.3, App. C "Adjoint
// rendering"); the proxy rectangles and the culling are constants.
// Per-Gaussian sums over pixels use a warp reduce-scatter per record, then
// one global atomicAdd per (warp footprint, record, field) in pass 1 and per
// (tile, record, field) in pass 2.  Work comes from the schedule of tile.cuh
// like the forward passes.
#include "backward.cuh"
#include "moments.cuh"
#include "preprocess.cuh"
#include "tile.cuh"

namespace mb {

__device__ __forceinline__ float load_m0(const Params& p, const void* moments, int64_t pix) {
    return reinterpret_cast<const float*>(moments)[pix];   // m0 is the first plane in every storage format
}

constexpr int GSTRIDE = 28;   // floats per record gradient (NGRAD padded)

// Per-warp scratch of the adjoint passes: the staged records of one chunk
// (tile.cuh) and their compact per-record sums.
constexpr int WARP_BWD_FLOATS = WARP_STAGE_FLOATS + 32 * NK_QUAD;

// Adds a chunk's per-record gradients (fields 0..nf-1, expanded from the
// compact sums s_sum[k][nk] of the warp's m staged records) to the record
// gradients: one atomicAdd per (footprint, record, non-zero field).
__device__ __forceinline__ void flush_chunk(const float* s_buf, const float* s_sum, int m, int nk, int nf,
                                            int64_t rec_base, float* __restrict__ grec) {
    const int* s_ids = reinterpret_cast<const int*>(s_buf + 32 * REC);
    for (int q = threadIdx.x & 31; q < m * nf; q += 32) {
        const int k = q / nf, f = q - k * nf;
        const float v = expand_geometry(s_buf + k * REC, s_sum + k * nk, f);
        if (v != 0.0f) atomicAdd(&grec[(rec_base + s_ids[k]) * GSTRIDE + f], v);
    }
}

// Per-pixel bound state of the adjoint passes and the pixel's moment adjoint
// from its summed query adjoints.
__device__ __forceinline__ void load_bound(const float* __restrict__ recon, int64_t npix, int64_t pix, Recon& R) {
    R = load_recon(recon, npix, pix);
}
__device__ __forceinline__ void load_bound(const float* __restrict__ recon, int64_t npix, int64_t pix, TrigRecon& T) {
    T = load_trig_recon(recon, npix, pix);
}
__device__ __forceinline__ void finish_pixel(const Params& p, const Recon& R, const float B[NB], float gm0,
                                             const void*, int64_t, int64_t, float psi[NPOLY]) {
    phi_monomials(R, B, psi);
    finish_moment_adjoint(p, R, gm0, psi);
}
__device__ __forceinline__ void finish_pixel(const Params& p, const TrigRecon&, const float A[NTRIG_ADJ], float gm0,
                                             const void* moments, int64_t npix, int64_t pix, float psi[NPOLY]) {
    float I[NMOM];
    load_moments(p, moments, npix, pix, I);
    trig_finish_adjoint(p, I, A, gm0, psi);
}

// ---------------------------------------------------------------- pass 1
// Per pair: the quadrature, penalty and bound-query adjoint.  The direct
// derivatives go through the record geometry to the per-record gradients;
// the bound derivatives sum per pixel (power moments: the polynomial Phi;
// trigonometric moments: the Verblunsky-coefficient adjoints), written out
// as the pixel's moment adjoint psi.  Warp-level units as in the forward passes: each
// warp walks its footprint's records, reduces every record's compact sums
// over its 32 pixels and adds them to the record gradients per chunk.
// SAVED: only the pixels whose bound queries the quadrature pass kept
// (pq_off + npp <= qcap), read instead of solved; otherwise the pixels that
// kept none (all pixels when qcap == 0), whose queries are solved again.
template <int NI, bool SAVED, class RecT, int QB = 16>
__global__ void __launch_bounds__(TPB, 2)
    k_bwd_quadrature(Params p, ViewTable vt, TileSched ts, const float* __restrict__ rec,
                     const int32_t* __restrict__ ids, const int2* __restrict__ ranges, int64_t P, int64_t npix,
                     const StatusWords* sw, const float* __restrict__ recon, const void* __restrict__ moments,
                     const float* __restrict__ saved, const float* __restrict__ dL_drgb,
                     const float* __restrict__ dL_dP, const float* __restrict__ dL_dT, float* __restrict__ psi_out,
                     float* __restrict__ grec, const int* __restrict__ npp, const long long* __restrict__ pq_off,
                     const char* __restrict__ pq, int64_t qcap) {
    extern __shared__ float4 s_raw[];
    float* s_buf = reinterpret_cast<float*>(s_raw) + (threadIdx.x >> 5) * WARP_BWD_FLOATS;
    float* s_sum = s_buf + WARP_STAGE_FLOATS;          // [32][NK_QUAD] compact sums of the chunk
    const bool any = sw->n_valid != 0;
    const int nq = (NI > 0 ? NI : p.n_intervals) + 1;
    const char* q_end = SAVED ? pq + (size_t)qcap * nq * QB : nullptr;   // end of the saved queries
    const int ridx = rs_index<NK_QUAD>(threadIdx.x & 31);   // compact sum this lane reduces
    int fp, fx0, fy0;
    for (int64_t tile = next_unit(ts, true, &fp); tile >= 0; tile = next_unit(ts, false, &fp)) {
        PixelCtx c = unit_ctx(vt, ranges, P, tile, fp, &fx0, &fy0);
        long long off = 0;
        if (c.inside && qcap > 0) {
            off = pq_off[c.pix];
            c.inside = (off + npp[c.pix] <= qcap) == SAVED;   // this launch's pixels
        }
        if (!any || !__any_sync(0xffffffffu, c.inside)) c.end = c.start;
        const char* qp = nullptr;
        RecT R;
        PixelAdj pa;
        constexpr int NACC = BoundAdj<RecT>::NACC;
        float B[NACC];
#pragma unroll
        for (int k = 0; k < NACC; ++k) B[k] = 0.0f;
        if (c.inside) {
            load_bound(recon, npix, c.pix, R);
            const float S[3] = {saved[c.pix], saved[npix + c.pix], saved[2 * npix + c.pix]};
            const float O = saved[3 * npix + c.pix];
            const float g[3] = {dL_drgb[3 * c.pix], dL_drgb[3 * c.pix + 1], dL_drgb[3 * c.pix + 2]};
            const float m0 = load_m0(p, moments, c.pix);
            pa = pixel_adjoint(p, m0, S, O, g, dL_dP ? dL_dP[c.pix] : 0.0f);
            if (dL_dT) pa.gm0 -= expf(-m0) * dL_dT[c.pix];   // T_final = e^{-m0}
            if (SAVED) qp = pq + (size_t)off * nq * QB;
        }
        const float fpx = (float)c.px + 0.5f, fpy = (float)c.py + 0.5f;
        for (int pos = c.start; pos < c.end; pos += 32) {
            const int m = stage_warp_chunk(s_buf, rec, ids, c.rec_base, pos, c.end, fx0, fy0);
            for (int k = 0; k < m; ++k) {
                const float* r = s_buf + k * REC;
                const bool active = c.inside && rect_contains(r, c.px, c.py);
                if (!__any_sync(0xffffffffu, active)) {
                    if (ridx >= 0) s_sum[k * NK_QUAD + ridx] = 0.0f;
                    continue;
                }
                float acc[NK_QUAD];
#pragma unroll
                for (int f = 0; f < NK_QUAD; ++f) acc[f] = 0.0f;
                if (active) {
                    // the pixel's saved queries are contiguous in pair order: start
                    // fetching the next pair's into L2 while this one is processed
                    if (SAVED && qp + 2 * nq * QB <= q_end)
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(qp + nq * QB));
                    const float dx = fpx - r[R_AX], dy = fpy - r[R_AY];
                    const Gauss1D g = pair_gaussian(r, dx, dy, c.rlen, c.r2);
                    const float a = pa.gS[0] * r[R_RGB] + pa.gS[1] * r[R_RGB + 1] + pa.gS[2] * r[R_RGB + 2] + pa.gO;
                    const PairOut po = pair_backward<NI, SAVED, RecT, QB>(p, R, g, a, pa.gP, B, qp);
                    if (SAVED) qp += nq * QB;
                    geometry_adjoint_compact(r, dx, dy, c.rlen, g, po.g_mu, po.g_Sig, po.g_what, acc);
                    acc[K_RGB + 0] = pa.gS[0] * po.O;
                    acc[K_RGB + 1] = pa.gS[1] * po.O;
                    acc[K_RGB + 2] = pa.gS[2] * po.O;
                }
                const float v = reduce_scatter<NK_QUAD>(acc);
                if (ridx >= 0) s_sum[k * NK_QUAD + ridx] = v;
            }
            __syncwarp();
            flush_chunk(s_buf, s_sum, m, NK_QUAD, NGRAD, c.rec_base, grec);
        }
        if (c.inside) {
            float psi[NPOLY];
            finish_pixel(p, R, B, pa.gm0, moments, npix, c.pix, psi);
#pragma unroll
            for (int k = 0; k < NPOLY; ++k) psi_out[k * npix + c.pix] = psi[k];
        }
    }
}

// Adds one staged batch's per-record gradients (fields 0..nf-1, expanded from
// the compact sums s_acc[k][nk]) to the record gradients.
__device__ __forceinline__ void flush_batch(const float* s_rec, const float* s_acc, int nb, int nk, int nf,
                                            const int32_t* __restrict__ ids, int first, int64_t rec_base,
                                            float* __restrict__ grec) {
    for (int q = threadIdx.x; q < nb * nf; q += TPB) {
        const int k = q / nf, f = q - k * nf;
        const float v = expand_geometry(s_rec + k * REC, s_acc + k * nk, f);
        if (v != 0.0f) atomicAdd(&grec[(rec_base + ids[first + k]) * GSTRIDE + f], v);
    }
}

// ---------------------------------------------------------------- pass 2
// Per pair: int psi d(d mu_i) through the reverse sweep of the moment
// recurrence (TRIG: the reverse of the trigonometric moments), chained to the
// record geometry (fields before G_RGB).  One CTA
// works on one tile at a time with record batches staged for the whole CTA:
// its per-record sums are combined over the tile's 256 pixels in shared
// memory before the global atomics (one per tile, record and field), which
// measured faster than per-footprint flushes for this light pass.
#ifndef MB_BWD_MOMENTS_MIN_CTAS
#define MB_BWD_MOMENTS_MIN_CTAS 4
#endif
template <bool TRIG>
__global__ void __launch_bounds__(TPB, MB_BWD_MOMENTS_MIN_CTAS)
    k_bwd_moments(Params p, ViewTable vt, TileSched ts, const float* __restrict__ rec, const int32_t* __restrict__ ids,
                  const int2* __restrict__ ranges, int64_t P, int64_t npix, const StatusWords* sw,
                  const float* __restrict__ recon, const float* __restrict__ psi_in, float* __restrict__ grec) {
    extern __shared__ float4 s_raw[];
    __shared__ int s_slot;
    float* s_rec = reinterpret_cast<float*>(s_raw);
    float* s_acc = s_rec + REC * p.batch;             // [batch][NK_MOM] compact sums
    const bool any = sw->n_valid != 0;
    const int lane = threadIdx.x & 31;
    for (int64_t tile = next_tile(ts, &s_slot, true); tile >= 0; tile = next_tile(ts, &s_slot, false)) {
        PixelCtx c = pixel_ctx(vt, ranges, P, tile);
        if (!any) c.end = c.start;
        Recon R;                                      // only the standardisation (c, 1/s) is used
        float psi[NPOLY];
        if (c.inside) {
            if (!TRIG) {
                R.c = recon[1 * npix + c.pix];
                R.inv_s = recon[2 * npix + c.pix];
            }
#pragma unroll
            for (int k = 0; k < NPOLY; ++k) psi[k] = psi_in[k * npix + c.pix];
        }
        const int n = c.end - c.start;
        const float fpx = (float)c.px + 0.5f, fpy = (float)c.py + 0.5f;
        for (int b = 0; b * p.batch < n; ++b) {
            for (int q = threadIdx.x; q < p.batch * NK_MOM; q += TPB) s_acc[q] = 0.0f;
            const int nb = stage_batch(s_rec, rec, ids, c.rec_base, c.start, c.end, b, p.batch);
            for (int k = 0; k < nb; ++k) {
                const float* r = s_rec + k * REC;
                const bool active = c.inside && rect_contains(r, c.px, c.py);
                if (!__any_sync(0xffffffffu, active)) continue;
                float acc[NK_MOM];
#pragma unroll
                for (int f = 0; f < NK_MOM; ++f) acc[f] = 0.0f;
                if (active) {
                    const float dx = fpx - r[R_AX], dy = fpy - r[R_AY];
                    const Gauss1D g = pair_gaussian(r, dx, dy, c.rlen, c.r2);
                    float g_mu = 0.0f, g_Sig = 0.0f, g_what = 0.0f;
                    if (TRIG) trig_moment_adjoint(p, g, psi, &g_mu, &g_Sig, &g_what);
                    else moment_adjoint(p, R, g, psi, &g_mu, &g_Sig, &g_what);
                    geometry_adjoint_compact(r, dx, dy, c.rlen, g, g_mu, g_Sig, g_what, acc);
                }
                const float v = reduce_scatter16(acc);
                if (lane < NK_MOM && v != 0.0f) atomicAdd(&s_acc[k * NK_MOM + lane], v);
            }
            __syncthreads();
            flush_batch(s_rec, s_acc, nb, NK_MOM, G_RGB, ids, c.start + b * p.batch, c.rec_base, grec);
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------- preprocessing adjoint
// float or double 3-vector helpers of the preprocessing adjoint
template <typename T>
MB_HD void cross3t(const T a[3], const T b[3], T c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
template <typename T>
MB_HD T dot3t(const T a[3], const T b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

template <typename T>
MB_HD void sh_grad_basis(const Params& p, T x, T y, T z, T Y[16], T dY[16][3]) {
    const T xx = x * x, yy = y * y, zz = z * z;
    const float* c = p.sh_c;
    Y[0] = c[0]; dY[0][0] = dY[0][1] = dY[0][2] = 0.0;
    Y[1] = -c[1] * y; dY[1][0] = 0; dY[1][1] = -c[1]; dY[1][2] = 0;
    Y[2] = c[2] * z; dY[2][0] = 0; dY[2][1] = 0; dY[2][2] = c[2];
    Y[3] = -c[3] * x; dY[3][0] = -c[3]; dY[3][1] = 0; dY[3][2] = 0;
    Y[4] = c[4] * x * y; dY[4][0] = c[4] * y; dY[4][1] = c[4] * x; dY[4][2] = 0;
    Y[5] = -c[5] * y * z; dY[5][0] = 0; dY[5][1] = -c[5] * z; dY[5][2] = -c[5] * y;
    Y[6] = c[6] * (2 * zz - xx - yy); dY[6][0] = -2 * c[6] * x; dY[6][1] = -2 * c[6] * y; dY[6][2] = 4 * c[6] * z;
    Y[7] = -c[7] * x * z; dY[7][0] = -c[7] * z; dY[7][1] = 0; dY[7][2] = -c[7] * x;
    Y[8] = c[8] * (xx - yy); dY[8][0] = 2 * c[8] * x; dY[8][1] = -2 * c[8] * y; dY[8][2] = 0;
    Y[9] = -c[9] * y * (3 * xx - yy); dY[9][0] = -6 * c[9] * x * y; dY[9][1] = -c[9] * (3 * xx - 3 * yy); dY[9][2] = 0;
    Y[10] = c[10] * x * y * z; dY[10][0] = c[10] * y * z; dY[10][1] = c[10] * x * z; dY[10][2] = c[10] * x * y;
    Y[11] = -c[11] * y * (4 * zz - xx - yy);
    dY[11][0] = 2 * c[11] * x * y; dY[11][1] = -c[11] * (4 * zz - xx - 3 * yy); dY[11][2] = -8 * c[11] * y * z;
    Y[12] = c[12] * z * (2 * zz - 3 * xx - 3 * yy);
    dY[12][0] = -6 * c[12] * x * z; dY[12][1] = -6 * c[12] * y * z; dY[12][2] = c[12] * (6 * zz - 3 * xx - 3 * yy);
    Y[13] = -c[13] * x * (4 * zz - xx - yy);
    dY[13][0] = -c[13] * (4 * zz - 3 * xx - yy); dY[13][1] = 2 * c[13] * x * y; dY[13][2] = -8 * c[13] * x * z;
    Y[14] = c[14] * z * (xx - yy); dY[14][0] = 2 * c[14] * x * z; dY[14][1] = -2 * c[14] * y * z; dY[14][2] = c[14] * (xx - yy);
    Y[15] = -c[15] * x * (xx - 3 * yy); dY[15][0] = -c[15] * (3 * xx - 3 * yy); dY[15][1] = 6 * c[15] * x * y; dY[15][2] = 0;
}

template <typename T>
MB_HD void preprocess_bwd_one(const Params& p, const ViewTable& vt, const float* __restrict__ means,
                              const float* __restrict__ scales, const float* __restrict__ quats,
                              const float* __restrict__ weights, const float* __restrict__ sh, int64_t P, int sh_deg,
                              const float* __restrict__ rec, const float* __restrict__ grec, int64_t i,
                              float* __restrict__ d_means, float* __restrict__ d_scales, float* __restrict__ d_quats,
                              float* __restrict__ d_weights, float* __restrict__ d_sh) {
    const int K = (sh_deg + 1) * (sh_deg + 1);
    T gmu[3] = {0, 0, 0}, gs[3] = {0, 0, 0}, gq[4] = {0, 0, 0, 0}, gw = 0;
    T gsh[48];
    for (int k = 0; k < 3 * K; ++k) gsh[k] = 0.0;
    T mu[3], s[3], q[4];
    for (int k = 0; k < 3; ++k) { mu[k] = means[3 * i + k]; s[k] = scales[3 * i + k]; }
    for (int k = 0; k < 4; ++k) q[k] = quats[4 * i + k];
    const T w = weights[i];
    const T qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    const T qw = q[0] / qn, qx = q[1] / qn, qy = q[2] / qn, qz = q[3] / qn;
    const T Rq[3][3] = {{1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy)},
                             {2 * (qx * qy + qw * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx)},
                             {2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), 1 - 2 * (qx * qx + qy * qy)}};
    T gRq[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int v = 0; v < vt.n_views; ++v) {
        const int64_t idx = (int64_t)v * P + i;
        const float* r = rec + idx * REC;
        const int flags = reinterpret_cast<const int*>(r)[R_FLAGS];
        if (!(flags & 1)) continue;
        const float* G = grec + idx * GSTRIDE;
        const ViewDesc& V = vt.v[v];
        T Rv[3][3], muc[3], Rg[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) Rv[a][b] = V.R[3 * a + b];
        for (int a = 0; a < 3; ++a) {
            muc[a] = Rv[a][0] * mu[0] + Rv[a][1] * mu[1] + Rv[a][2] * mu[2] + (T)V.t[a];
            for (int b = 0; b < 3; ++b) Rg[a][b] = Rv[a][0] * Rq[0][b] + Rv[a][1] * Rq[1][b] + Rv[a][2] * Rq[2][b];
        }
        T M[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) M[a][b] = Rg[b][a] / s[a];
        const T fx = V.fx, fy = V.fy, cx = V.cx, cy = V.cy;
        const T da[3] = {((T)r[R_AX] - cx) / fx, ((T)r[R_AY] - cy) / fy, 1.0};
        T ga[3], mx[3], my[3], og[3];
        for (int a = 0; a < 3; ++a) {
            ga[a] = M[a][0] * da[0] + M[a][1] * da[1] + M[a][2];
            mx[a] = M[a][0] / fx;
            my[a] = M[a][1] / fy;
            og[a] = -(M[a][0] * muc[0] + M[a][1] * muc[1] + M[a][2] * muc[2]);
        }
        T Gc0[3], Gcx[3], Gcy[3];
        for (int k = 0; k < 3; ++k) { Gc0[k] = G[G_C0 + k]; Gcx[k] = G[G_CX + k]; Gcy[k] = G[G_CY + k]; }
        const T Go0 = G[G_O], Gox = G[G_O + 1], Goy = G[G_O + 2];
        // c = a x b: dL/da = b x G, dL/db = G x a
        T Gog[3], Gga[3], Gmx[3], Gmy[3], t1[3], t2[3], t3[3];
        cross3t(ga, Gc0, t1); cross3t(mx, Gcx, t2); cross3t(my, Gcy, t3);
        for (int k = 0; k < 3; ++k) Gog[k] = t1[k] + t2[k] + t3[k] + Go0 * ga[k] + Gox * mx[k] + Goy * my[k];
        cross3t(Gc0, og, t1);
        for (int k = 0; k < 3; ++k) Gga[k] = t1[k] + (T)G[G_GA + k] + Go0 * og[k];
        cross3t(Gcx, og, t1);
        for (int k = 0; k < 3; ++k) Gmx[k] = t1[k] + (T)G[G_MX + k] + Gox * og[k];
        cross3t(Gcy, og, t1);
        for (int k = 0; k < 3; ++k) Gmy[k] = t1[k] + (T)G[G_MY + k] + Goy * og[k];
        T GM[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                GM[a][b] = -Gog[a] * muc[b] + Gga[a] * da[b] + (b == 0 ? Gmx[a] / fx : 0.0) + (b == 1 ? Gmy[a] / fy : 0.0);
        T Gmuc[3];
        for (int b = 0; b < 3; ++b) Gmuc[b] = -(M[0][b] * Gog[0] + M[1][b] * Gog[1] + M[2][b] * Gog[2]);
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) gs[a] -= GM[a][b] * Rg[b][a] / (s[a] * s[a]);
        T GRg[3][3];
        for (int b = 0; b < 3; ++b)
            for (int a = 0; a < 3; ++a) GRg[b][a] = GM[a][b] / s[a];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) gRq[a][b] += Rv[0][a] * GRg[0][b] + Rv[1][a] * GRg[1][b] + Rv[2][a] * GRg[2][b];
        for (int b = 0; b < 3; ++b) gmu[b] += Rv[0][b] * Gmuc[0] + Rv[1][b] * Gmuc[1] + Rv[2][b] * Gmuc[2];
        gw += (T)G[G_LNW] / w;
        // SH colour at normalize(mu - eye)
        T eye[3];
        for (int a = 0; a < 3; ++a) eye[a] = -(Rv[0][a] * V.t[0] + Rv[1][a] * V.t[1] + Rv[2][a] * V.t[2]);
        T dv[3] = {mu[0] - eye[0], mu[1] - eye[1], mu[2] - eye[2]};
        const T dn = sqrt(dot3t(dv, dv));
        const T d[3] = {dv[0] / dn, dv[1] / dn, dv[2] / dn};
        T Y[16], dY[16][3];
        sh_grad_basis<T>(p, d[0], d[1], d[2], Y, dY);
        T gd[3] = {0, 0, 0};
        for (int ch = 0; ch < 3; ++ch) {
            if (!(r[R_RGB + ch] > 0.0f)) continue;   // colour clamped at 0 in the forward record
            const T gc = G[G_RGB + ch];
            for (int k = 0; k < K; ++k) {
                gsh[k * 3 + ch] += gc * Y[k];
                const T f = sh[(i * K + k) * 3 + ch];
                for (int a = 0; a < 3; ++a) gd[a] += gc * f * dY[k][a];
            }
        }
        const T dg = dot3t(d, gd);
        for (int a = 0; a < 3; ++a) gmu[a] += (gd[a] - d[a] * dg) / dn;
    }
    // R(q-hat) and the normalisation q-hat = q / |q|
    T gqh[4];
    gqh[0] = 2 * (-qz * gRq[0][1] + qy * gRq[0][2] + qz * gRq[1][0] - qx * gRq[1][2] - qy * gRq[2][0] + qx * gRq[2][1]);
    gqh[1] = 2 * (qy * gRq[0][1] + qz * gRq[0][2] + qy * gRq[1][0] - 2 * qx * gRq[1][1] - qw * gRq[1][2] +
                  qz * gRq[2][0] + qw * gRq[2][1] - 2 * qx * gRq[2][2]);
    gqh[2] = 2 * (-2 * qy * gRq[0][0] + qx * gRq[0][1] + qw * gRq[0][2] + qx * gRq[1][0] + qz * gRq[1][2] -
                  qw * gRq[2][0] + qz * gRq[2][1] - 2 * qy * gRq[2][2]);
    gqh[3] = 2 * (-2 * qz * gRq[0][0] - qw * gRq[0][1] + qx * gRq[0][2] + qw * gRq[1][0] - 2 * qz * gRq[1][1] +
                  qy * gRq[1][2] + qx * gRq[2][0] + qy * gRq[2][1]);
    const T qh[4] = {qw, qx, qy, qz};
    const T pr = qh[0] * gqh[0] + qh[1] * gqh[1] + qh[2] * gqh[2] + qh[3] * gqh[3];
    for (int k = 0; k < 4; ++k) gq[k] = (gqh[k] - qh[k] * pr) / qn;
    for (int k = 0; k < 3; ++k) {
        d_means[3 * i + k] = (float)gmu[k];
        d_scales[3 * i + k] = (float)gs[k];
    }
    for (int k = 0; k < 4; ++k) d_quats[4 * i + k] = (float)gq[k];
    d_weights[i] = (float)gw;
    for (int k = 0; k < 3 * K; ++k) d_sh[i * 3 * K + k] = (float)gsh[k];
}

__global__ void k_preprocess_bwd(Params p, ViewTable vt, const float* __restrict__ means,
                                 const float* __restrict__ scales, const float* __restrict__ quats,
                                 const float* __restrict__ weights, const float* __restrict__ sh, int64_t P,
                                 int sh_deg, const float* __restrict__ rec, const float* __restrict__ grec,
                                 float* __restrict__ d_means, float* __restrict__ d_scales,
                                 float* __restrict__ d_quats, float* __restrict__ d_weights, float* __restrict__ d_sh) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    // FP32: the chain rule needs no more (gradients to ~1e-6 relative); the
    // forward keeps FP64 for the cancelling record coefficients
    preprocess_bwd_one<float>(p, vt, means, scales, quats, weights, sh, P, sh_deg, rec, grec, i, d_means, d_scales,
                              d_quats, d_weights, d_sh);
}

// Pass 1 (zeroes the record gradients first).
int launch_backward_quadrature(const Params& p, const ViewTable& vt, const Layout& L, char* ws,
                               const float* dL_drgb, const float* dL_dP, const float* dL_dT, cudaStream_t st) {
    float* grec = reinterpret_cast<float*>(ws + L.grec);
    if (cudaMemsetAsync(grec, 0, sizeof(float) * GSTRIDE * (size_t)L.VP, st) != cudaSuccess) return MB3DGS_ERR_CUDA;
    if (L.n_tiles == 0) return MB3DGS_OK;
    const size_t smem = sizeof(float) * WARP_BWD_FLOATS * WARPS;
    const bool kept = L.qcap > 0;
    // with kept queries: one launch for the pixels that kept theirs, one for
    // the rest (those beyond the capacity; the launch exits early when none)
    for (int pass = kept ? 0 : 1; pass < 2; ++pass) {
        const bool saved_q = pass == 0;
        auto k1 = p.basis == MB3DGS_BASIS_TRIG
                      ? (saved_q ? (p.n_intervals == 3   ? k_bwd_quadrature<3, true, TrigRecon>
                                    : p.n_intervals == 5 ? k_bwd_quadrature<5, true, TrigRecon>
                                                         : k_bwd_quadrature<0, true, TrigRecon>)
                                 : (p.n_intervals == 3   ? k_bwd_quadrature<3, false, TrigRecon>
                                    : p.n_intervals == 5 ? k_bwd_quadrature<5, false, TrigRecon>
                                                         : k_bwd_quadrature<0, false, TrigRecon>))
                  : saved_q && p.qbytes == 8
                      ? (p.n_intervals == 3 ? k_bwd_quadrature<3, true, Recon, 8> : k_bwd_quadrature<0, true, Recon, 8>)
                  : p.n_intervals == 3 ? (saved_q ? k_bwd_quadrature<3, true, Recon> : k_bwd_quadrature<3, false, Recon>)
                                       : (saved_q ? k_bwd_quadrature<0, true, Recon> : k_bwd_quadrature<0, false, Recon>);
        if (!allow_dynamic_smem((const void*)k1, smem)) return MB3DGS_ERR_CUDA;
        const TileLaunch t1 = tile_launch(p, L, ws, Q_BWD_QUAD, (const void*)k1, smem, st);
        count_launch();
        k1<<<t1.grid, TPB, smem, st>>>(
            p, vt, t1.ts, reinterpret_cast<const float*>(ws + L.rec),
            reinterpret_cast<const int32_t*>(ws + L.vals[L.final_buf]), reinterpret_cast<const int2*>(ws + L.ranges),
            L.P, L.npix, reinterpret_cast<const StatusWords*>(ws + L.status),
            reinterpret_cast<const float*>(ws + L.recon), ws + L.moments, reinterpret_cast<const float*>(ws + L.saved),
            dL_drgb, dL_dP, dL_dT, reinterpret_cast<float*>(ws + L.dm), grec,
            kept ? reinterpret_cast<const int*>(ws + L.npp) : nullptr,
            kept ? reinterpret_cast<const long long*>(ws + L.pq_off) : nullptr,
            kept ? ws + L.pq : nullptr, L.qcap);
    }
    return MB3DGS_OK;
}

// Pass 2.
int launch_backward_moments(const Params& p, const ViewTable& vt, const Layout& L, char* ws, cudaStream_t st) {
    if (L.n_tiles == 0) return MB3DGS_OK;
    const size_t smem = sizeof(float) * (REC + NK_MOM) * p.batch;
    auto k2 = p.basis == MB3DGS_BASIS_TRIG ? k_bwd_moments<true> : k_bwd_moments<false>;
    if (!allow_dynamic_smem((const void*)k2, sizeof(float) * (REC + NK_MOM) * TPB)) return MB3DGS_ERR_CUDA;
    const TileLaunch t2 = tile_launch(p, L, ws, Q_BWD_MOM, (const void*)k2, smem, st);
    count_launch();
    k2<<<t2.grid, TPB, smem, st>>>(
        p, vt, t2.ts, reinterpret_cast<const float*>(ws + L.rec),
        reinterpret_cast<const int32_t*>(ws + L.vals[L.final_buf]), reinterpret_cast<const int2*>(ws + L.ranges), L.P,
        L.npix, reinterpret_cast<const StatusWords*>(ws + L.status), reinterpret_cast<const float*>(ws + L.recon),
        reinterpret_cast<const float*>(ws + L.dm), reinterpret_cast<float*>(ws + L.grec));
    return MB3DGS_OK;
}

// Chain rule through the preprocessing to the Gaussian parameters.
int launch_backward_preprocess(const Params& p, const ViewTable& vt, const Layout& L, char* ws,
                               const mb3dgs_gaussians& g, const mb3dgs_gaussian_grads& gr, cudaStream_t st) {
    if (L.P == 0) return MB3DGS_OK;
    if (!gr.means || !gr.scales || !gr.quats || !gr.weights || !gr.sh) return MB3DGS_ERR_INVALID_ARG;
    count_launch();
    k_preprocess_bwd<<<(unsigned)ceil_div64(L.P, 64), 64, 0, st>>>(
        p, vt, g.means, g.scales, g.quats, g.weights, g.sh, L.P, g.sh_degree,
        reinterpret_cast<const float*>(ws + L.rec), reinterpret_cast<const float*>(ws + L.grec), gr.means, gr.scales,
        gr.quats, gr.weights, gr.sh);
    return MB3DGS_OK;
}

}  // namespace mb
