// Stages 3-5: moment pass, per-pixel reconstruction, quadrature pass.
//
// CTAs of 256 threads; every warp takes 8 x 4-pixel footprints of tiles from
// the schedule of tile.cuh (one lane per pixel) and stages the records of
// its footprint, in list order (ascending id), into its own shared memory
// with cp.async.  The moment pass tests each lane's pixel centre against
// each record's rectangle and accumulates in registers; the quadrature pass
// queues the pairs and shades them 32 at a time (below).  Either way each
// pixel sums its Gaussians in list order, so the sums are deterministic and
// the same for every tile shape, batch and schedule.
#include "moments.cuh"
#include "table.cuh"
#include "tile.cuh"

namespace mb {

// ---------------------------------------------------------------- moment pass
__global__ void __launch_bounds__(TPB) k_moments(Params p, ViewTable vt, TileSched ts, const float* __restrict__ rec,
                                                 const int32_t* __restrict__ ids, const int2* __restrict__ ranges,
                                                 int64_t P, int64_t npix, StatusWords* sw,
                                                 void* __restrict__ moments, int* __restrict__ npp) {
    extern __shared__ float4 s_raw[];
    float* s_buf = reinterpret_cast<float*>(s_raw) + (threadIdx.x >> 5) * WARP_STAGE_FLOATS;
    const bool any = sw->n_valid != 0;
    int fp, fx0, fy0;
    for (int64_t tile = next_unit(ts, true, &fp); tile >= 0; tile = next_unit(ts, false, &fp)) {
        PixelCtx c = unit_ctx(vt, ranges, P, tile, fp, &fx0, &fy0);
        if (!any) c.end = c.start;
        float acc[NMOM];
#pragma unroll
        for (int k = 0; k < NMOM; ++k) acc[k] = 0.0f;
        const float fpx = (float)c.px + 0.5f, fpy = (float)c.py + 0.5f;
        int cnt = 0;
        for (int pos = c.start; pos < c.end; pos += 32) {
            const int m = stage_warp_chunk(s_buf, rec, ids, c.rec_base, pos, c.end, fx0, fy0);
            if (c.inside) {
                for (int k = 0; k < m; ++k) {
                    const float* r = s_buf + k * REC;
                    if (!rect_contains(r, c.px, c.py)) continue;
                    const Gauss1D g = pair_gaussian(r, fpx - r[R_AX], fpy - r[R_AY], c.rlen, c.r2);
                    if (p.basis == MB3DGS_BASIS_TRIG) trig_moments(p, g, acc);
                    else legendre_moments(p, g, acc);
                    ++cnt;
                }
            }
        }
        if (c.inside) {
            if (npp) npp[c.pix] = cnt;
            store_moments(p, acc, npix, c.pix, moments);
        }
    }
}

// paper's power moments m-hat_k = int u^k d(measure), u = (y + 1) / 2; with
// the trigonometric basis the moments themselves {m0, Re m1, Im m1, ..}
__global__ void k_moments_to_power(Params p, const void* __restrict__ moments, int64_t npix, float* __restrict__ out) {
    const int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= npix) return;
    float I[NMOM];
    load_moments(p, moments, npix, pix, I);
    if (p.basis == MB3DGS_BASIS_TRIG) {
#pragma unroll
        for (int k = 0; k < NMOM; ++k) out[pix * NMOM + k] = I[k];
        return;
    }
#pragma unroll
    for (int k = 0; k < NMOM; ++k) {
        float s = 0.0f;
#pragma unroll
        for (int l = 0; l < NMOM; ++l) s = fmaf(p.leg_to_pow[k * NMOM + l], I[l], s);
        out[pix * NMOM + k] = s;
    }
}

// ---------------------------------------------------------------- reconstruction
__global__ void k_reconstruct(Params p, const void* __restrict__ moments, int64_t npix, float* __restrict__ recon,
                              const float* __restrict__ eta, int Q, float* __restrict__ T_out) {
    const int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= npix) return;
    float I[NMOM];
    load_moments(p, moments, npix, pix, I);
    if (p.basis == MB3DGS_BASIS_TRIG) {
        TrigRecon T;
        reconstruct_trig(p, I, T);
        store_trig_recon(T, recon, npix, pix);
        if (Q > 0 && eta != nullptr && T_out != nullptr)
            for (int q = 0; q < Q; ++q) T_out[pix * Q + q] = expf(-trig_optical_depth(p, T, eta[pix * Q + q]));
        return;
    }
    Recon R;
    reconstruct_pixel(p, I, R);
    store_recon(R, recon, npix, pix);
    if (Q > 0 && eta != nullptr && T_out != nullptr) {
        for (int q = 0; q < Q; ++q) {
            const float y = fmaf(2.0f, eta[pix * Q + q], -1.0f);
            T_out[pix * Q + q] = expf(-optical_depth(R, p.beta, y));
        }
    }
}

// Per-pixel table of the tabulated transmittance (table.cuh): segment edges
// and M + 1 knots a segment, one thread per pixel.
__global__ void k_build_table(Params p, int64_t npix, const float* __restrict__ recon, float* __restrict__ tab_e,
                              float2* __restrict__ tab) {
    const int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= npix) return;
    const Recon R = load_recon(recon, npix, pix);
    float e[4];
    table_edges(R, e);
#pragma unroll
    for (int k = 0; k < 4; ++k) tab_e[k * npix + pix] = e[k];
    const int M = p.tab_m;
#pragma unroll 1
    for (int s = 0; s < TAB_SEGS; ++s)
#pragma unroll 1
        for (int i = 0; i <= M; ++i) tab[(size_t)(s * (M + 1) + i) * npix + pix] = table_knot(p, R, e, s, i, M);
}

// ---------------------------------------------------------------- quadrature pass
struct TableArgs {
    const float2* tab;
    const float* tab_e;
    int M;
};

__device__ __forceinline__ void load_pixel_state(const float* __restrict__ rc, int64_t npix, int64_t pix,
                                                 const TableArgs&, Recon& R) {
    R = load_recon(rc, npix, pix);
}
__device__ __forceinline__ void load_pixel_state(const float* __restrict__ rc, int64_t npix, int64_t pix,
                                                 const TableArgs&, TrigRecon& T) {
    T = load_trig_recon(rc, npix, pix);
}
__device__ __forceinline__ void load_pixel_state(const float* __restrict__ rc, int64_t npix, int64_t pix,
                                                 const TableArgs& ta, TabPixel& T) {
    T.m0 = rc[pix];
#pragma unroll
    for (int k = 0; k < 4; ++k) T.e[k] = ta.tab_e[k * npix + pix];
    T.tab = ta.tab;
    T.pix = pix;
    T.npix = npix;
    T.M = ta.M;
}

#ifndef MB_SHADE_MIN_CTAS
#define MB_SHADE_MIN_CTAS 3      // resident CTAs per SM the register budget is sized for
#endif

// Power-moment and tabulated shading works on (pixel, Gaussian) pairs
// compacted across the warp.  A rectangle covers on average 3/4 of an 8 x 4
// footprint it overlaps at 1M Gaussians (2/3 at 200k), so shading record by
// record leaves a quarter or more of the lanes idle.  Instead the records of
// a chunk are enumerated in list order, each lane appends the pairs of its own
// pixel to a per-warp queue, and every full round of 32 queued pairs is shaded
// with one pair per lane.  The pixel's state (its reconstruction, ray
// constants and kept-query slot) sits in shared memory for the lane that
// shades the pair; the pair's O_i and P_i go back through shared memory and
// the pixel's own lane adds them in list order, so every per-pixel sum is
// formed from the same terms in the same order as record by record.  The
// trigonometric node solve diverges too much between Gaussians for mixed
// rounds to pay: that basis shades record by record.
template <class RecT>
struct QueuedShading {
    static constexpr bool on = true;
};
template <>
struct QueuedShading<TrigRecon> {
    static constexpr bool on = false;
};

template <class RecT>
struct alignas(16) ShadePixel {
    RecT R;
    float fpx, fpy, rlen, r2;
    char* qp;                  // the pixel's kept queries (nullptr: not kept)
};

template <class RecT>
struct ShadeWarp {
    float rec[32 * REC];       // staged records (stage_warp_chunk's layout: records, then their ids)
    int ids[32];
    ShadePixel<RecT> pix[32];
    int ent[64];               // queued pairs: record k of the chunk | pixel lane << 5
    int ord[64];               // the pair's ordinal among its pixel's pairs (its kept-query slot)
    float2 res[32];            // O_i and P_i of the round's pairs
};

template <class RecT>
constexpr size_t shade_smem_bytes() {
    return QueuedShading<RecT>::on ? sizeof(ShadeWarp<RecT>) * WARPS : sizeof(float) * WARP_STAGE_FLOATS * WARPS;
}
// MB_SHADE_MIN_CTAS CTAs must fit the SM's 228 KB of shared memory (1 KB of
// it reserved per CTA) for the register budget of __launch_bounds__ to pay.
static_assert(MB_SHADE_MIN_CTAS * (shade_smem_bytes<Recon>() + 1024) <= 228 * 1024 &&
                  MB_SHADE_MIN_CTAS * (shade_smem_bytes<TabPixel>() + 1024) <= 228 * 1024,
              "queued shading: shared memory per CTA too large for the resident CTAs");

template <int NI, bool SAVE, class RecT, int QB = 16>
__global__ void __launch_bounds__(TPB, MB_SHADE_MIN_CTAS) k_shade(Params p, ViewTable vt, TileSched ts, const float* __restrict__ rec,
                                               const int32_t* __restrict__ ids, const int2* __restrict__ ranges,
                                               int64_t P, int64_t npix, const StatusWords* sw,
                                               const float* __restrict__ recon, const void* __restrict__ moments,
                                               float* __restrict__ rgb,
                                               float* __restrict__ T_final, float* __restrict__ penalty,
                                               float* __restrict__ saved, const int* __restrict__ npp,
                                               const long long* __restrict__ pq_off, char* __restrict__ pq,
                                               int64_t qcap, TableArgs ta) {
    extern __shared__ float4 s_raw[];
    const int lane = threadIdx.x & 31;
    const bool any = sw->n_valid != 0;
    // saved queries: a pixel's pairs from pq_off[pix], N+1 queries of QB bytes
    // each, for the pixels all of whose pairs fit the capacity (a prefix in
    // pixel order)
    const int nq = (NI > 0 ? NI : p.n_intervals) + 1;
    int fp, fx0, fy0;
    for (int64_t tile = next_unit(ts, true, &fp); tile >= 0; tile = next_unit(ts, false, &fp)) {
        PixelCtx c = unit_ctx(vt, ranges, P, tile, fp, &fx0, &fy0);
        if (!any) c.end = c.start;
        float S0 = 0.0f, S1 = 0.0f, S2 = 0.0f, O = 0.0f, Pen = 0.0f;
        const float fpx = (float)c.px + 0.5f, fpy = (float)c.py + 0.5f;
        char* qp = nullptr;
        if (SAVE && c.inside) {
            const long long off = pq_off[c.pix];
            if (off + npp[c.pix] <= qcap) qp = pq + (size_t)off * nq * QB;
        }
        if constexpr (QueuedShading<RecT>::on) {
            ShadeWarp<RecT>* W = reinterpret_cast<ShadeWarp<RecT>*>(s_raw) + (threadIdx.x >> 5);
            const unsigned lanes_below = (1u << lane) - 1u;
            __syncwarp();                 // the previous unit's pixel states are no longer read
            {
                ShadePixel<RecT>& me = W->pix[lane];
                if (c.inside) load_pixel_state(recon, npix, c.pix, ta, me.R);
                me.fpx = fpx;
                me.fpy = fpy;
                me.rlen = c.rlen;
                me.r2 = c.r2;
                me.qp = qp;
            }
            int nown = 0;                 // pairs of this lane's pixel queued so far
            for (int pos = c.start; pos < c.end; pos += 32) {
                const int m = stage_warp_chunk(W->rec, rec, ids, c.rec_base, pos, c.end, fx0, fy0);
                int k = 0, pending = 0;
                unsigned long long mine = 0;  // queue slots holding this lane's pairs
                for (;;) {
                    // enqueue records until a round is full (at most 63 pairs queued)
                    for (; k < m && pending < 32; ++k) {
                        const bool act = c.inside && rect_contains(W->rec + k * REC, c.px, c.py);
                        const unsigned mask = __ballot_sync(0xffffffffu, act);
                        if (act) {
                            const int slot = pending + __popc(mask & lanes_below);
                            W->ent[slot] = k | lane << 5;
                            W->ord[slot] = nown++;
                            mine |= 1ull << slot;
                        }
                        pending += __popc(mask);
                    }
                    if (pending == 0) break;
                    const int n = pending < 32 ? pending : 32;
                    __syncwarp();         // queued pairs visible to every lane
                    float Oi = 0.0f, Pi = 0.0f;
                    if (lane < n) {
                        const int e = W->ent[lane];
                        const ShadePixel<RecT>& px = W->pix[e >> 5];
                        const RecT R = px.R;
                        const float* r = W->rec + (e & 31) * REC;
                        const Gauss1D g = pair_gaussian(r, px.fpx - r[R_AX], px.fpy - r[R_AY], px.rlen, px.r2);
                        char* q = SAVE && px.qp ? px.qp + (size_t)W->ord[lane] * nq * QB : nullptr;
                        Oi = pair_quadrature<NI, SAVE, RecT, QB>(p, R, g, &Pi, q);
                    }
                    W->res[lane] = make_float2(Oi, Pi);
                    __syncwarp();         // the round's results visible to every lane
                    for (unsigned own = (unsigned)mine; own != 0u; own &= own - 1u) {
                        const int s = __ffs(own) - 1;
                        const float2 v = W->res[s];
                        const float* r = W->rec + (W->ent[s] & 31) * REC;
                        S0 = fmaf(r[R_RGB + 0], v.x, S0);
                        S1 = fmaf(r[R_RGB + 1], v.x, S1);
                        S2 = fmaf(r[R_RGB + 2], v.x, S2);
                        O += v.x;
                        Pen += v.y;
                    }
                    // move the pairs queued beyond the round to the front
                    const int rest = pending - n;
                    int e2 = 0, o2 = 0;
                    if (lane < rest) { e2 = W->ent[32 + lane]; o2 = W->ord[32 + lane]; }
                    __syncwarp();         // every read of slots 0..31 done
                    if (lane < rest) { W->ent[lane] = e2; W->ord[lane] = o2; }
                    mine >>= 32;
                    pending = rest;
                }
            }
        } else {
            float* s_buf = reinterpret_cast<float*>(s_raw) + (threadIdx.x >> 5) * WARP_STAGE_FLOATS;
            RecT R;
            if (c.inside) load_pixel_state(recon, npix, c.pix, ta, R);
            else R.m0 = 0.0f;
            for (int pos = c.start; pos < c.end; pos += 32) {
                const int m = stage_warp_chunk(s_buf, rec, ids, c.rec_base, pos, c.end, fx0, fy0);
                if (c.inside) {
                    for (int k = 0; k < m; ++k) {
                        const float* r = s_buf + k * REC;
                        if (!rect_contains(r, c.px, c.py)) continue;
                        const Gauss1D g = pair_gaussian(r, fpx - r[R_AX], fpy - r[R_AY], c.rlen, c.r2);
                        const float Oi = pair_quadrature<NI, SAVE, RecT, QB>(p, R, g, &Pen, qp);
                        if (SAVE && qp) qp += nq * QB;
                        S0 = fmaf(r[R_RGB + 0], Oi, S0);
                        S1 = fmaf(r[R_RGB + 1], Oi, S1);
                        S2 = fmaf(r[R_RGB + 2], Oi, S2);
                        O += Oi;
                    }
                }
            }
        }
        if (c.inside) {
            // Eq. 15: L-hat = (1 - e^{-m0}) / max(eps, O) sum L_i + e^{-m0} L_bg
            const float m0 = reinterpret_cast<const float*>(moments)[c.pix];   // m0: first plane in every storage
            const float Tf = expf(-m0);           // total optical depth m0 is exact (Sec. 3.2)
            const float scale = -expm1f(-m0) / fmaxf(p.eps, O);
            rgb[3 * c.pix + 0] = fmaf(scale, S0, Tf * p.bg[0]);
            rgb[3 * c.pix + 1] = fmaf(scale, S1, Tf * p.bg[1]);
            rgb[3 * c.pix + 2] = fmaf(scale, S2, Tf * p.bg[2]);
            T_final[c.pix] = Tf;
            if (penalty) penalty[c.pix] = Pen;
            saved[0 * npix + c.pix] = S0;
            saved[1 * npix + c.pix] = S1;
            saved[2 * npix + c.pix] = S2;
            saved[3 * npix + c.pix] = O;
        }
    }
}

// ---------------------------------------------------------------- launchers
void exclusive_scan64(const int* in, long long* out, int64_t n, long long* tmp, cudaStream_t st);

void launch_moments(const Params& p, const ViewTable& vt, const Layout& L, char* ws, cudaStream_t st) {
    if (L.n_tiles == 0) return;
    const size_t smem = sizeof(float) * WARP_STAGE_FLOATS * WARPS;
    int* npp = L.qcap > 0 ? reinterpret_cast<int*>(ws + L.npp) : nullptr;
    const TileLaunch tl = tile_launch(p, L, ws, Q_MOMENTS, (const void*)k_moments, smem, st);
    count_launch();
    k_moments<<<tl.grid, TPB, smem, st>>>(
        p, vt, tl.ts, reinterpret_cast<const float*>(ws + L.rec),
        reinterpret_cast<const int32_t*>(ws + L.vals[L.final_buf]), reinterpret_cast<const int2*>(ws + L.ranges), L.P,
        L.npix, reinterpret_cast<StatusWords*>(ws + L.status), ws + L.moments, npp);
    if (npp)
        exclusive_scan64(npp, reinterpret_cast<long long*>(ws + L.pq_off), L.npix,
                         reinterpret_cast<long long*>(ws + L.scan_tmp), st);
}

void launch_moments_to_power(const Params& p, const Layout& L, char* ws, float* out, cudaStream_t st) {
    if (L.npix == 0) return;
    count_launch();
    k_moments_to_power<<<(unsigned)ceil_div64(L.npix, 256), 256, 0, st>>>(p, ws + L.moments, L.npix, out);
}

void launch_reconstruct(const Params& p, const Layout& L, char* ws, const float* eta, int Q, float* T_out,
                        cudaStream_t st) {
    if (L.npix == 0) return;
    count_launch();
    k_reconstruct<<<(unsigned)ceil_div64(L.npix, 128), 128, 0, st>>>(
        p, ws + L.moments, L.npix, reinterpret_cast<float*>(ws + L.recon), eta, Q, T_out);
    if (L.tab_m > 0) {
        count_launch();
        k_build_table<<<(unsigned)ceil_div64(L.npix, 128), 128, 0, st>>>(
            p, L.npix, reinterpret_cast<const float*>(ws + L.recon), reinterpret_cast<float*>(ws + L.tab_e),
            reinterpret_cast<float2*>(ws + L.tab));
    }
}

int launch_shade(const Params& p, const ViewTable& vt, const Layout& L, char* ws, float* rgb, float* T_final,
                 float* penalty, cudaStream_t st) {
    if (L.n_tiles == 0) return MB3DGS_OK;
    const size_t smem = p.basis == MB3DGS_BASIS_TRIG ? shade_smem_bytes<TrigRecon>()
                        : L.tab_m > 0                ? shade_smem_bytes<TabPixel>()
                                                     : shade_smem_bytes<Recon>();
    const bool save = L.qcap > 0;
    auto kern = p.basis == MB3DGS_BASIS_TRIG
                    ? (save ? (p.n_intervals == 3   ? k_shade<3, true, TrigRecon>
                               : p.n_intervals == 5 ? k_shade<5, true, TrigRecon> : k_shade<0, true, TrigRecon>)
                            : (p.n_intervals == 3   ? k_shade<3, false, TrigRecon>
                               : p.n_intervals == 5 ? k_shade<5, false, TrigRecon> : k_shade<0, false, TrigRecon>))
              : L.tab_m > 0
                    ? (p.n_intervals == 3 ? k_shade<3, false, TabPixel>
                       : p.n_intervals == 5 ? k_shade<5, false, TabPixel> : k_shade<0, false, TabPixel>)
              : save && p.qbytes == 8
                    ? (p.n_intervals == 3 ? k_shade<3, true, Recon, 8> : k_shade<0, true, Recon, 8>)
              : p.n_intervals == 3 ? (save ? k_shade<3, true, Recon> : k_shade<3, false, Recon>)
              : p.n_intervals == 5 ? (save ? k_shade<5, true, Recon> : k_shade<5, false, Recon>)
                                   : (save ? k_shade<0, true, Recon> : k_shade<0, false, Recon>);
    if (!allow_dynamic_smem((const void*)kern, smem)) return MB3DGS_ERR_CUDA;
    const TileLaunch tl = tile_launch(p, L, ws, Q_SHADE, (const void*)kern, smem, st);
    count_launch();
    kern<<<tl.grid, TPB, smem, st>>>(
        p, vt, tl.ts, reinterpret_cast<const float*>(ws + L.rec),
        reinterpret_cast<const int32_t*>(ws + L.vals[L.final_buf]), reinterpret_cast<const int2*>(ws + L.ranges), L.P,
        L.npix, reinterpret_cast<const StatusWords*>(ws + L.status), reinterpret_cast<const float*>(ws + L.recon),
        ws + L.moments, rgb, T_final, penalty, reinterpret_cast<float*>(ws + L.saved),
        save ? reinterpret_cast<const int*>(ws + L.npp) : nullptr,
        save ? reinterpret_cast<const long long*>(ws + L.pq_off) : nullptr,
        save ? ws + L.pq : nullptr, L.qcap,
        TableArgs{L.tab_m > 0 ? reinterpret_cast<const float2*>(ws + L.tab) : nullptr,
                  L.tab_m > 0 ? reinterpret_cast<const float*>(ws + L.tab_e) : nullptr, L.tab_m});
    return MB3DGS_OK;
}

}  // namespace mb
