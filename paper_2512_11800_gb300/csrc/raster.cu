// Stages 3-5: moment pass, per-pixel reconstruction, quadrature pass.
//
// One CTA per 16x16 tile, one thread per pixel.  The tile's Gaussian list
// (ascending id) is walked in batches of 256 records staged in shared memory
// with cp.async (each thread copies 8 x 16 B; no multicast); every thread
// tests its pixel centre against each record's rectangle and accumulates in
// registers, so per-pixel sums are in a fixed order (deterministic).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"

namespace mb {

struct StatusWordsR {
    int status;
    int pad;
    long long n_total;
    long long n_valid;
    unsigned long long nonfinite;
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::); }

// Stage the records of list[start + b*TPB .. ) into shared memory.
__device__ __forceinline__ int stage_batch(float* s_rec, const float* __restrict__ rec, const int32_t* __restrict__ ids,
                                           int64_t rec_base, int start, int end, int b) {
    const int first = start + b * TPB;
    const int nb = min(TPB, end - first);
#pragma unroll
    for (int j = 0; j < REC / 4; ++j) {
        const int lin = j * TPB + threadIdx.x;
        const int rr = lin >> 3, cc = lin & 7;
        if (rr < nb) {
            const int64_t gi = rec_base + ids[first + rr];
            cp_async16(s_rec + rr * REC + cc * 4, rec + gi * REC + cc * 4);
        }
    }
    cp_async_wait_all();
    __syncthreads();
    return nb;
}

struct PixelCtx {
    int v;
    int px, py;
    bool inside;
    int64_t pix;       // global pixel index
    float rlen, r2;    // |K^-1 (p + 1/2, 1)| and its square
    int start, end;    // tile list range
    int64_t rec_base;  // v * P
};

__device__ __forceinline__ PixelCtx pixel_ctx(const ViewTable& vt, const int2* __restrict__ ranges, int64_t P,
                                              int64_t tile) {
    PixelCtx c;
    c.v = find_view(vt, tile);
    const ViewDesc& V = vt.v[c.v];
    const int lt = (int)(tile - V.tile_base);
    const int tx = lt % V.tiles_x, ty = lt / V.tiles_x;
    // each warp covers an 8x4 block of the tile (fewer partially covered warps
    // than 16x2 rows for rectangle-shaped footprints)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    c.px = tx * TILE + (warp & 1) * 8 + (lane & 7);
    c.py = ty * TILE + (warp >> 1) * 4 + (lane >> 3);
    c.inside = c.px < V.width && c.py < V.height;
    c.pix = V.pixel_base + (int64_t)c.py * V.width + c.px;
    const float ux = ((float)c.px + 0.5f - V.cx) / V.fx;
    const float uy = ((float)c.py + 0.5f - V.cy) / V.fy;
    c.r2 = fmaf(ux, ux, fmaf(uy, uy, 1.0f));
    c.rlen = sqrtf(c.r2);
    const int2 rg = ranges[tile];
    c.start = rg.x;
    c.end = rg.y;
    c.rec_base = (int64_t)c.v * P;
    return c;
}

// ---------------------------------------------------------------- moment pass
__global__ void __launch_bounds__(TPB) k_moments(Params p, ViewTable vt, const float* __restrict__ rec,
                                                 const int32_t* __restrict__ ids, const int2* __restrict__ ranges,
                                                 int64_t P, int64_t npix, const StatusWordsR* sw,
                                                 void* __restrict__ moments) {
    extern __shared__ float4 s_raw[];
    float* s_rec = reinterpret_cast<float*>(s_raw);
    const int64_t tile = blockIdx.x;
    PixelCtx c = pixel_ctx(vt, ranges, P, tile);
    if (sw->n_valid == 0) c.end = c.start;
    float acc[NMOM];
#pragma unroll
    for (int k = 0; k < NMOM; ++k) acc[k] = 0.0f;
    const int n = c.end - c.start;
    const float fpx = (float)c.px + 0.5f, fpy = (float)c.py + 0.5f;
    for (int b = 0; b * TPB < n; ++b) {
        const int nb = stage_batch(s_rec, rec, ids, c.rec_base, c.start, c.end, b);
        if (c.inside) {
            for (int k = 0; k < nb; ++k) {
                const float* r = s_rec + k * REC;
                if (!rect_contains(r, c.px, c.py)) continue;
                const Gauss1D g = pair_gaussian(r, fpx - r[R_AX], fpy - r[R_AY], c.rlen, c.r2);
                legendre_moments(p, g, acc);
            }
        }
        __syncthreads();
    }
    if (!c.inside) return;
    if (p.moment_dtype == MB3DGS_MOMENTS_F32) {
        float* m = reinterpret_cast<float*>(moments);
#pragma unroll
        for (int k = 0; k < NMOM; ++k) m[k * npix + c.pix] = acc[k];
    } else {
        // m0 in FP32, I_k / m0 (k >= 1; |.| <~ 1) in 16 bits: per-pixel scaling
        float* m0 = reinterpret_cast<float*>(moments);
        m0[c.pix] = acc[0];
        const float inv = acc[0] > 0.0f ? 1.0f / acc[0] : 0.0f;
        uint16_t* h = reinterpret_cast<uint16_t*>(m0 + npix);
#pragma unroll
        for (int k = 1; k < NMOM; ++k) {
            const float x = acc[k] * inv;
            uint16_t bits;
            if (p.moment_dtype == MB3DGS_MOMENTS_BF16) {
                __nv_bfloat16 hb = __float2bfloat16_rn(x);
                bits = *reinterpret_cast<uint16_t*>(&hb);
            } else {
                __half hh = __float2half_rn(x);
                bits = *reinterpret_cast<uint16_t*>(&hh);
            }
            h[(k - 1) * npix + c.pix] = bits;
        }
    }
}

__device__ __forceinline__ void load_moments(const Params& p, const void* __restrict__ moments, int64_t npix,
                                             int64_t pix, float I[NMOM]) {
    if (p.moment_dtype == MB3DGS_MOMENTS_F32) {
        const float* m = reinterpret_cast<const float*>(moments);
#pragma unroll
        for (int k = 0; k < NMOM; ++k) I[k] = m[k * npix + pix];
    } else {
        const float* m0 = reinterpret_cast<const float*>(moments);
        I[0] = m0[pix];
        const uint16_t* h = reinterpret_cast<const uint16_t*>(m0 + npix);
#pragma unroll
        for (int k = 1; k < NMOM; ++k) {
            uint16_t bits = h[(k - 1) * npix + pix];
            float x;
            if (p.moment_dtype == MB3DGS_MOMENTS_BF16) {
                __nv_bfloat16 hb = *reinterpret_cast<__nv_bfloat16*>(&bits);
                x = __bfloat162float(hb);
            } else {
                __half hh = *reinterpret_cast<__half*>(&bits);
                x = __half2float(hh);
            }
            I[k] = x * I[0];
        }
    }
}

// paper's power moments m-hat_k = int u^k d(measure), u = (y + 1) / 2
__global__ void k_moments_to_power(Params p, const void* __restrict__ moments, int64_t npix, float* __restrict__ out) {
    const int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= npix) return;
    float I[NMOM];
    load_moments(p, moments, npix, pix, I);
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

// ---------------------------------------------------------------- quadrature pass
template <int NI>
__global__ void __launch_bounds__(TPB, 3) k_shade(Params p, ViewTable vt, const float* __restrict__ rec,
                                               const int32_t* __restrict__ ids, const int2* __restrict__ ranges,
                                               int64_t P, int64_t npix, const StatusWordsR* sw,
                                               const float* __restrict__ recon, const void* __restrict__ moments,
                                               float* __restrict__ rgb,
                                               float* __restrict__ T_final, float* __restrict__ penalty,
                                               float* __restrict__ saved) {
    extern __shared__ float4 s_raw[];
    float* s_rec = reinterpret_cast<float*>(s_raw);
    const int64_t tile = blockIdx.x;
    PixelCtx c = pixel_ctx(vt, ranges, P, tile);
    if (sw->n_valid == 0) c.end = c.start;
    Recon R;
    if (c.inside) R = load_recon(recon, npix, c.pix);
    else R.m0 = 0.0f;
    float S0 = 0.0f, S1 = 0.0f, S2 = 0.0f, O = 0.0f, Pen = 0.0f;
    const int n = c.end - c.start;
    const float fpx = (float)c.px + 0.5f, fpy = (float)c.py + 0.5f;
    for (int b = 0; b * TPB < n; ++b) {
        const int nb = stage_batch(s_rec, rec, ids, c.rec_base, c.start, c.end, b);
        if (c.inside) {
            for (int k = 0; k < nb; ++k) {
                const float* r = s_rec + k * REC;
                if (!rect_contains(r, c.px, c.py)) continue;
                const Gauss1D g = pair_gaussian(r, fpx - r[R_AX], fpy - r[R_AY], c.rlen, c.r2);
                const float Oi = pair_quadrature<NI>(p, R, g, &Pen);
                S0 = fmaf(r[R_RGB + 0], Oi, S0);
                S1 = fmaf(r[R_RGB + 1], Oi, S1);
                S2 = fmaf(r[R_RGB + 2], Oi, S2);
                O += Oi;
            }
        }
        __syncthreads();
    }
    if (!c.inside) return;
    // Eq. 15: L-hat = (1 - e^{-m0}) / max(eps, O) sum L_i + e^{-m0} L_bg
    float I[NMOM];
    load_moments(p, moments, npix, c.pix, I);
    const float m0 = I[0];           // total optical depth, exact (Sec. 3.2)
    const float Tf = expf(-m0);
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

// ---------------------------------------------------------------- launchers
void launch_moments(const Params& p, const ViewTable& vt, const Layout& L, char* ws, cudaStream_t st) {
    if (L.n_tiles == 0) return;
    const size_t smem = sizeof(float) * REC * TPB;
    count_launch();
    k_moments<<<(unsigned)L.n_tiles, TPB, smem, st>>>(
        p, vt, reinterpret_cast<const float*>(ws + L.rec), reinterpret_cast<const int32_t*>(ws + L.vals[L.final_buf]),
        reinterpret_cast<const int2*>(ws + L.ranges), L.P, L.npix, reinterpret_cast<const StatusWordsR*>(ws + L.status),
        ws + L.moments);
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
}

void launch_shade(const Params& p, const ViewTable& vt, const Layout& L, char* ws, float* rgb, float* T_final,
                  float* penalty, cudaStream_t st) {
    if (L.n_tiles == 0) return;
    const size_t smem = sizeof(float) * REC * TPB;
    auto kern = p.n_intervals == 3 ? k_shade<3> : (p.n_intervals == 5 ? k_shade<5> : k_shade<0>);
    count_launch();
    kern<<<(unsigned)L.n_tiles, TPB, smem, st>>>(
        p, vt, reinterpret_cast<const float*>(ws + L.rec), reinterpret_cast<const int32_t*>(ws + L.vals[L.final_buf]),
        reinterpret_cast<const int2*>(ws + L.ranges), L.P, L.npix, reinterpret_cast<const StatusWordsR*>(ws + L.status),
        reinterpret_cast<const float*>(ws + L.recon), ws + L.moments, rgb, T_final, penalty,
        reinterpret_cast<float*>(ws + L.saved));
}

}  // namespace mb
