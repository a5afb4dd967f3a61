// Storage of the per-pixel moments in the workspace: FP32 planes, or the FP32
// m0 plane plus eight 16-bit moments scaled by 1/m0 per pixel.  Shared by the
// moment pass (store), the reconstruction and shading passes and the adjoint
// (load).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"

namespace mb {

// 16-bit storage: the FP32 m0 plane, then (16-byte aligned) one uint4 of
// eight 16-bit scaled moments per pixel.
__device__ __forceinline__ size_t packed_offset(int64_t npix) { return ((size_t)npix * 4 + 15) & ~(size_t)15; }
__device__ __forceinline__ void store_moments(const Params& p, const float acc[NMOM], int64_t npix, int64_t pix,
                                              void* __restrict__ moments) {
    if (p.moment_dtype == MB3DGS_MOMENTS_F32) {
        float* m = reinterpret_cast<float*>(moments);
#pragma unroll
        for (int k = 0; k < NMOM; ++k) m[k * npix + pix] = acc[k];
    } else {
        // m0 in FP32, I_k / m0 (k >= 1; |.| <~ 1) in 16 bits: per-pixel scaling;
        // a pixel's eight 16-bit values are one 16-byte vector store
        float* m0 = reinterpret_cast<float*>(moments);
        m0[pix] = acc[0];
        const float inv = acc[0] > 0.0f ? 1.0f / acc[0] : 0.0f;
        uint32_t w[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float x0 = acc[2 * k + 1] * inv, x1 = acc[2 * k + 2] * inv;
            if (p.moment_dtype == MB3DGS_MOMENTS_BF16) {
                const __nv_bfloat162 v = __floats2bfloat162_rn(x0, x1);
                w[k] = *reinterpret_cast<const uint32_t*>(&v);
            } else {
                const __half2 v = __floats2half2_rn(x0, x1);
                w[k] = *reinterpret_cast<const uint32_t*>(&v);
            }
        }
        reinterpret_cast<uint4*>(static_cast<char*>(moments) + packed_offset(npix))[pix] =
            make_uint4(w[0], w[1], w[2], w[3]);
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
        const uint4 v = reinterpret_cast<const uint4*>(static_cast<const char*>(moments) + packed_offset(npix))[pix];
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float2 x;
            if (p.moment_dtype == MB3DGS_MOMENTS_BF16) x = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[k]));
            else x = __half22float2(*reinterpret_cast<const __half2*>(&w[k]));
            I[2 * k + 1] = x.x * I[0];
            I[2 * k + 2] = x.y * I[0];
        }
    }
}

}  // namespace mb
