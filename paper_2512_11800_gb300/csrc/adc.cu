// Adaptive density control (Sec. 3.4 "Training and Densification"; App. D
// "Adaptive Density Control"): the per-Gaussian rules between optimiser
// steps, one thread per Gaussian (HBM-bound: a Gaussian's 236 bytes in, up to
// twice that out).
//
// Densification is two launches around a scan: the first decides each
// input's action and how many of its resulting particles survive pruning,
// the exclusive scan of those counts gives every input its output slot, and
// the second decides again (the same float32 arithmetic, so the same answer)
// and writes.  Threshold tests use round-to-nearest intrinsics in a fixed
// order (no fused multiply-add), so that decisions are reproducible
// bit-for-bit by a float32 evaluation of the same expressions.
#include <cmath>
#include <cstring>

#include <cuda_runtime.h>

#include "common.cuh"

namespace mb {

void exclusive_scan(const int* in, int* out, int64_t n, int* tmp, cudaStream_t st);
size_t scan_tmp_elems(int64_t n);

constexpr float SQRT_2PI_F = 2.50662827463100050f;

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr int ADC_TPB = 256;

struct AdcParams {
    float grad_threshold;
    float tau_min;       // -log(1 - prune_opacity): opacity >= o_min  <=>  sqrt(2 pi) w min(s) >= tau_min
    float dense_limit;   // percent_dense x scene_extent
    float big_limit;     // big_world x scene_extent (+inf when off)
    float gamma, delta;
};

__global__ void k_vi_opacity(const float* __restrict__ w, const float* __restrict__ s, int64_t P,
                             float* __restrict__ o) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const float smin = fminf(fminf(s[3 * i], s[3 * i + 1]), s[3 * i + 2]);
    o[i] = -expm1f(-SQRT_2PI_F * w[i] * smin);
}

__global__ void k_init_weights(const float* __restrict__ o, const float* __restrict__ s, int64_t P,
                               float* __restrict__ w) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const float avg = (s[3 * i] + s[3 * i + 1] + s[3 * i + 2]) * (1.0f / 3.0f);
    w[i] = -log1pf(-o[i]) / (SQRT_2PI_F * avg);
}

__global__ void k_grad_stats(const float* __restrict__ d, const uint8_t* __restrict__ vis, int64_t P,
                             float* __restrict__ abs_sum, int32_t* __restrict__ count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const float dx = d[3 * i], dy = d[3 * i + 1], dz = d[3 * i + 2];
    const bool v = vis ? vis[i] != 0 : (dx != 0.0f || dy != 0.0f || dz != 0.0f);
    if (!v) return;
    abs_sum[3 * i] = __fadd_rn(abs_sum[3 * i], fabsf(dx));
    abs_sum[3 * i + 1] = __fadd_rn(abs_sum[3 * i + 1], fabsf(dy));
    abs_sum[3 * i + 2] = __fadd_rn(abs_sum[3 * i + 2], fabsf(dz));
    count[i] += 1;
}

// Pruning test of one resulting particle.
__device__ __forceinline__ bool adc_keep(const AdcParams& a, float w, float s0, float s1, float s2) {
    const float dens = __fmul_rn(__fmul_rn(SQRT_2PI_F, w), fminf(fminf(s0, s1), s2));
    if (!(dens >= a.tau_min)) return false;
    return !(fmaxf(fmaxf(s0, s1), s2) > a.big_limit);
}

struct AdcDecision {
    int action;       // 0 kept as is, 1 clone, 2 split
    int k;            // split axis (largest scale, first on ties)
    float s[3];       // scales of the resulting particles
    float w;          // their peak density
    bool keep[2];     // survive pruning (one result for action 0)
};

__device__ __forceinline__ AdcDecision adc_decide(const AdcParams& a, const float* __restrict__ scales,
                                                  const float* __restrict__ weights, const float* __restrict__ abs_sum,
                                                  const int32_t* __restrict__ count, int64_t i) {
    AdcDecision d;
    d.s[0] = scales[3 * i];
    d.s[1] = scales[3 * i + 1];
    d.s[2] = scales[3 * i + 2];
    d.w = weights[i];
    const int n = count[i];
    bool grow = false;
    if (n > 0) {
        const float ax = abs_sum[3 * i], ay = abs_sum[3 * i + 1], az = abs_sum[3 * i + 2];
        float n2 = __fadd_rn(__fmul_rn(ax, ax), __fmul_rn(ay, ay));
        n2 = __fadd_rn(n2, __fmul_rn(az, az));
        grow = __fdiv_rn(__fsqrt_rn(n2), (float)n) >= a.grad_threshold;
    }
    d.k = 0;
    if (d.s[1] > d.s[d.k]) d.k = 1;
    if (d.s[2] > d.s[d.k]) d.k = 2;
    const float smax = d.s[d.k];
    d.action = grow ? (smax <= a.dense_limit ? 1 : 2) : 0;
    if (d.action == 1) {
        d.w = d.w * 0.5f;
    } else if (d.action == 2) {
        d.s[d.k] = __fmul_rn(a.gamma, smax);
    }
    d.keep[0] = adc_keep(a, d.w, d.s[0], d.s[1], d.s[2]);
    d.keep[1] = d.action != 0 && d.keep[0];   // both results of a clone or a split have the same shape
    return d;
}

__global__ void k_densify_count(AdcParams a, const float* __restrict__ scales, const float* __restrict__ weights,
                                const float* __restrict__ abs_sum, const int32_t* __restrict__ count, int64_t P,
                                int* __restrict__ n_out, int8_t* __restrict__ action) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const AdcDecision d = adc_decide(a, scales, weights, abs_sum, count, i);
    n_out[i] = (int)d.keep[0] + (int)d.keep[1];
    if (action) action[i] = (int8_t)d.action;
}

__global__ void k_densify_total(const int* __restrict__ n_out, const int* __restrict__ off, int64_t P,
                                int64_t* __restrict__ total) {
    *total = P > 0 ? (int64_t)off[P - 1] + n_out[P - 1] : 0;
}

// The small fields of a result are written by its input's thread; the SH
// coefficients (192 bytes a particle at degree 3), copied once per result,
// by the whole warp for one input at a time, so that loads and stores are
// coalesced.
__global__ void k_densify_write(AdcParams a, mb3dgs_gaussians g, const float* __restrict__ abs_sum,
                                const int32_t* __restrict__ count, const int* __restrict__ off,
                                mb3dgs_gaussians_out out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool active = i < g.P;
    int nres = 0;
    int64_t o = 0;
    if (active) {
        const AdcDecision d = adc_decide(a, g.scales, g.weights, abs_sum, count, i);
        if (d.keep[0]) {
            nres = d.action == 0 ? 1 : 2;
            o = off[i];
            const float m[3] = {g.means[3 * i], g.means[3 * i + 1], g.means[3 * i + 2]};
            const float q[4] = {g.quats[4 * i], g.quats[4 * i + 1], g.quats[4 * i + 2], g.quats[4 * i + 3]};
            float v[3] = {0.0f, 0.0f, 0.0f};
            if (d.action == 2) {
                // column k of R(q) (Sigma = R S^2 R^T): the axis of the largest scale
                const float inv = rsqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
                const float w = q[0] * inv, x = q[1] * inv, y = q[2] * inv, z = q[3] * inv;
                if (d.k == 0) { v[0] = 1.0f - 2.0f * (y * y + z * z); v[1] = 2.0f * (x * y + w * z); v[2] = 2.0f * (x * z - w * y); }
                else if (d.k == 1) { v[0] = 2.0f * (x * y - w * z); v[1] = 1.0f - 2.0f * (x * x + z * z); v[2] = 2.0f * (y * z + w * x); }
                else { v[0] = 2.0f * (x * z + w * y); v[1] = 2.0f * (y * z - w * x); v[2] = 1.0f - 2.0f * (x * x + y * y); }
                const float step = a.delta * g.scales[3 * i + d.k];   // delta times the unsplit s_max
                for (int c = 0; c < 3; ++c) v[c] *= step;
            }
            for (int r = 0; r < nres; ++r) {
                const int64_t t = o + r;
                const float sign = r == 0 ? -1.0f : 1.0f;   // split: minus offset first
                for (int c = 0; c < 3; ++c) {
                    out.means[3 * t + c] = d.action == 2 ? fmaf(sign, v[c], m[c]) : m[c];
                    out.scales[3 * t + c] = d.s[c];
                }
                for (int c = 0; c < 4; ++c) out.quats[4 * t + c] = q[c];
                out.weights[t] = d.w;
            }
        }
    }
    const int K3 = 3 * (g.sh_degree + 1) * (g.sh_degree + 1);
    unsigned todo = __ballot_sync(0xffffffffu, nres > 0);
    // four inputs at a time: their loads are issued before their stores
    constexpr int G = 4, MAXC = 2;   // K3 <= 48 <= MAXC x 32 floats a lane covers (8 measured slower)
    while (todo) {
        long long si[G], so[G];
        int n[G];
#pragma unroll
        for (int u = 0; u < G; ++u) {
            const int src = todo ? __ffs(todo) - 1 : 0;
            const bool has = todo != 0;
            todo &= todo - 1;
            si[u] = __shfl_sync(0xffffffffu, (long long)i, src);
            so[u] = __shfl_sync(0xffffffffu, (long long)o, src);
            n[u] = has ? __shfl_sync(0xffffffffu, nres, src) : 0;
        }
        float x[G][MAXC];
#pragma unroll
        for (int u = 0; u < G; ++u)
#pragma unroll
            for (int t = 0; t < MAXC; ++t) {
                const int c = lane + 32 * t;
                x[u][t] = (n[u] > 0 && c < K3) ? g.sh[(size_t)si[u] * K3 + c] : 0.0f;
            }
#pragma unroll
        for (int u = 0; u < G; ++u)
#pragma unroll
            for (int t = 0; t < MAXC; ++t) {
                const int c = lane + 32 * t;
                if (n[u] > 0 && c < K3) {
                    out.sh[(size_t)so[u] * K3 + c] = x[u][t];
                    if (n[u] == 2) out.sh[(size_t)(so[u] + 1) * K3 + c] = x[u][t];
                }
            }
    }
}

static int adc_params(const mb3dgs_adc_config* c, AdcParams& a) {
    if (!c) return MB3DGS_ERR_INVALID_ARG;
    if (!(c->grad_threshold >= 0.0f) || !(c->prune_opacity >= 0.0f && c->prune_opacity < 1.0f) ||
        !(c->percent_dense >= 0.0f) || !(c->scene_extent > 0.0f) || !(c->big_world >= 0.0f) ||
        !(c->split_gamma > 0.0f && c->split_gamma <= 1.0f) || !(c->split_delta >= 0.0f))
        return MB3DGS_ERR_INVALID_ARG;
    a.grad_threshold = c->grad_threshold;
    a.tau_min = (float)(-std::log1p(-(double)c->prune_opacity));
    a.dense_limit = (float)((double)c->percent_dense * (double)c->scene_extent);
    a.big_limit = c->big_world > 0.0f ? (float)((double)c->big_world * (double)c->scene_extent) : INFINITY;
    a.gamma = c->split_gamma;
    a.delta = c->split_delta;
    return MB3DGS_OK;
}

static size_t densify_ws_bytes(int64_t P) {
    const size_t n = (size_t)(P > 0 ? P : 1);
    return align256(sizeof(int) * n) * 2 + align256(sizeof(int) * scan_tmp_elems((int64_t)n));
}

}  // namespace mb

using namespace mb;

static inline unsigned adc_grid(int64_t P) { return (unsigned)ceil_div64(P, ADC_TPB); }

extern "C" int mb3dgs_adc_config_default(mb3dgs_adc_config* c) {
    if (!c) return MB3DGS_ERR_INVALID_ARG;
    c->grad_threshold = 1e-4f;
    c->prune_opacity = 0.005f;
    c->percent_dense = 0.01f;
    c->scene_extent = 1.0f;
    c->big_world = 0.1f;
    c->split_gamma = 0.6385502815246582f;
    c->split_delta = 0.6128153090966912f;
    return MB3DGS_OK;
}

extern "C" int mb3dgs_view_independent_opacity(const float* d_weights, const float* d_scales, int64_t P,
                                               float* d_opacity, mb3dgs_stream_t stream) {
    if (P < 0 || (P > 0 && (!d_weights || !d_scales || !d_opacity))) return MB3DGS_ERR_INVALID_ARG;
    if (P == 0) return MB3DGS_OK;
    count_launch();
    k_vi_opacity<<<adc_grid(P), ADC_TPB, 0, reinterpret_cast<cudaStream_t>(stream)>>>(d_weights, d_scales, P,
                                                                                      d_opacity);
    return cudaGetLastError() == cudaSuccess ? MB3DGS_OK : MB3DGS_ERR_CUDA;
}

extern "C" int mb3dgs_init_weights(const float* d_opacity, const float* d_scales, int64_t P, float* d_weights,
                                   mb3dgs_stream_t stream) {
    if (P < 0 || (P > 0 && (!d_weights || !d_scales || !d_opacity))) return MB3DGS_ERR_INVALID_ARG;
    if (P == 0) return MB3DGS_OK;
    count_launch();
    k_init_weights<<<adc_grid(P), ADC_TPB, 0, reinterpret_cast<cudaStream_t>(stream)>>>(d_opacity, d_scales, P,
                                                                                        d_weights);
    return cudaGetLastError() == cudaSuccess ? MB3DGS_OK : MB3DGS_ERR_CUDA;
}

extern "C" int mb3dgs_accumulate_grad_stats(const float* d_dmeans, const uint8_t* d_visible, int64_t P,
                                            float* d_abs_sum, int32_t* d_count, mb3dgs_stream_t stream) {
    if (P < 0 || (P > 0 && (!d_dmeans || !d_abs_sum || !d_count))) return MB3DGS_ERR_INVALID_ARG;
    if (P == 0) return MB3DGS_OK;
    count_launch();
    k_grad_stats<<<adc_grid(P), ADC_TPB, 0, reinterpret_cast<cudaStream_t>(stream)>>>(d_dmeans, d_visible, P,
                                                                                      d_abs_sum, d_count);
    return cudaGetLastError() == cudaSuccess ? MB3DGS_OK : MB3DGS_ERR_CUDA;
}

extern "C" int mb3dgs_densify_workspace_size(int64_t P, size_t* bytes) {
    if (P < 0 || !bytes) return MB3DGS_ERR_INVALID_ARG;
    *bytes = densify_ws_bytes(P);
    return MB3DGS_OK;
}

extern "C" int mb3dgs_densify(const mb3dgs_adc_config* cfg, const mb3dgs_gaussians* g, const float* d_abs_sum,
                              const int32_t* d_count, void* ws, size_t ws_bytes, const mb3dgs_gaussians_out* out,
                              int64_t* d_P_out, int8_t* d_action, int32_t* d_first, mb3dgs_stream_t stream) {
    AdcParams a;
    int rc = adc_params(cfg, a);
    if (rc) return rc;
    if (!g || !out || !d_P_out || g->P < 0 || g->sh_degree < 0 || g->sh_degree > 3) return MB3DGS_ERR_INVALID_ARG;
    const int64_t P = g->P;
    if (P > (int64_t(1) << 30) || out->capacity < 2 * P) return MB3DGS_ERR_INVALID_ARG;
    if (P > 0 && (!g->means || !g->scales || !g->quats || !g->weights || !g->sh || !d_abs_sum || !d_count ||
                  !out->means || !out->scales || !out->quats || !out->weights || !out->sh || !ws))
        return MB3DGS_ERR_INVALID_ARG;
    if (ws_bytes < densify_ws_bytes(P)) return MB3DGS_ERR_WORKSPACE_TOO_SMALL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (P == 0) {
        if (cudaMemsetAsync(d_P_out, 0, sizeof(int64_t), st) != cudaSuccess) return MB3DGS_ERR_CUDA;
        return MB3DGS_OK;
    }
    char* w = static_cast<char*>(ws);
    int* n_out = reinterpret_cast<int*>(w);
    int* off = reinterpret_cast<int*>(w + align256(sizeof(int) * (size_t)P));
    int* tmp = reinterpret_cast<int*>(w + 2 * align256(sizeof(int) * (size_t)P));
    count_launch();
    k_densify_count<<<adc_grid(P), ADC_TPB, 0, st>>>(a, g->scales, g->weights, d_abs_sum, d_count, P, n_out,
                                                      d_action);
    exclusive_scan(n_out, off, P, tmp, st);
    count_launch();
    k_densify_total<<<1, 1, 0, st>>>(n_out, off, P, d_P_out);
    if (d_first && cudaMemcpyAsync(d_first, off, sizeof(int) * (size_t)P, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return MB3DGS_ERR_CUDA;
    count_launch();
    k_densify_write<<<adc_grid(P), ADC_TPB, 0, st>>>(a, *g, d_abs_sum, d_count, off, *out);
    return cudaGetLastError() == cudaSuccess ? MB3DGS_OK : MB3DGS_ERR_CUDA;
}
