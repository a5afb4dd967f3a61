// Stage 1: per (view, Gaussian) preprocessing in FP64.
//
// Culling (Sec. 3.3: bounding sphere r = r_mult * max diag(S)), the
// confidence-interval proxy (Eq. 17-21, App. C), SH emission (Sec. 3.1) and
// the coefficients of the ray-parameterised Gaussian (Eq. 4-6, App. A) in a
// form whose per-pixel evaluation is well conditioned in FP32:
//   d_g(p) = S^-1 R^T K^-1 (p, 1) = g_a + dx m_x + dy m_y   (dx, dy: pixel offset
//   from an anchor pixel centre), o_g = S^-1 R^T (o - mu) = -S^-1 R^T mu_c,
//   o_g x d_g = c0 + dx cx + dy cy,  |d_g|^2 quadratic in (dx, dy),
//   o_g . d_g linear in (dx, dy).
// With d = d_g / |K^-1 (p,1)|: Sigma^2 = |K^-1 p|^2 / |d_g|^2,
// mu = -(o_g.d_g) |K^-1 p| / |d_g|^2, K = -|o_g x d_g|^2 / (2 |d_g|^2).
#include "preprocess.cuh"

namespace mb {

__global__ void k_preprocess(Params p, ViewTable vt, const float* __restrict__ means,
                             const float* __restrict__ scales, const float* __restrict__ quats,
                             const float* __restrict__ weights, const float* __restrict__ sh, int64_t P,
                             int sh_deg, float* __restrict__ rec, int* __restrict__ counts, StatusWords* sw) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long area = 0;
    if (idx < P * vt.n_views) {
        const int v = (int)(idx / P);
        const int64_t i = idx - (int64_t)v * P;
        bool bad = false;
        int cnt = 0;
        float* r = rec + idx * REC;
        preprocess_one(p, vt.v[v], means, scales, quats, weights, sh, i, sh_deg, r, &cnt, &bad);
        counts[idx] = cnt;
        const int* ri = reinterpret_cast<const int*>(r);
        if (cnt > 0)
            area = (unsigned long long)(ri[R_RECT + 2] - ri[R_RECT + 0] + 1) *
                   (unsigned long long)(ri[R_RECT + 3] - ri[R_RECT + 1] + 1);
        if (bad) {
            atomicAdd(&sw->nonfinite, 1ull);
            if (p.strict) set_status(&sw->status, MB3DGS_ERR_NUMERIC);
        }
    }
    // (pixel, Gaussian) pairs: the clipped rectangle's pixel count
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) area += __shfl_xor_sync(0xffffffffu, area, o);
    if ((threadIdx.x & 31) == 0 && area) atomicAdd(&sw->n_pixpairs, area);
}

void launch_preprocess(const Params& p, const ViewTable& vt, const mb3dgs_gaussians& g, float* rec, int* counts,
                       StatusWords* sw, cudaStream_t st) {
    const int64_t n = g.P * vt.n_views;
    if (n == 0) return;
    const int tpb = 128;
    count_launch();
    k_preprocess<<<(unsigned)ceil_div64(n, tpb), tpb, 0, st>>>(p, vt, g.means, g.scales, g.quats, g.weights, g.sh,
                                                              g.P, g.sh_degree, rec, counts, sw);
}

}  // namespace mb
