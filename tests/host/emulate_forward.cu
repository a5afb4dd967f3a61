// Host build of the CUDA path's per-pixel forward arithmetic, for the CPU
// regression test (tests/test_host_emulation.py).  It runs the same device
// functions (preprocess_one, pair_gaussian, legendre_moments,
// reconstruct_pixel, pair_quadrature, the Eq. 15 epilogue, and the
// transmittance query optical_depth) compiled for the host, with the host's libm for exp/erf and exact division in place of the
// approximate one.  It covers the arithmetic only: binning, tiling,
// scheduling and every kernel launch are left out (contributing Gaussians are
// found by rectangle tests).
//
// argv[1] = input file (int64 P, int32 sh_degree, float32 SoA means, scales,
// quats, weights, sh, mb3dgs_camera, int32 region x0 y0 w h), argv[2] =
// output file (float32 rgb [h][w][3], T [h][w], T(eta_q) [h][w][17] at the
// warped depths eta_q = q/16), argv[3] (optional) = N intervals (default 3;
// other values run the runtime-N template), argv[4] (optional) = moment basis
// (0 power, 1 trigonometric: trig_moments, reconstruct_trig and the
// trigonometric bound queries), argv[5] (optional) = knots M of the tabulated
// transmittance (power basis; 0: every query solved).
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "../../paper_2512_11800_gb300/csrc/preprocess.cuh"
#include "../../paper_2512_11800_gb300/csrc/api.cu"
#include "../../paper_2512_11800_gb300/csrc/table.cuh"

namespace mb {   // the launchers api.cu refers to; never called here
void launch_preprocess(const Params&, const ViewTable&, const mb3dgs_gaussians&, float*, int*, StatusWords*,
                       cudaStream_t) {}
void launch_binning(const ViewTable&, const Layout&, char*, cudaStream_t) {}
void launch_tile_order(const Layout&, char*, cudaStream_t) {}
size_t scan_tmp_elems(int64_t) { return 0; }
void launch_moments(const Params&, const ViewTable&, const Layout&, char*, cudaStream_t) {}
void launch_moments_to_power(const Params&, const Layout&, char*, float*, cudaStream_t) {}
void launch_reconstruct(const Params&, const Layout&, char*, const float*, int, float*, cudaStream_t) {}
int launch_shade(const Params&, const ViewTable&, const Layout&, char*, float*, float*, float*, cudaStream_t) {
    return 0;
}
int launch_backward_quadrature(const Params&, const ViewTable&, const Layout&, char*, const float*, const float*,
                               const float*, cudaStream_t) { return 0; }
int launch_backward_moments(const Params&, const ViewTable&, const Layout&, char*, cudaStream_t) { return 0; }
int launch_backward_preprocess(const Params&, const ViewTable&, const Layout&, char*, const mb3dgs_gaussians&,
                               const mb3dgs_gaussian_grads&, cudaStream_t) { return 0; }
}  // namespace mb
using namespace mb;

template <class T>
static void rd(FILE* f, T* x, size_t n) {
    if (fread(x, sizeof(T), n, f) != n) {
        fprintf(stderr, "short read\n");
        exit(1);
    }
}

int main(int argc, char** argv) {
    if (argc < 3 || argc > 6) return 2;
    FILE* f = fopen(argv[1], "rb");
    if (!f) return 2;
    int64_t P;
    int deg;
    rd(f, &P, 1);
    rd(f, &deg, 1);
    const int K = (deg + 1) * (deg + 1);
    std::vector<float> means(3 * P), scales(3 * P), quats(4 * P), w(P), sh(P * K * 3);
    rd(f, means.data(), 3 * P);
    rd(f, scales.data(), 3 * P);
    rd(f, quats.data(), 4 * P);
    rd(f, w.data(), P);
    rd(f, sh.data(), P * K * 3);
    mb3dgs_camera cam;
    rd(f, &cam, 1);
    int reg[4];
    rd(f, reg, 4);
    fclose(f);
    mb3dgs_config cfg;
    mb3dgs_config_default(&cfg);
    if (argc >= 4) cfg.n_intervals = atoi(argv[3]);
    if (argc >= 5) cfg.basis = atoi(argv[4]);
    if (argc >= 6) cfg.tau_table = atoi(argv[5]);
    const bool trig = cfg.basis == MB3DGS_BASIS_TRIG;
    Params p;
    make_params(&cfg, p);
    ViewTable vt;
    int64_t npix, nt;
    if (make_views(&cfg, &cam, 1, vt, npix, nt) != MB3DGS_OK) return 3;
    const ViewDesc& V = vt.v[0];
    const int x0 = reg[0], y0 = reg[1], W = reg[2], H = reg[3];
    std::vector<float> rec(P * REC);
    std::vector<int64_t> list;   // visible Gaussians whose rectangle meets the region, ascending id
    for (int64_t i = 0; i < P; ++i) {
        int cnt;
        bool bad;
        preprocess_one(p, V, means.data(), scales.data(), quats.data(), w.data(), sh.data(), i, deg, &rec[i * REC],
                       &cnt, &bad);
        const int* ri = reinterpret_cast<const int*>(&rec[i * REC + R_RECT]);
        if (ri[0] <= ri[2] && ri[2] >= x0 && ri[0] < x0 + W && ri[3] >= y0 && ri[1] < y0 + H) list.push_back(i);
    }
    constexpr int NPROBE = 17;
    std::vector<float> out_rgb(3 * W * H), out_T(W * H), out_probe(NPROBE * W * H);
    for (int q = 0; q < W * H; ++q) {
        const int px = x0 + q % W, py = y0 + q / W;
        const float ux = ((float)px + 0.5f - V.cx) / V.fx, uy = ((float)py + 0.5f - V.cy) / V.fy;
        const float r2 = fmaf(ux, ux, fmaf(uy, uy, 1.0f)), rl = sqrtf(r2);
        float acc[NMOM] = {0};
        for (int64_t i : list) {
            const float* r = &rec[i * REC];
            if (!rect_contains(r, px, py)) continue;
            const Gauss1D g = pair_gaussian(r, (float)px + 0.5f - r[R_AX], (float)py + 0.5f - r[R_AY], rl, r2);
            if (trig) trig_moments(p, g, acc);
            else legendre_moments(p, g, acc);
        }
        Recon R;
        TrigRecon TR;
        if (trig) reconstruct_trig(p, acc, TR);
        else reconstruct_pixel(p, acc, R);
        // tabulated transmittance: this pixel's table (npix = 1 layout)
        const int M = p.tab_m;
        std::vector<float2> tab(M > 0 ? TAB_SEGS * (M + 1) : 1);
        TabPixel TP;
        if (M > 0) {
            table_edges(R, TP.e);
            for (int s = 0; s < TAB_SEGS; ++s)
                for (int i = 0; i <= M; ++i) tab[s * (M + 1) + i] = table_knot(p, R, TP.e, s, i, M);
            TP.m0 = R.m0;
            TP.tab = tab.data();
            TP.pix = 0;
            TP.npix = 1;
            TP.M = M;
        }
        float S[3] = {0, 0, 0}, O = 0, Pen = 0;
        for (int64_t i : list) {
            const float* r = &rec[i * REC];
            if (!rect_contains(r, px, py)) continue;
            const Gauss1D g = pair_gaussian(r, (float)px + 0.5f - r[R_AX], (float)py + 0.5f - r[R_AY], rl, r2);
            float Oi;
            if (trig) Oi = p.n_intervals == 5 ? pair_quadrature<5, false, TrigRecon>(p, TR, g, &Pen)
                                              : pair_quadrature<0, false, TrigRecon>(p, TR, g, &Pen);
            else if (M > 0) Oi = pair_quadrature<0, false, TabPixel>(p, TP, g, &Pen);
            else Oi = p.n_intervals == 3 ? pair_quadrature<3>(p, R, g, &Pen) : pair_quadrature<0>(p, R, g, &Pen);
            for (int c = 0; c < 3; ++c) S[c] += r[R_RGB + c] * Oi;
            O += Oi;
        }
        const float m0 = acc[0], Tf = expf(-m0), sc = -expm1f(-m0) / fmaxf(p.eps, O);
        for (int c = 0; c < 3; ++c) out_rgb[3 * q + c] = sc * S[c] + Tf * p.bg[c];
        out_T[q] = Tf;
        for (int k = 0; k < NPROBE; ++k)
            out_probe[q * NPROBE + k] = trig ? expf(-trig_optical_depth(p, TR, (float)k / 16.0f))
                                      : M > 0 ? expf(-table_depth(TP, (float)k / 16.0f))
                                             : expf(-optical_depth(R, p.beta, 2.0f * ((float)k / 16.0f) - 1.0f));
    }
    FILE* o = fopen(argv[2], "wb");
    if (!o) return 2;
    fwrite(out_rgb.data(), 4, out_rgb.size(), o);
    fwrite(out_T.data(), 4, out_T.size(), o);
    fwrite(out_probe.data(), 4, out_probe.size(), o);
    fclose(o);
    return 0;
}
