// Host build of the CUDA path's backward arithmetic, for the CPU regression
// test (tests/test_host_emulation.py).  Per pixel it runs, compiled for the
// host, the device functions the kernels run:
//   forward: pair_quadrature;
//   pass 1: pixel_adjoint, pair_backward, geometry_adjoint_compact,
//           phi_monomials, finish_moment_adjoint (trig_finish_adjoint);
//   pass 2: moment_adjoint (trig_moment_adjoint), geometry_adjoint_compact;
//   per record: expand_geometry, preprocess_bwd_one.
// The per-record sums are plain host sums in place of the warp, shared-memory
// and global reductions; binning, tiling and launches are left out.  With
// argv[3] == "saved" the bound queries kept by the forward feed pass 1
// ("compact": kept in the 8-byte form and restored by pass 1), else pass 1
// solves them again.  argv[4] (optional): N intervals (default 3; other
// values run the runtime-N templates).  argv[5] (optional): moment basis (0
// power, 1 trigonometric: trig_moments, reconstruct_trig, the trigonometric
// pair_backward, trig_finish_adjoint and trig_moment_adjoint; "saved" keeps
// their queries in the 16-byte trigonometric form).
//
// argv[1]: input file (as for emulate_forward, then float32 dL/drgb [h][w][3]
// and dL/dP [h][w] of the region); argv[2]: output file (float32 gradients of
// means, scales, quats, weights, sh, in that order).
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>
#include "../../paper_2512_11800_gb300/csrc/api.cu"
#include "../../paper_2512_11800_gb300/csrc/backward.cu"

namespace mb {   // launchers and schedule helpers referenced by api.cu / backward.cu; never called here
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
TileLaunch tile_launch(const Params&, const Layout&, char*, int, const void*, size_t, cudaStream_t) {
    return TileLaunch{};
}
bool allow_dynamic_smem(const void*, size_t) { return false; }
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
    if (argc < 4 || argc > 6) return 2;
    const bool compact = strcmp(argv[3], "compact") == 0;
    const bool saved = compact || strcmp(argv[3], "saved") == 0;
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
    const int x0 = reg[0], y0 = reg[1], W = reg[2], H = reg[3];
    std::vector<float> dl_rgb(3 * W * H), dl_P(W * H);
    rd(f, dl_rgb.data(), dl_rgb.size());
    rd(f, dl_P.data(), dl_P.size());
    fclose(f);
    mb3dgs_config cfg;
    mb3dgs_config_default(&cfg);
    if (argc >= 5) cfg.n_intervals = atoi(argv[4]);
    if (argc >= 6) cfg.basis = atoi(argv[5]);
    const bool trig = cfg.basis == MB3DGS_BASIS_TRIG;
    Params p;
    make_params(&cfg, p);
    ViewTable vt;
    int64_t npix, nt;
    if (make_views(&cfg, &cam, 1, vt, npix, nt) != MB3DGS_OK) return 3;
    const ViewDesc& V = vt.v[0];
    std::vector<float> rec(P * REC);
    std::vector<int64_t> list;
    for (int64_t i = 0; i < P; ++i) {
        int cnt;
        bool bad;
        preprocess_one(p, V, means.data(), scales.data(), quats.data(), w.data(), sh.data(), i, deg, &rec[i * REC],
                       &cnt, &bad);
        const int* ri = reinterpret_cast<const int*>(&rec[i * REC + R_RECT]);
        if (ri[0] <= ri[2] && ri[2] >= x0 && ri[0] < x0 + W && ri[3] >= y0 && ri[1] < y0 + H) list.push_back(i);
    }
    std::vector<double> s_quad(P * NK_QUAD, 0.0), s_mom(P * NK_MOM, 0.0);
    const int nq = p.n_intervals + 1;
    for (int q = 0; q < W * H; ++q) {
        const int px = x0 + q % W, py = y0 + q / W;
        const float ux = ((float)px + 0.5f - V.cx) / V.fx, uy = ((float)py + 0.5f - V.cy) / V.fy;
        const float r2 = fmaf(ux, ux, fmaf(uy, uy, 1.0f)), rl = sqrtf(r2);
        const float fpx = (float)px + 0.5f, fpy = (float)py + 0.5f;
        std::vector<int64_t> mine;
        for (int64_t i : list)
            if (rect_contains(&rec[i * REC], px, py)) mine.push_back(i);
        // forward of the pixel
        float acc[NMOM] = {0};
        for (int64_t i : mine) {
            const float* r = &rec[i * REC];
            const Gauss1D g = pair_gaussian(r, fpx - r[R_AX], fpy - r[R_AY], rl, r2);
            if (trig) trig_moments(p, g, acc);
            else legendre_moments(p, g, acc);
        }
        Recon R;
        TrigRecon TR;
        if (trig) reconstruct_trig(p, acc, TR);
        else reconstruct_pixel(p, acc, R);
        float S[3] = {0, 0, 0}, O = 0, Pen = 0;
        std::vector<float4> qs16(mine.size() * nq);   // 16 bytes a query (8 used when compact)
        char* qs = reinterpret_cast<char*>(qs16.data());
        const int QBY = compact ? 8 : 16;
        for (size_t k = 0; k < mine.size(); ++k) {
            const float* r = &rec[mine[k] * REC];
            const Gauss1D g = pair_gaussian(r, fpx - r[R_AX], fpy - r[R_AY], rl, r2);
            const float Oi = trig ? (saved ? pair_quadrature<0, true, TrigRecon>(p, TR, g, &Pen, qs + k * nq * 16)
                                           : pair_quadrature<0, false, TrigRecon>(p, TR, g, &Pen))
                             : compact ? (p.n_intervals == 3 ? pair_quadrature<3, true, Recon, 8>(p, R, g, &Pen, qs + k * nq * QBY)
                                                             : pair_quadrature<0, true, Recon, 8>(p, R, g, &Pen, qs + k * nq * QBY))
                             : p.n_intervals == 3 ? pair_quadrature<3, true>(p, R, g, &Pen, qs + k * nq * QBY)
                                                  : pair_quadrature<0, true>(p, R, g, &Pen, qs + k * nq * QBY);
            for (int c = 0; c < 3; ++c) S[c] += r[R_RGB + c] * Oi;
            O += Oi;
        }
        // pass 1
        const float gimg[3] = {dl_rgb[3 * q], dl_rgb[3 * q + 1], dl_rgb[3 * q + 2]};
        const PixelAdj pa = pixel_adjoint(p, acc[0], S, O, gimg, dl_P[q]);
        float B[NB];
        for (int k = 0; k < NB; ++k) B[k] = 0.0f;
        for (size_t k = 0; k < mine.size(); ++k) {
            const float* r = &rec[mine[k] * REC];
            const float dx = fpx - r[R_AX], dy = fpy - r[R_AY];
            const Gauss1D g = pair_gaussian(r, dx, dy, rl, r2);
            const float a = pa.gS[0] * r[R_RGB] + pa.gS[1] * r[R_RGB + 1] + pa.gS[2] * r[R_RGB + 2] + pa.gO;
            PairOut po;
            if (trig)
                po = saved ? pair_backward<0, true, TrigRecon>(p, TR, g, a, pa.gP, B, qs + k * nq * 16)
                           : pair_backward<0, false, TrigRecon>(p, TR, g, a, pa.gP, B);
            else if (p.n_intervals == 3)
                po = compact ? pair_backward<3, true, Recon, 8>(p, R, g, a, pa.gP, B, qs + k * nq * QBY)
                   : saved ? pair_backward<3, true>(p, R, g, a, pa.gP, B, qs + k * nq * QBY)
                           : pair_backward<3, false>(p, R, g, a, pa.gP, B);
            else
                po = compact ? pair_backward<0, true, Recon, 8>(p, R, g, a, pa.gP, B, qs + k * nq * QBY)
                   : saved ? pair_backward<0, true>(p, R, g, a, pa.gP, B, qs + k * nq * QBY)
                           : pair_backward<0, false>(p, R, g, a, pa.gP, B);
            float c[NK_QUAD];
            for (int f2 = 0; f2 < NK_QUAD; ++f2) c[f2] = 0.0f;
            geometry_adjoint_compact(r, dx, dy, rl, g, po.g_mu, po.g_Sig, po.g_what, c);
            for (int ch = 0; ch < 3; ++ch) c[K_RGB + ch] = pa.gS[ch] * po.O;
            for (int f2 = 0; f2 < NK_QUAD; ++f2) s_quad[mine[k] * NK_QUAD + f2] += c[f2];
        }
        float psi[NPOLY];
        if (trig) {
            trig_finish_adjoint(p, acc, B, pa.gm0, psi);
        } else {
            phi_monomials(R, B, psi);
            finish_moment_adjoint(p, R, pa.gm0, psi);
        }
        // pass 2
        for (int64_t i : mine) {
            const float* r = &rec[i * REC];
            const float dx = fpx - r[R_AX], dy = fpy - r[R_AY];
            const Gauss1D g = pair_gaussian(r, dx, dy, rl, r2);
            float g_mu = 0.0f, g_Sig = 0.0f, g_what = 0.0f;
            if (trig) trig_moment_adjoint(p, g, psi, &g_mu, &g_Sig, &g_what);
            else moment_adjoint(p, R, g, psi, &g_mu, &g_Sig, &g_what);
            float c[NK_MOM];
            for (int f2 = 0; f2 < NK_MOM; ++f2) c[f2] = 0.0f;
            geometry_adjoint_compact(r, dx, dy, rl, g, g_mu, g_Sig, g_what, c);
            for (int f2 = 0; f2 < NK_MOM; ++f2) s_mom[i * NK_MOM + f2] += c[f2];
        }
    }
    // per record: expand the compact sums, then the preprocessing adjoint
    std::vector<float> grec(P * GSTRIDE, 0.0f);
    for (int64_t i : list) {
        float sq[NK_QUAD], sm[NK_MOM];
        for (int f2 = 0; f2 < NK_QUAD; ++f2) sq[f2] = (float)s_quad[i * NK_QUAD + f2];
        for (int f2 = 0; f2 < NK_MOM; ++f2) sm[f2] = (float)s_mom[i * NK_MOM + f2];
        for (int f2 = 0; f2 < NGRAD; ++f2) {
            float v = expand_geometry(&rec[i * REC], sq, f2);
            if (f2 < G_RGB) v += expand_geometry(&rec[i * REC], sm, f2);
            grec[i * GSTRIDE + f2] = v;
        }
    }
    std::vector<float> d_means(3 * P, 0.0f), d_scales(3 * P, 0.0f), d_quats(4 * P, 0.0f), d_w(P, 0.0f),
        d_sh(P * K * 3, 0.0f);
    for (int64_t i = 0; i < P; ++i)
        preprocess_bwd_one<float>(p, vt, means.data(), scales.data(), quats.data(), w.data(), sh.data(), P, deg,
                                  rec.data(), grec.data(), i, d_means.data(), d_scales.data(), d_quats.data(),
                                  d_w.data(), d_sh.data());
    FILE* o = fopen(argv[2], "wb");
    if (!o) return 2;
    fwrite(d_means.data(), 4, d_means.size(), o);
    fwrite(d_scales.data(), 4, d_scales.size(), o);
    fwrite(d_quats.data(), 4, d_quats.size(), o);
    fwrite(d_w.data(), 4, d_w.size(), o);
    fwrite(d_sh.data(), 4, d_sh.size(), o);
    fclose(o);
    return 0;
}
