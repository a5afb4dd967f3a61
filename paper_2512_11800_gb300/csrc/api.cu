// C ABI entry points (include/mb3dgs.h): argument validation, workspace
// layout, kernel parameters and launch order.  No device allocation.
#include <cmath>
#include <atomic>
#include <cstring>
#include <mutex>

#include "common.cuh"

namespace mb {
void launch_preprocess(const Params&, const ViewTable&, const mb3dgs_gaussians&, float*, int*, StatusWords*,
                       cudaStream_t);
void launch_binning(const ViewTable&, const Layout&, char*, cudaStream_t);
void launch_tile_order(const Layout&, char*, cudaStream_t);
size_t scan_tmp_elems(int64_t);
void launch_moments(const Params&, const ViewTable&, const Layout&, char*, cudaStream_t);
void launch_moments_to_power(const Params&, const Layout&, char*, float*, cudaStream_t);
void launch_reconstruct(const Params&, const Layout&, char*, const float*, int, float*, cudaStream_t);
int launch_shade(const Params&, const ViewTable&, const Layout&, char*, float*, float*, float*, cudaStream_t);
int launch_backward_quadrature(const Params&, const ViewTable&, const Layout&, char*, const float*, const float*,
                               const float*,
                               cudaStream_t);
int launch_backward_moments(const Params&, const ViewTable&, const Layout&, char*, cudaStream_t);
int launch_backward_preprocess(const Params&, const ViewTable&, const Layout&, char*, const mb3dgs_gaussians&,
                               const mb3dgs_gaussian_grads&, cudaStream_t);

static std::atomic<long long> g_launches{0};
void count_launch(int n) { g_launches += n; }

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
static size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Phi^-1(p) by bisection + Newton on Phi(x) = erfc(-x / sqrt 2) / 2 (double)
static double inv_normal_cdf(double p) {
    double lo = -12.0, hi = 12.0;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (0.5 * std::erfc(-mid / std::sqrt(2.0)) < p) lo = mid; else hi = mid;
    }
    double x = 0.5 * (lo + hi);
    for (int it = 0; it < 3; ++it) {
        const double f = 0.5 * std::erfc(-x / std::sqrt(2.0)) - p;
        const double d = std::exp(-0.5 * x * x) / std::sqrt(2.0 * M_PI);
        x -= f / d;
    }
    return x;
}

static int check_cfg(const mb3dgs_config* c) {
    if (!c) return MB3DGS_ERR_INVALID_ARG;
    if (c->n != 4) return MB3DGS_ERR_UNSUPPORTED;
    if (c->n_intervals < 1 || c->n_intervals > MAX_NODES - 1) return MB3DGS_ERR_UNSUPPORTED;
    if (!(c->kappa > 0) || !(c->beta >= 0 && c->beta <= 1) || !(c->conf_c > 0 && c->conf_c < 1) ||
        !(c->t_near > 0) || !(c->t_far > c->t_near) || !(c->eps > 0) || !(c->bias_alpha >= 0 && c->bias_alpha < 1) ||
        !(c->m_min >= 0) || !(c->r_mult > 0) || c->warp_lambda == 0.0f || c->warp_lambda == 1.0f)
        return MB3DGS_ERR_INVALID_ARG;
    if (c->moment_dtype < 0 || c->moment_dtype > 2) return MB3DGS_ERR_INVALID_ARG;
    if (c->basis != MB3DGS_BASIS_POWER && c->basis != MB3DGS_BASIS_TRIG) return MB3DGS_ERR_INVALID_ARG;
    if (c->basis == MB3DGS_BASIS_TRIG && !(c->trig_theta > 0.0f && c->trig_theta < (float)(2.0 * M_PI)))
        return MB3DGS_ERR_INVALID_ARG;
    if (c->tau_table != 0 && (c->tau_table < 8 || c->tau_table > 128)) return MB3DGS_ERR_INVALID_ARG;
    if (c->compact_queries != 0 && c->compact_queries != 1) return MB3DGS_ERR_INVALID_ARG;
    if (c->compact_queries && c->basis != MB3DGS_BASIS_POWER) return MB3DGS_ERR_UNSUPPORTED;   // power-moment roots only
    if (c->tau_table != 0 && c->basis != MB3DGS_BASIS_POWER) return MB3DGS_ERR_UNSUPPORTED;
    if (c->tile_w != 0 || c->tile_h != 0) {
        const int tw = c->tile_w, th = c->tile_h;
        if (!(tw == 8 || tw == 16 || tw == 32 || tw == 64) || tw * th != TPB) return MB3DGS_ERR_UNSUPPORTED;
    }
    if (c->batch < 0 || c->batch > TPB || c->batch % 32 != 0) return MB3DGS_ERR_UNSUPPORTED;
    if (c->schedule != MB3DGS_SCHEDULE_QUEUE && c->schedule != MB3DGS_SCHEDULE_GRID) return MB3DGS_ERR_INVALID_ARG;
    return MB3DGS_OK;
}

static void tile_shape(const mb3dgs_config* cfg, int& tw, int& th) {
    tw = cfg && cfg->tile_w > 0 ? cfg->tile_w : 16;
    th = cfg && cfg->tile_h > 0 ? cfg->tile_h : 16;
}

static int make_views(const mb3dgs_config* cfg, const mb3dgs_camera* cams, int n_views, ViewTable& vt,
                      int64_t& npix, int64_t& ntiles) {
    if (!cams || n_views < 1 || n_views > MB3DGS_MAX_VIEWS) return MB3DGS_ERR_INVALID_ARG;
    int tw, th;
    tile_shape(cfg, tw, th);
    std::memset(&vt, 0, sizeof(vt));
    vt.n_views = n_views;
    npix = 0;
    ntiles = 0;
    for (int v = 0; v < n_views; ++v) {
        const mb3dgs_camera& c = cams[v];
        if (c.width <= 0 || c.height <= 0 || c.width > 65536 || c.height > 65536 || !(c.fx > 0) || !(c.fy > 0))
            return MB3DGS_ERR_INVALID_ARG;
        ViewDesc& d = vt.v[v];
        for (int a = 0; a < 3; ++a) {
            for (int b = 0; b < 3; ++b) d.R[3 * a + b] = c.viewmat[4 * a + b];
            d.t[a] = c.viewmat[4 * a + 3];
        }
        d.fx = c.fx; d.fy = c.fy; d.cx = c.cx; d.cy = c.cy;
        d.width = c.width; d.height = c.height;
        d.tile_w = tw;
        d.tile_h = th;
        d.tiles_x = (c.width + tw - 1) / tw;
        d.tiles_y = (c.height + th - 1) / th;
        d.tile_base = (int)ntiles;
        d.pixel_base = npix;
        ntiles += (int64_t)d.tiles_x * d.tiles_y;
        npix += (int64_t)c.width * c.height;
    }
    if (ntiles >= (int64_t(1) << 31)) return MB3DGS_ERR_INVALID_ARG;
    return MB3DGS_OK;
}

static int make_layout(const mb3dgs_config* cfg, const ViewTable& vt, int64_t npix, int64_t ntiles, int64_t P,
                       int64_t cap, Layout& L) {
    if (P < 0 || cap < 0 || cap >= (int64_t(1) << 31)) return MB3DGS_ERR_INVALID_ARG;
    std::memset(&L, 0, sizeof(L));
    L.P = P;
    L.VP = P * vt.n_views;
    if (L.VP >= (int64_t(1) << 31)) return MB3DGS_ERR_INVALID_ARG;
    L.npix = npix;
    L.cap = cap;
    L.n_tiles = ntiles;
    L.n_views = vt.n_views;
    L.nb_sort = (int)std::max<int64_t>(1, ceil_div64(cap, 4096));
    int bits = 0;
    while ((int64_t(1) << bits) < ntiles) ++bits;
    L.sort_passes = (bits + 7) / 8;
    L.final_buf = L.sort_passes % 2;
    L.qcap = cfg && cfg->tau_table == 0 ? cfg->query_capacity : 0;
    if (L.qcap < 0 || L.qcap >= (int64_t(1) << 40)) return MB3DGS_ERR_INVALID_ARG;
    L.scan_tmp_elems = std::max(scan_tmp_elems(L.VP), scan_tmp_elems((int64_t)256 * L.nb_sort));
    if (L.qcap > 0) L.scan_tmp_elems = std::max(L.scan_tmp_elems, 2 * scan_tmp_elems(npix));   // 64-bit scan
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o = align256(o + bytes); return r; };
    L.status = take(64);
    L.rec = take(sizeof(float) * REC * (size_t)L.VP);
    L.counts = take(sizeof(int) * (size_t)L.VP);
    L.offsets = take(sizeof(int) * (size_t)L.VP);
    L.scan_tmp = take(sizeof(int) * L.scan_tmp_elems);
    L.keys[0] = take(sizeof(uint32_t) * (size_t)cap);
    L.keys[1] = take(sizeof(uint32_t) * (size_t)cap);
    L.vals[0] = take(sizeof(int32_t) * (size_t)cap);
    L.vals[1] = take(sizeof(int32_t) * (size_t)cap);
    L.hist = take(sizeof(uint32_t) * 256 * (size_t)L.nb_sort);
    L.ranges = take(sizeof(int) * 2 * (size_t)ntiles);
    L.order = take(sizeof(int) * (size_t)ntiles);
    L.sched = take(SCHED_BYTES);
    const int md = cfg ? cfg->moment_dtype : 0;
    // 16-bit storage: m0 plane (FP32) then one 16-byte vector of 8 halves per pixel; the
    // plane is padded to 16 bytes so that the vectors are aligned
    L.moments = take(md == MB3DGS_MOMENTS_F32 ? sizeof(float) * NMOM * (size_t)npix
                                              : align16(sizeof(float) * (size_t)npix) + 16 * (size_t)npix);
    L.recon = take(sizeof(float) * RECON * (size_t)npix);
    L.saved = take(sizeof(float) * 4 * (size_t)npix);
    L.dm = take(sizeof(float) * NMOM * (size_t)npix);
    L.grec = take(sizeof(float) * 28 * (size_t)L.VP);
    L.tab_m = cfg && cfg->basis == MB3DGS_BASIS_POWER ? cfg->tau_table : 0;
    if (L.tab_m > 0) {
        L.tab_e = take(sizeof(float) * 4 * (size_t)npix);
        L.tab = take(sizeof(float) * 2 * TAB_SEGS * (size_t)(L.tab_m + 1) * (size_t)npix);
    }
    if (L.qcap > 0) {
        L.npp = take(sizeof(int) * (size_t)npix);
        L.pq_off = take(sizeof(long long) * (size_t)npix);
        const size_t qb = cfg->compact_queries ? 8 : 16;   // bytes a query
        L.pq = take(qb * (size_t)(cfg->n_intervals + 1) * (size_t)L.qcap);
    }
    L.total = o;
    return MB3DGS_OK;
}

static void make_params(const mb3dgs_config* c, Params& p) {
    std::memset(&p, 0, sizeof(p));
    p.n_intervals = c->n_intervals;
    p.batch = c->batch > 0 ? c->batch : TPB;
    p.schedule = c->schedule;
    p.kappa = c->kappa; p.beta = c->beta; p.conf_c = c->conf_c; p.t_near = c->t_near; p.t_far = c->t_far;
    p.eps = c->eps; p.bias_alpha = c->bias_alpha; p.m_min = c->m_min; p.r_mult = c->r_mult;
    for (int k = 0; k < 3; ++k) p.bg[k] = c->bg[k];
    p.warp_lambda = c->warp_lambda;
    const double lam = c->warp_lambda, a = std::fabs(lam - 1.0);
    auto f = [&](double x) { return (a / lam) * (std::pow(x / a + 1.0, lam) - 1.0); };
    const double fn = f(2.0 * c->t_near), ff = f(2.0 * c->t_far);
    const double G1 = (a / lam) / (ff - fn);
    p.G1 = (float)G1;
    p.G0 = (float)((-a / lam - fn) / (ff - fn));
    p.G2 = (float)(G1 * lam * 2.0 / a);
    p.G3 = (float)(G1 * lam * 2.0 / a * (lam - 1.0) * 2.0 / a);
    {
        const double r1 = std::sqrt(5.0 - 2.0 * std::sqrt(10.0 / 7.0)) / 3.0;
        const double r2 = std::sqrt(5.0 + 2.0 * std::sqrt(10.0 / 7.0)) / 3.0;
        const double w1 = (322.0 + 13.0 * std::sqrt(70.0)) / 900.0, w2 = (322.0 - 13.0 * std::sqrt(70.0)) / 900.0;
        const double ys[5] = {-r2, -r1, 0.0, r1, r2}, ws[5] = {w2, w1, 128.0 / 225.0, w1, w2};
        for (int m = 0; m < 5; ++m) { p.gl_y[m] = (float)ys[m]; p.gl_w[m] = (float)(0.5 * ws[m]); }
    }
    p.two_over_a = (float)(2.0 / a);
    p.lam_is_m15 = c->warp_lambda == -1.5f;
    const int N = c->n_intervals;
    for (int j = 0; j <= N; ++j) {
        p.x_nodes[j] = (float)inv_normal_cdf((j + 0.5) / (N + 1));
        const double b = (double)p.kappa * (double)p.x_nodes[j] / std::sqrt(2.0);
        p.x_erf[j] = (float)std::erf(b);
        p.x_gau[j] = (float)std::exp(-b * b);
    }
    const double pi = M_PI;
    const double c0 = 0.5 / std::sqrt(pi), c1 = std::sqrt(3.0 / (4.0 * pi)), c2 = 0.5 * std::sqrt(15.0 / pi),
                 c20 = 0.25 * std::sqrt(5.0 / pi), c22 = 0.25 * std::sqrt(15.0 / pi),
                 c33 = 0.25 * std::sqrt(35.0 / (2.0 * pi)), c32 = 0.5 * std::sqrt(105.0 / pi),
                 c31 = 0.25 * std::sqrt(21.0 / (2.0 * pi)), c30 = 0.25 * std::sqrt(7.0 / pi),
                 c32b = 0.25 * std::sqrt(105.0 / pi);
    const double shc[16] = {c0, c1, c1, c1, c2, c2, c20, c2, c22, c33, c32, c31, c30, c31, c32b, c33};
    for (int k = 0; k < 16; ++k) p.sh_c[k] = (float)shc[k];
    // u^k = ((1 + y)/2)^k in the Legendre basis: y^j -> Legendre by y P_l = ((l+1) P_{l+1} + l P_{l-1})/(2l+1)
    double ypow[NMOM][NMOM] = {};  // ypow[j][l]: y^j = sum_l ypow[j][l] P_l
    ypow[0][0] = 1.0;
    for (int j = 0; j + 1 < NMOM; ++j)
        for (int l = 0; l < NMOM; ++l) {
            const double cf = ypow[j][l];
            if (cf == 0.0) continue;
            if (l + 1 < NMOM) ypow[j + 1][l + 1] += cf * (l + 1) / (2.0 * l + 1);
            if (l >= 1) ypow[j + 1][l - 1] += cf * l / (2.0 * l + 1);
        }
    for (int k = 0; k < NMOM; ++k) {
        double binom = 1.0;
        for (int j = 0; j <= k; ++j) {
            if (j > 0) binom = binom * (k - j + 1) / j;
            for (int l = 0; l < NMOM; ++l) p.leg_to_pow[k * NMOM + l] += (float)(binom * ypow[j][l] / std::pow(2.0, k));
        }
    }
    p.strict = c->strict;
    p.moment_dtype = c->moment_dtype;
    p.basis = c->basis;
    p.tab_m = c->basis == MB3DGS_BASIS_POWER ? c->tau_table : 0;
    p.qbytes = c->compact_queries ? 8 : 16;
    if (c->basis == MB3DGS_BASIS_TRIG) {
        const double A = 2.0 * M_PI - (double)c->trig_theta;
        p.trig_A = (float)A;
        p.trig_lo = (float)(-0.5 * (double)c->trig_theta);
        // c*_k = (e^{i k A} - 1) / (i k A): moments of the uniform distribution on [0, A]
        for (int k = 1; k <= 4; ++k) {
            const double ka = k * A;
            p.cstar_re[k - 1] = (float)(std::sin(ka) / ka);
            p.cstar_im[k - 1] = (float)((1.0 - std::cos(ka)) / ka);
        }
    }
}

struct Ctx {
    Params p;
    ViewTable vt;
    Layout L;
};

static int setup(const mb3dgs_config* cfg, const mb3dgs_camera* cams, int n_views, int64_t P, int64_t cap,
                 size_t ws_bytes, const void* ws, Ctx& c) {
    int rc = check_cfg(cfg);
    if (rc) return rc;
    int64_t npix, ntiles;
    rc = make_views(cfg, cams, n_views, c.vt, npix, ntiles);
    if (rc) return rc;
    rc = make_layout(cfg, c.vt, npix, ntiles, P, cap, c.L);
    if (rc) return rc;
    if (ws == nullptr && c.L.total > 0) return MB3DGS_ERR_INVALID_ARG;
    if (ws_bytes < c.L.total) return MB3DGS_ERR_WORKSPACE_TOO_SMALL;
    make_params(cfg, c.p);
    return MB3DGS_OK;
}

static thread_local const char* g_last_cuda_error = "no error";
static int cuda_ok() {
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) return MB3DGS_OK;
    g_last_cuda_error = cudaGetErrorString(e);
    return MB3DGS_ERR_CUDA;
}

}  // namespace mb

using namespace mb;

extern "C" {

const char* mb3dgs_status_string(int code) {
    switch (code) {
        case MB3DGS_OK: return "ok";
        case MB3DGS_ERR_INVALID_ARG: return "invalid argument";
        case MB3DGS_ERR_CUDA: return "CUDA error";
        case MB3DGS_ERR_WORKSPACE_TOO_SMALL: return "workspace too small";
        case MB3DGS_ERR_TIMEOUT: return "device wait timed out";
        case MB3DGS_ERR_NUMERIC: return "non-finite Gaussian parameters";
        case MB3DGS_ERR_UNSUPPORTED: return "unsupported configuration";
        case MB3DGS_ERR_CAPACITY: return "tile-pair capacity exceeded";
        default: return "unknown status";
    }
}

const char* mb3dgs_last_cuda_error(void) { return g_last_cuda_error; }

int mb3dgs_config_default(mb3dgs_config* c) {
    if (!c) return MB3DGS_ERR_INVALID_ARG;
    std::memset(c, 0, sizeof(*c));
    c->n = 4;
    c->n_intervals = 3;
    c->kappa = 3.0f;
    c->beta = 0.25f;
    c->conf_c = 0.01f;
    c->warp_lambda = -1.5f;
    c->t_near = 0.01f;
    c->t_far = 1.0e6f;
    c->eps = 1.0e-6f;
    c->bias_alpha = 1.0e-3f;
    c->m_min = 1.0e-7f;
    c->r_mult = 3.0f;
    c->moment_dtype = MB3DGS_MOMENTS_F32;
    c->strict = 0;
    c->basis = MB3DGS_BASIS_POWER;
    c->trig_theta = (float)(0.5 * M_PI);
    return MB3DGS_OK;
}

int64_t mb3dgs_launch_count(void) { return (int64_t)g_launches.load(); }

int64_t mb3dgs_num_tiles(const mb3dgs_config* cfg, const mb3dgs_camera* cams, int n_views) {
    if (cfg && check_cfg(cfg)) return -1;
    ViewTable vt;
    int64_t npix, nt;
    if (make_views(cfg, cams, n_views, vt, npix, nt)) return -1;
    return nt;
}

int mb3dgs_workspace_size(const mb3dgs_config* cfg, const mb3dgs_camera* cams, int n_views, int64_t P,
                          int64_t pair_capacity, size_t* bytes) {
    if (!bytes) return MB3DGS_ERR_INVALID_ARG;
    Ctx c;
    int rc = check_cfg(cfg);
    if (rc) return rc;
    int64_t npix, nt;
    rc = make_views(cfg, cams, n_views, c.vt, npix, nt);
    if (rc) return rc;
    rc = make_layout(cfg, c.vt, npix, nt, P, pair_capacity, c.L);
    if (rc) return rc;
    *bytes = c.L.total;
    return MB3DGS_OK;
}

int mb3dgs_preprocess(const mb3dgs_config* cfg, const mb3dgs_gaussians* g, const mb3dgs_camera* cams, int n_views,
                      void* ws, size_t ws_bytes, int64_t pair_capacity, mb3dgs_stream_t stream) {
    if (!g || g->P < 0 || g->sh_degree < 0 || g->sh_degree > 3) return MB3DGS_ERR_INVALID_ARG;
    if (g->P > 0 && (!g->means || !g->scales || !g->quats || !g->weights || !g->sh)) return MB3DGS_ERR_INVALID_ARG;
    Ctx c;
    int rc = setup(cfg, cams, n_views, g->P, pair_capacity, ws_bytes, ws, c);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char* w = static_cast<char*>(ws);
    if (cudaMemsetAsync(w + c.L.status, 0, 64, st) != cudaSuccess) return MB3DGS_ERR_CUDA;
    StatusWords* sw = reinterpret_cast<StatusWords*>(w + c.L.status);
    launch_preprocess(c.p, c.vt, *g, reinterpret_cast<float*>(w + c.L.rec), reinterpret_cast<int*>(w + c.L.counts),
                      sw, st);
    return cuda_ok();
}

int mb3dgs_bin_tiles(const mb3dgs_config* cfg, const mb3dgs_camera* cams, int n_views, int64_t P,
                     int64_t pair_capacity, void* ws, size_t ws_bytes, mb3dgs_stream_t stream) {
    Ctx c;
    int rc = setup(cfg, cams, n_views, P, pair_capacity, ws_bytes, ws, c);
    if (rc) return rc;
    launch_binning(c.vt, c.L, static_cast<char*>(ws), reinterpret_cast<cudaStream_t>(stream));
    if (c.p.schedule == MB3DGS_SCHEDULE_QUEUE)
        launch_tile_order(c.L, static_cast<char*>(ws), reinterpret_cast<cudaStream_t>(stream));
    return cuda_ok();
}

int mb3dgs_accumulate_moments(const mb3dgs_config* cfg, const mb3dgs_camera* cams, int n_views, int64_t P,
                              int64_t pair_capacity, void* ws, size_t ws_bytes, float* d_moments_out,
                              mb3dgs_stream_t stream) {
    Ctx c;
    int rc = setup(cfg, cams, n_views, P, pair_capacity, ws_bytes, ws, c);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char* w = static_cast<char*>(ws);
    launch_moments(c.p, c.vt, c.L, w, st);
    if (d_moments_out) launch_moments_to_power(c.p, c.L, w, d_moments_out, st);
    return cuda_ok();
}

int mb3dgs_reconstruct_transmittance(const mb3dgs_config* cfg, const mb3dgs_camera* cams, int n_views, int64_t P,
                                     int64_t pair_capacity, void* ws, size_t ws_bytes, const float* d_eta, int Q,
                                     float* d_T_out, mb3dgs_stream_t stream) {
    if (Q < 0 || (Q > 0 && (!d_eta || !d_T_out))) return MB3DGS_ERR_INVALID_ARG;
    Ctx c;
    int rc = setup(cfg, cams, n_views, P, pair_capacity, ws_bytes, ws, c);
    if (rc) return rc;
    launch_reconstruct(c.p, c.L, static_cast<char*>(ws), d_eta, Q, d_T_out, reinterpret_cast<cudaStream_t>(stream));
    return cuda_ok();
}

int mb3dgs_shade(const mb3dgs_config* cfg, const mb3dgs_camera* cams, int n_views, int64_t P, int64_t pair_capacity,
                 void* ws, size_t ws_bytes, float* d_rgb, float* d_T_final, float* d_penalty, mb3dgs_stream_t stream) {
    if (!d_rgb || !d_T_final) return MB3DGS_ERR_INVALID_ARG;
    Ctx c;
    int rc = setup(cfg, cams, n_views, P, pair_capacity, ws_bytes, ws, c);
    if (rc) return rc;
    rc = launch_shade(c.p, c.vt, c.L, static_cast<char*>(ws), d_rgb, d_T_final, d_penalty,
                      reinterpret_cast<cudaStream_t>(stream));
    if (rc) return rc;
    return cuda_ok();
}

int mb3dgs_render(const mb3dgs_config* cfg, const mb3dgs_gaussians* g, const mb3dgs_camera* cams, int n_views,
                  void* ws, size_t ws_bytes, int64_t pair_capacity, float* d_rgb, float* d_T_final, float* d_penalty,
                  mb3dgs_stream_t stream) {
    if (!d_rgb || !d_T_final) return MB3DGS_ERR_INVALID_ARG;
    int rc = mb3dgs_preprocess(cfg, g, cams, n_views, ws, ws_bytes, pair_capacity, stream);
    if (rc) return rc;
    Ctx c;
    rc = setup(cfg, cams, n_views, g->P, pair_capacity, ws_bytes, ws, c);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char* w = static_cast<char*>(ws);
    launch_binning(c.vt, c.L, w, st);
    if (c.p.schedule == MB3DGS_SCHEDULE_QUEUE) launch_tile_order(c.L, w, st);
    launch_moments(c.p, c.vt, c.L, w, st);
    launch_reconstruct(c.p, c.L, w, nullptr, 0, nullptr, st);
    if ((rc = launch_shade(c.p, c.vt, c.L, w, d_rgb, d_T_final, d_penalty, st))) return rc;
    return cuda_ok();
}

static int check_grads(const mb3dgs_gaussians* g, const mb3dgs_gaussian_grads* gr) {
    if (!g || !gr || g->P < 0) return MB3DGS_ERR_INVALID_ARG;
    if (g->P > 0 && (!g->means || !g->scales || !g->quats || !g->weights || !g->sh || !gr->means || !gr->scales ||
                     !gr->quats || !gr->weights || !gr->sh))
        return MB3DGS_ERR_INVALID_ARG;
    return MB3DGS_OK;
}

int mb3dgs_backward_quadrature(const mb3dgs_config* cfg, const mb3dgs_camera* cams, int n_views, int64_t P,
                               int64_t pair_capacity, void* ws, size_t ws_bytes, const float* d_dL_drgb,
                               const float* d_dL_dpenalty, const float* d_dL_dT, mb3dgs_stream_t stream) {
    if (!d_dL_drgb) return MB3DGS_ERR_INVALID_ARG;
    Ctx c;
    int rc = setup(cfg, cams, n_views, P, pair_capacity, ws_bytes, ws, c);
    if (rc) return rc;
    rc = launch_backward_quadrature(c.p, c.vt, c.L, static_cast<char*>(ws), d_dL_drgb, d_dL_dpenalty, d_dL_dT,
                                    reinterpret_cast<cudaStream_t>(stream));
    return rc ? rc : cuda_ok();
}

int mb3dgs_backward_moments(const mb3dgs_config* cfg, const mb3dgs_camera* cams, int n_views, int64_t P,
                            int64_t pair_capacity, void* ws, size_t ws_bytes, mb3dgs_stream_t stream) {
    Ctx c;
    int rc = setup(cfg, cams, n_views, P, pair_capacity, ws_bytes, ws, c);
    if (rc) return rc;
    rc = launch_backward_moments(c.p, c.vt, c.L, static_cast<char*>(ws), reinterpret_cast<cudaStream_t>(stream));
    return rc ? rc : cuda_ok();
}

int mb3dgs_backward_preprocess(const mb3dgs_config* cfg, const mb3dgs_gaussians* g, const mb3dgs_camera* cams,
                               int n_views, void* ws, size_t ws_bytes, int64_t pair_capacity,
                               const mb3dgs_gaussian_grads* grads, mb3dgs_stream_t stream) {
    int rc = check_grads(g, grads);
    if (rc) return rc;
    Ctx c;
    rc = setup(cfg, cams, n_views, g->P, pair_capacity, ws_bytes, ws, c);
    if (rc) return rc;
    rc = launch_backward_preprocess(c.p, c.vt, c.L, static_cast<char*>(ws), *g, *grads,
                                    reinterpret_cast<cudaStream_t>(stream));
    return rc ? rc : cuda_ok();
}

int mb3dgs_backward(const mb3dgs_config* cfg, const mb3dgs_gaussians* g, const mb3dgs_camera* cams, int n_views,
                    void* ws, size_t ws_bytes, int64_t pair_capacity, const float* d_dL_drgb,
                    const float* d_dL_dpenalty, const float* d_dL_dT, const mb3dgs_gaussian_grads* grads,
                    mb3dgs_stream_t stream) {
    int rc = check_grads(g, grads);
    if (rc) return rc;
    if (!d_dL_drgb) return MB3DGS_ERR_INVALID_ARG;
    Ctx c;
    rc = setup(cfg, cams, n_views, g->P, pair_capacity, ws_bytes, ws, c);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char* w = static_cast<char*>(ws);
    if ((rc = launch_backward_quadrature(c.p, c.vt, c.L, w, d_dL_drgb, d_dL_dpenalty, d_dL_dT, st))) return rc;
    if ((rc = launch_backward_moments(c.p, c.vt, c.L, w, st))) return rc;
    if ((rc = launch_backward_preprocess(c.p, c.vt, c.L, w, *g, *grads, st))) return rc;
    return cuda_ok();
}

int mb3dgs_get_status(const void* ws, size_t ws_bytes, int* status, int64_t* n_pairs, mb3dgs_stream_t stream) {
    if (!ws || ws_bytes < 64) return MB3DGS_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    StatusWords h;
    if (cudaMemcpyAsync(&h, ws, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess) return MB3DGS_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return MB3DGS_ERR_CUDA;
    if (status) *status = h.status;
    if (n_pairs) *n_pairs = h.n_total;
    return MB3DGS_OK;
}

int mb3dgs_get_pair_counts(const void* ws, size_t ws_bytes, int64_t* tile_pairs, int64_t* pixel_pairs,
                           mb3dgs_stream_t stream) {
    if (!ws || ws_bytes < 64) return MB3DGS_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    StatusWords h;
    if (cudaMemcpyAsync(&h, ws, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess) return MB3DGS_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return MB3DGS_ERR_CUDA;
    if (tile_pairs) *tile_pairs = h.n_total;
    if (pixel_pairs) *pixel_pairs = (int64_t)h.n_pixpairs;
    return MB3DGS_OK;
}

int mb3dgs_autotune(mb3dgs_config* cfg, const mb3dgs_gaussians* g, const mb3dgs_camera* cams, int n_views,
                    void* ws, size_t ws_bytes, float* d_rgb, float* d_T_final, const float* d_dL_drgb,
                    const mb3dgs_gaussian_grads* grads, float* best_ms, mb3dgs_stream_t stream) {
    if (!cfg || !g || !d_rgb || !d_T_final || (d_dL_drgb && !grads)) return MB3DGS_ERR_INVALID_ARG;
    int rc = check_cfg(cfg);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    static const int shapes[3][2] = {{16, 16}, {32, 8}, {8, 32}};
    static const int schedules[2] = {MB3DGS_SCHEDULE_QUEUE, MB3DGS_SCHEDULE_GRID};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return MB3DGS_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return MB3DGS_ERR_CUDA;
    }
    mb3dgs_config best = *cfg;
    float best_t = -1.0f;
    rc = MB3DGS_OK;
    for (int si = 0; si < 3 && rc == MB3DGS_OK; ++si) {
        mb3dgs_config c = *cfg;
        c.tile_w = shapes[si][0];
        c.tile_h = shapes[si][1];
        c.batch = 0;
        c.schedule = MB3DGS_SCHEDULE_GRID;
        // this tile shape's pair count (counting pass at zero capacity)
        mb3dgs_config cc = c;
        cc.query_capacity = 0;
        size_t need = 0;
        if (mb3dgs_workspace_size(&cc, cams, n_views, g->P, 0, &need) != MB3DGS_OK || need > ws_bytes) continue;
        if ((rc = mb3dgs_preprocess(&cc, g, cams, n_views, ws, ws_bytes, 0, stream)) != MB3DGS_OK) break;
        if ((rc = mb3dgs_bin_tiles(&cc, cams, n_views, g->P, 0, ws, ws_bytes, stream)) != MB3DGS_OK) break;
        int64_t cap = 0;
        if ((rc = mb3dgs_get_pair_counts(ws, ws_bytes, &cap, nullptr, stream)) != MB3DGS_OK) break;
        if (mb3dgs_workspace_size(&c, cams, n_views, g->P, cap, &need) != MB3DGS_OK || need > ws_bytes) continue;
        for (int ki = 0; ki < 2 && rc == MB3DGS_OK; ++ki) {
                c.schedule = schedules[ki];
                float t_min = -1.0f;
                for (int it = 0; it < 3 && rc == MB3DGS_OK; ++it) {
                    if (it > 0 && cudaEventRecord(e0, st) != cudaSuccess) rc = MB3DGS_ERR_CUDA;
                    if (rc == MB3DGS_OK)
                        rc = mb3dgs_render(&c, g, cams, n_views, ws, ws_bytes, cap, d_rgb, d_T_final, nullptr, stream);
                    if (rc == MB3DGS_OK && d_dL_drgb)
                        rc = mb3dgs_backward(&c, g, cams, n_views, ws, ws_bytes, cap, d_dL_drgb, nullptr, nullptr, grads,
                                             stream);
                    if (rc == MB3DGS_OK && it > 0) {
                        float ms = 0.0f;
                        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                            rc = MB3DGS_ERR_CUDA;
                        else if (t_min < 0.0f || ms < t_min)
                            t_min = ms;
                    }
                }
                if (rc == MB3DGS_OK && t_min >= 0.0f && (best_t < 0.0f || t_min < best_t)) {
                    best_t = t_min;
                    best = c;
                }
            }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != MB3DGS_OK) return rc;
    if (best_t < 0.0f) return MB3DGS_ERR_WORKSPACE_TOO_SMALL;
    cfg->tile_w = best.tile_w;
    cfg->tile_h = best.tile_h;
    cfg->batch = best.batch;
    cfg->schedule = best.schedule;
    if (best_ms) *best_ms = best_t;
    return cuda_ok();
}

int mb3dgs_debug_tile_lists(const mb3dgs_config* cfg, const mb3dgs_camera* cams, int n_views, int64_t P,
                            int64_t pair_capacity, const void* ws, size_t ws_bytes, int32_t* d_ids, int32_t* d_ranges,
                            int32_t* d_rects, mb3dgs_stream_t stream) {
    Ctx c;
    int rc = setup(cfg, cams, n_views, P, pair_capacity, ws_bytes, ws, c);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int64_t cap = pair_capacity;
    const char* w = static_cast<const char*>(ws);
    if (d_ids && cap > 0)
        if (cudaMemcpyAsync(d_ids, w + c.L.vals[c.L.final_buf], sizeof(int32_t) * cap, cudaMemcpyDeviceToDevice, st))
            return MB3DGS_ERR_CUDA;
    if (d_ranges && c.L.n_tiles > 0)
        if (cudaMemcpyAsync(d_ranges, w + c.L.ranges, sizeof(int32_t) * 2 * c.L.n_tiles, cudaMemcpyDeviceToDevice, st))
            return MB3DGS_ERR_CUDA;
    if (d_rects && c.L.VP > 0)
        if (cudaMemcpy2DAsync(d_rects, 4 * sizeof(int32_t), w + c.L.rec + sizeof(float) * R_RECT, sizeof(float) * REC,
                              4 * sizeof(int32_t), (size_t)c.L.VP, cudaMemcpyDeviceToDevice, st))
            return MB3DGS_ERR_CUDA;
    return cuda_ok();
}

}  // extern "C"

// ----------------------------------------------------------------------------
// Render without any device allocation by the caller or the library.
//
// Some callers cannot call cudaMalloc (or cannot hand the library a workspace
// from an allocator): code running where allocation is forbidden or unsafe,
// such as plug-ins inside a host that owns all device memory, real-time loops
// that must not allocate, or code paths that run while another component holds
// the allocator.  For them mb3dgs_render_noalloc uses a workspace that is a
// file-scope static device array of fixed size, reserved on every GPU that
// loads this library until the process exits.
// ----------------------------------------------------------------------------
namespace mb {
static __device__ __align__(256) unsigned char g_noalloc_ws[MB3DGS_NOALLOC_WORKSPACE_BYTES];

// The device address of the array belongs to the CUDA context that loaded the
// module: a cudaDeviceReset (or a primary context torn down and created again)
// gives the array a new address.  So the address is cached per device together
// with the unique id of the context it was looked up in (cuCtxGetId, reached
// through the runtime's driver entry points, no link against libcuda), and
// looked up again when the current context's id differs.  Without those entry
// points it is looked up on every call.
typedef int (*ctx_get_current_fn)(void**);
typedef int (*ctx_get_id_fn)(void*, unsigned long long*);

static std::mutex g_noalloc_mutex;
static void* g_noalloc_ptr[256] = {};
static unsigned long long g_noalloc_ctx[256] = {};

static bool current_context_id(unsigned long long* id) {
    static ctx_get_current_fn get_current = nullptr;
    static ctx_get_id_fn get_id = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* f0 = nullptr;
        void* f1 = nullptr;
        cudaDriverEntryPointQueryResult q0, q1;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            q0 == cudaDriverEntryPointSuccess && q1 == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<ctx_get_current_fn>(f0);
            get_id = reinterpret_cast<ctx_get_id_fn>(f1);
        }
        cudaGetLastError();
    }
    if (!get_current || !get_id) return false;
    void* ctx = nullptr;
    if (get_current(&ctx) != 0 || ctx == nullptr) return false;   // no context yet: the lookup creates it
    return get_id(ctx, id) == 0;
}

// Device address of the static workspace in the current device's context (the
// array's host-side name is only a stand-in, not a device address).  Called
// with the device current; the first call in a context looks the address up.
static int noalloc_workspace(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return MB3DGS_ERR_CUDA;
    unsigned long long ctx = 0;
    const bool have_id = current_context_id(&ctx);
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!have_id || !g_noalloc_ptr[dev] || g_noalloc_ctx[dev] != ctx) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_ws);
        if (e != cudaSuccess || p == nullptr) {
            g_last_cuda_error = cudaGetErrorString(e);
            return MB3DGS_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = p;
        g_noalloc_ctx[dev] = have_id ? ctx : 0;
    }
    *out = g_noalloc_ptr[dev];
    return MB3DGS_OK;
}
}  // namespace mb

extern "C" int mb3dgs_render_noalloc(const mb3dgs_config* cfg, const mb3dgs_gaussians* g, const mb3dgs_camera* cams,
                                     int n_views, float* d_rgb, float* d_T_final, float* d_penalty, int32_t* d_status,
                                     mb3dgs_stream_t stream) {
    if (!g || !d_rgb || !d_T_final || !d_status) return MB3DGS_ERR_INVALID_ARG;
    int rc = check_cfg(cfg);
    if (rc) return rc;
    ViewTable vt;
    int64_t npix, nt;
    rc = make_views(cfg, cams, n_views, vt, npix, nt);
    if (rc) return rc;
    const size_t cap_bytes = (size_t)MB3DGS_NOALLOC_WORKSPACE_BYTES;
    Layout L;
    rc = make_layout(cfg, vt, npix, nt, g->P, 0, L);
    if (rc) return rc;
    if (L.total > cap_bytes) return MB3DGS_ERR_WORKSPACE_TOO_SMALL;   // P / pixels beyond the fixed maximum
    // Largest pair capacity whose layout still fits the static array.  Every
    // region of the layout grows with the capacity or does not depend on it
    // (pair keys and values, radix histograms), so the total is non-decreasing
    // in the capacity and the fitting capacities form a prefix [0, lo]: a
    // bisection over 31 bits finds its end (host arithmetic only).
    int64_t lo = 0, hi = (int64_t(1) << 31) - 1;
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo + 1) / 2;
        Layout t;
        if (make_layout(cfg, vt, npix, nt, g->P, mid, t) == MB3DGS_OK && t.total <= cap_bytes) lo = mid;
        else hi = mid - 1;
    }
    void* ws = nullptr;
    rc = noalloc_workspace(&ws);
    if (rc) return rc;
    rc = mb3dgs_render(cfg, g, cams, n_views, ws, cap_bytes, lo, d_rgb, d_T_final, d_penalty, stream);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // the status word (first int of the workspace header) goes to the caller's output
    if (cudaMemcpyAsync(d_status, ws, sizeof(int32_t), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return MB3DGS_ERR_CUDA;
    return cuda_ok();
}
