/*
 * mb3dgs.h -- C ABI of the GB300 moment-based Gaussian rasterizer.
 *
 * Implements the rendering hot path of "Moment-Based 3D Gaussian Splatting"
 * (MB3DGS, arXiv 2512.11800): a two-pass, sort-free tile rasterizer in which
 *   (a) every pixel accumulates the analytic density moments of all Gaussians
 *       covering it (Sec. 3.2, Eq. 10-12, App. C),
 *   (b) every pixel reconstructs a transmittance function from its moments
 *       via moment bounds (Sec. 3.2, Eq. 8), and
 *   (c) a second pass evaluates the per-Gaussian quadrature of the volume
 *       rendering integral (Eq. 7, App. B) and rescales the opacity (Eq. 15),
 * plus the adjoint of both passes (Sec. 3.3 "Adjoint Rendering", Eq. 22).
 *
 * Conventions (all calls):
 *  - Every pointer named d_* or documented "device" is CUDA device memory owned
 *    by the caller; the library never allocates or frees device memory.
 *  - Calls are asynchronous on the given stream unless documented otherwise.
 *  - Cameras are OpenCV pinholes (x right, y down, z forward); viewmat is the
 *    4x4 row-major world->camera transform; pixel (x, y) has its centre at
 *    (x + 0.5, y + 0.5); ray directions are unit vectors, so ray distances t
 *    are metric.
 *  - Gaussians are float32 structure-of-arrays: means[P][3], scales[P][3]
 *    (positive), quats[P][4] (w,x,y,z, normalised inside), weights[P] (peak
 *    density w >= 0), sh[P][K][3] with K = (sh_degree+1)^2, sh_degree <= 3.
 *  - Images are row-major; rgb is [H][W][3], transmittance/penalty [H][W];
 *    with several views the per-view images are concatenated in view order.
 *  - The staged calls (bin_tiles .. shade, backward, debug) must be given the
 *    same cfg, cameras, P and pair_capacity as the mb3dgs_preprocess (or
 *    mb3dgs_render) call that filled the workspace; the workspace layout is a
 *    pure function of those values.
 *  - Return value: MB3DGS_OK (0) or a negative MB3DGS_ERR_* code; nothing
 *    aborts the process.  Errors detected on the device (pair-capacity
 *    overflow, non-finite inputs in strict mode) are recorded in a status word
 *    inside the workspace and read with mb3dgs_get_status().
 */
#ifndef MB3DGS_H
#define MB3DGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* mb3dgs_stream_t; /* == cudaStream_t; NULL = legacy default stream */

enum {
    MB3DGS_OK = 0,
    MB3DGS_ERR_INVALID_ARG = -1,       /* null pointer, bad size, bad config value */
    MB3DGS_ERR_CUDA = -2,              /* a CUDA launch or copy failed */
    MB3DGS_ERR_WORKSPACE_TOO_SMALL = -3,
    MB3DGS_ERR_TIMEOUT = -4,           /* a bounded device wait expired */
    MB3DGS_ERR_NUMERIC = -5,           /* non-finite Gaussian parameters seen with strict = 1 */
    MB3DGS_ERR_UNSUPPORTED = -6,       /* configuration outside what the kernels implement */
    MB3DGS_ERR_CAPACITY = -7           /* tile-pair count exceeded the workspace's pair capacity */
};

enum { MB3DGS_MOMENTS_F32 = 0, MB3DGS_MOMENTS_BF16 = 1, MB3DGS_MOMENTS_F16 = 2 };
/* Moment basis.  POWER: power moments of the warped depth (Sec. 3.2,
 * Eq. 10-12) with the bounds of Eq. 8.  TRIG: trigonometric moments (Sec. 3.2,
 * Eq. 13-14; App. C) of the angle (2 pi - theta) g-hat, with the bounds of the
 * Gauss-Szego rule on the unit circle cut in the middle of the wrapping zone.
 * Both bases have the adjoint calls and keep their bound queries as
 * query_capacity says. */
enum { MB3DGS_BASIS_POWER = 0, MB3DGS_BASIS_TRIG = 1 };
/* How the per-tile passes map tiles of all views to CTAs.  QUEUE: one wave of
 * persistent CTAs takes tiles from an atomic queue in decreasing order of
 * their Gaussian-list length; GRID: one CTA per tile in view/raster order. */
enum { MB3DGS_SCHEDULE_QUEUE = 0, MB3DGS_SCHEDULE_GRID = 1 };
enum { MB3DGS_MAX_VIEWS = 32 };

/* Method parameters.  Defaults (mb3dgs_config_default) are the paper's values
 * where it prints them and documented readings where it does not. */
typedef struct mb3dgs_config {
    int n;              /* 2n+1 power moments; n = 4 (Sec. 3.2).  Only 4 is implemented. */
    int n_intervals;    /* N quadrature intervals, N+1 sample points (Eq. 7); 1..8, default 3 */
    float kappa;        /* sample spacing t_j = mu + kappa Sigma x_j (App. B); 3 */
    float beta;         /* tau = m0 ((1-beta) L + beta U) (Sec. 3.2); 0.25 */
    float conf_c;       /* proxy confidence level c (App. C); 0.01 */
    float warp_lambda;  /* power-transform lambda of the depth warp (Sec. 3.2); -1.5 */
    float t_near;       /* t_n; 0.01 (reading) */
    float t_far;        /* t_f; 1e6 (App. C) */
    float eps;          /* rescaling clamp of Eq. 15; 1e-6 */
    float bias_alpha;   /* moment bias towards U[0,1] moments (reading); 1e-3 */
    float m_min;        /* pixels with m0 < m_min have tau == 0; 1e-7 */
    float r_mult;       /* culling sphere radius = r_mult * max(scale) (Sec. 3.3); 3 */
    float bg[3];        /* background radiance L_bg (Eq. 2); black */
    int moment_dtype;   /* storage of the per-pixel moment buffer: MB3DGS_MOMENTS_* */
    int strict;         /* 1: non-finite Gaussian parameters set MB3DGS_ERR_NUMERIC */
    /* Execution shape (no effect on the results: every pixel visits its
     * Gaussians in ascending id order whatever the tiling; mb3dgs_autotune
     * picks them).  tile_w x tile_h pixels per tile with tile_w * tile_h = 256,
     * tile_w in {8, 16, 32, 64} (0, 0: 16 x 16); in every pass but the
     * moment adjoint each warp of a tile works on an 8 x 4 footprint and
     * stages the records that overlap it in chunks of 32; batch: records
     * staged per CTA batch in the moment-adjoint pass, a multiple of 32 up to
     * 256 (0: 256); schedule: MB3DGS_SCHEDULE_*. */
    int tile_w, tile_h;
    int batch;
    int schedule;
    int64_t query_capacity; /* (pixel, Gaussian) pair slots in which mb3dgs_shade keeps
                           the N+1 bound queries of every pair (16 (N+1) bytes a
                           pair: 64 at N = 3; 8 (N+1) with compact_queries) for
                           mb3dgs_backward, which then
                           reads them instead of solving them again.  Pixels
                           are served in pixel order while all of a pixel's
                           pairs fit; the backward solves the queries of the
                           remaining pixels again (a memory / time trade the
                           caller sets; the results are the same).  0 (default):
                           all are recomputed; the pixel-pair count of
                           mb3dgs_get_pair_counts keeps all.  Below 2^40.
                           TRIG: {tau, node angles x_0, x_1, j | ns} in 16 bytes.
                           Ignored with a table (tau_table). */
    int basis;          /* MB3DGS_BASIS_*; default POWER */
    float trig_theta;   /* TRIG: wrapping angle theta in (0, 2 pi) (reading); pi/2 */
    int tau_table;      /* POWER: 0 (default) solves every bound query of the quadrature
                           pass; M in [8, 128] has mb3dgs_reconstruct_transmittance
                           tabulate tau(eta) and dtau/deta per pixel at M + 1 knots on each of
                           the (at most five) segments between the Gauss nodes in [0, 1],
                           and the quadrature pass interpolates them (cubic Hermite) instead
                           (40 (M + 1) bytes a pixel).  An approximation of Eq. 8: its error
                           against the solved bounds falls like M^-4.  The adjoint calls
                           differentiate the solved bounds that the table approximates
                           (pass 1 solves its queries again; query_capacity is ignored). */
    int compact_queries; /* 0 (default): a kept bound query takes 16 bytes {tau, x_0, x_1,
                           j | nroot}.  1: 8 bytes {tau, the roots as 16-bit positions in
                           their brackets}; the backward recomputes j from the query
                           (the same operations give the same value) and restores each
                           root by one Laguerre step from its position (the gradients
                           agree with the 16-byte form to rounding), so twice as many
                           pairs keep their queries in the same memory, at some cost in
                           the backward.  POWER only (MB3DGS_ERR_UNSUPPORTED otherwise). */
} mb3dgs_config;

/* Device pointers, caller-owned, layout as in the file comment. */
typedef struct mb3dgs_gaussians {
    const float* means;
    const float* scales;
    const float* quats;
    const float* weights;
    const float* sh;
    int64_t P;
    int sh_degree;
} mb3dgs_gaussians;

/* Host struct (passed by value into kernels). */
typedef struct mb3dgs_camera {
    float viewmat[16];   /* world -> camera, row-major 4x4 */
    float fx, fy, cx, cy;
    int width, height;
} mb3dgs_camera;

/* Parameter gradients, device, same shapes as mb3dgs_gaussians; written (not
 * accumulated) by mb3dgs_backward. */
typedef struct mb3dgs_gaussian_grads {
    float* means;
    float* scales;
    float* quats;
    float* weights;
    float* sh;
} mb3dgs_gaussian_grads;

const char* mb3dgs_status_string(int code);

/* Text of the CUDA error behind the calling thread's last MB3DGS_ERR_CUDA. */
const char* mb3dgs_last_cuda_error(void);

/* Fills *cfg with the defaults listed above. */
int mb3dgs_config_default(mb3dgs_config* cfg);

/* Bytes of device workspace needed to render n_views cameras of P Gaussians
 * with room for pair_capacity (tile, Gaussian) pairs.  Host only. */
int mb3dgs_workspace_size(const mb3dgs_config* cfg, const mb3dgs_camera* cams, int n_views, int64_t P,
                          int64_t pair_capacity, size_t* bytes);

/* Stage 1 -- per (view, Gaussian): frustum culling with the bounding sphere
 * (Sec. 3.3), camera-space ray-parameterisation coefficients of Eq. 4-6
 * (App. A), SH emission (Sec. 3.1), the confidence-interval proxy ellipse and
 * its pixel rectangle (Eq. 17-21, App. C) and its tile count.  Computed in
 * FP64, stored FP32.  Resets the workspace status word. */
int mb3dgs_preprocess(const mb3dgs_config* cfg, const mb3dgs_gaussians* g, const mb3dgs_camera* cams,
                      int n_views, void* ws, size_t ws_bytes, int64_t pair_capacity, mb3dgs_stream_t stream);

/* Stage 2 -- tile binning by tile key only, no depth sort: exclusive scan of
 * the tile counts, emission of (tile, Gaussian) pairs and a stable LSD radix
 * sort by tile, so each tile's list holds ascending Gaussian ids.  Sets
 * MB3DGS_ERR_CAPACITY in the status word (and renders nothing) if the pair
 * count exceeds the capacity given to mb3dgs_preprocess. */
int mb3dgs_bin_tiles(const mb3dgs_config* cfg, const mb3dgs_camera* cams, int n_views, int64_t P,
                     int64_t pair_capacity, void* ws, size_t ws_bytes, mb3dgs_stream_t stream);

/* Stage 3 -- moment pass (Sec. 3.3, App. C): per pixel, sum over the Gaussians
 * whose rectangle contains the pixel centre of the analytic moments
 * (Eq. 10-12).  Accumulated in FP32 in an orthonormal Legendre basis of the
 * warped depth (same moment space as the paper's power moments) and stored
 * in the workspace with cfg->moment_dtype.  If d_moments_out != NULL it also
 * receives the paper's power moments m-hat_0..m-hat_2n, layout
 * [pixel][2n+1] over all views. */
int mb3dgs_accumulate_moments(const mb3dgs_config* cfg, const mb3dgs_camera* cams, int n_views, int64_t P,
                              int64_t pair_capacity, void* ws, size_t ws_bytes, float* d_moments_out,
                              mb3dgs_stream_t stream);

/* Stage 4 -- per-pixel reconstruction (Sec. 3.2, Eq. 8): normalise and bias
 * the moments, compute the recurrence (Jacobi) coefficients of the moment
 * measure's orthogonal polynomials and its Gauss nodes, stored in the
 * workspace for the shading pass.  If Q > 0 it also evaluates the
 * transmittance T(eta) = exp(-tau(eta)), tau = m0 ((1-beta) L + beta U), at
 * the warped depths d_eta[pixel][Q] into d_T_out[pixel][Q]. */
int mb3dgs_reconstruct_transmittance(const mb3dgs_config* cfg, const mb3dgs_camera* cams, int n_views,
                                     int64_t P, int64_t pair_capacity, void* ws, size_t ws_bytes,
                                     const float* d_eta, int Q, float* d_T_out, mb3dgs_stream_t stream);

/* Stage 5 -- quadrature pass (Eq. 7, App. B) with the consistency penalty
 * (App. D) and the opacity rescaling epilogue (Eq. 15).  Writes d_rgb
 * [pixel][3], d_T_final [pixel] = exp(-m0) and, if non-NULL, d_penalty
 * [pixel] = sum_i P_i.  Keeps sum_i L_i and O in the workspace for backward,
 * and, when cfg->query_capacity > 0, each pair's bound queries (optical
 * depths and kernel-polynomial roots). */
int mb3dgs_shade(const mb3dgs_config* cfg, const mb3dgs_camera* cams, int n_views, int64_t P,
                 int64_t pair_capacity, void* ws, size_t ws_bytes, float* d_rgb, float* d_T_final,
                 float* d_penalty, mb3dgs_stream_t stream);

/* Stages 1-5 in order on one stream; no host synchronisation. */
int mb3dgs_render(const mb3dgs_config* cfg, const mb3dgs_gaussians* g, const mb3dgs_camera* cams, int n_views,
                  void* ws, size_t ws_bytes, int64_t pair_capacity, float* d_rgb, float* d_T_final,
                  float* d_penalty, mb3dgs_stream_t stream);

/* Adjoint of mb3dgs_render (Sec. 3.3 "Adjoint Rendering", Eq. 22, App. C):
 * an adjoint-moment pass producing per-pixel dL/dm, then a gradient pass
 * reducing per-Gaussian gradients over covered pixels, then the chain rule
 * through the preprocessing to the Gaussian parameters.  Requires the
 * workspace of the matching mb3dgs_render call (same cfg, g, cams).
 * d_dL_drgb [pixel][3]; d_dL_dpenalty [pixel] or NULL; d_dL_dT [pixel] or NULL:
 * the gradient with respect to the final transmittance T_final = e^{-m0}
 * (it reaches the Gaussians through m0, dT_final/dm0 = -T_final).  The proxy rectangles
 * and culling are treated as constants. */
int mb3dgs_backward(const mb3dgs_config* cfg, const mb3dgs_gaussians* g, const mb3dgs_camera* cams,
                    int n_views, void* ws, size_t ws_bytes, int64_t pair_capacity, const float* d_dL_drgb,
                    const float* d_dL_dpenalty, const float* d_dL_dT, const mb3dgs_gaussian_grads* grads,
                    mb3dgs_stream_t stream);

/* The three stages of mb3dgs_backward, for callers that time or interleave
 * them (same requirements as mb3dgs_backward; call them in this order).
 * backward_quadrature (pass 1): per (pixel, Gaussian) pair the adjoint of the
 *   quadrature, penalty and bound queries (saved by mb3dgs_shade when
 *   cfg->query_capacity > 0, else solved again); direct derivatives go to
 *   per-record gradients in the workspace (zeroed first), the bound
 *   derivatives to the per-pixel moment adjoint (TRIG: through the
 *   Verblunsky coefficients and reverse-mode Levinson-Durbin to the raw
 *   trigonometric moments).
 * backward_moments (pass 2): per pair the moment adjoint through the reverse
 *   sweep of the moment recurrence (Eq. 10-12; TRIG: of Eq. 14) into the
 *   record gradients.
 * backward_preprocess: chain rule through stage 1 to the Gaussian parameters
 *   (every entry of *grads is written). */
int mb3dgs_backward_quadrature(const mb3dgs_config* cfg, const mb3dgs_camera* cams, int n_views, int64_t P,
                               int64_t pair_capacity, void* ws, size_t ws_bytes, const float* d_dL_drgb,
                               const float* d_dL_dpenalty, const float* d_dL_dT, mb3dgs_stream_t stream);
int mb3dgs_backward_moments(const mb3dgs_config* cfg, const mb3dgs_camera* cams, int n_views, int64_t P,
                            int64_t pair_capacity, void* ws, size_t ws_bytes, mb3dgs_stream_t stream);
int mb3dgs_backward_preprocess(const mb3dgs_config* cfg, const mb3dgs_gaussians* g, const mb3dgs_camera* cams,
                               int n_views, void* ws, size_t ws_bytes, int64_t pair_capacity,
                               const mb3dgs_gaussian_grads* grads, mb3dgs_stream_t stream);

/* Size of the fixed device workspace used by mb3dgs_render_noalloc. */
#define MB3DGS_NOALLOC_WORKSPACE_BYTES (64u << 20)

/* mb3dgs_render without any device allocation, for callers that cannot call
 * cudaMalloc or hand the library memory from an allocator (plug-ins in a host
 * that owns all device memory, loops that must not allocate).  The paper has
 * no counterpart; this is a deployment convenience.
 * The workspace is a static device array of MB3DGS_NOALLOC_WORKSPACE_BYTES
 * (64 MiB) that every GPU loading the library reserves until process exit.
 * Inputs and outputs are the caller's, as in mb3dgs_render; d_status (one
 * int32, device) receives the call's status word (MB3DGS_OK or e.g.
 * MB3DGS_ERR_CAPACITY when the frame has more (tile, Gaussian) pairs than fit
 * in the space left after the per-Gaussian and per-pixel buffers).
 * Returns MB3DGS_ERR_WORKSPACE_TOO_SMALL, before launching anything, when the
 * Gaussians, views and pixels alone need more than the fixed size.
 * The first call on a device looks up the array's device address (with that
 * device current) and keeps it for the device's CUDA context; after a
 * cudaDeviceReset the next call looks it up again.  Make the first call on a
 * device (and the first after a reset) before any stream capture.  Every call uses the same array: calls that overlap on the GPU
 * (other streams, other host threads) race and must be serialised by the caller.
 * Allocates nothing (no cudaMalloc / cudaFree). */
int mb3dgs_render_noalloc(const mb3dgs_config* cfg, const mb3dgs_gaussians* g, const mb3dgs_camera* cams,
                          int n_views, float* d_rgb, float* d_T_final, float* d_penalty, int32_t* d_status,
                          mb3dgs_stream_t stream);

/* Synchronises the stream and reads the workspace status word (an MB3DGS_*
 * code) and the number of (tile, Gaussian) pairs of the last binning. */
int mb3dgs_get_status(const void* ws, size_t ws_bytes, int* status, int64_t* n_pairs, mb3dgs_stream_t stream);

/* Synchronises the stream and reads, after mb3dgs_preprocess, the number of
 * (tile, Gaussian) pairs (the pair_capacity the frame needs; valid after
 * mb3dgs_bin_tiles) and of (pixel, Gaussian) pairs, i.e. pixel centres inside
 * a Gaussian's proxy rectangle (the query_capacity the frame needs).
 * Either output may be NULL. */
int mb3dgs_get_pair_counts(const void* ws, size_t ws_bytes, int64_t* tile_pairs, int64_t* pixel_pairs,
                           mb3dgs_stream_t stream);

/* Autotuner of the execution shape (the paper has none; its tiling is its
 * own hardware's).  For each candidate tile shape (16x16, 32x8, 8x32) and
 * schedule (QUEUE, GRID) whose workspace fits ws_bytes it
 * counts the frame's pairs, renders once untimed and times mb3dgs_render --
 * and mb3dgs_backward when d_dL_drgb and grads are given -- with CUDA events
 * on the stream (best of two), then writes the fastest shape into
 * cfg->tile_w, tile_h and schedule (batch 0) and its time in ms into *best_ms
 * (may be NULL).  cfg->query_capacity is kept.  Outputs go to the caller's
 * d_rgb [pixel][3] and d_T_final [pixel]; the other fields of cfg and the
 * scene are those of the frames to be rendered.  The forward results of
 * every candidate are identical.  Synchronises the stream; allocates nothing;
 * returns MB3DGS_ERR_WORKSPACE_TOO_SMALL if no candidate fits. */
int mb3dgs_autotune(mb3dgs_config* cfg, const mb3dgs_gaussians* g, const mb3dgs_camera* cams, int n_views,
                    void* ws, size_t ws_bytes, float* d_rgb, float* d_T_final, const float* d_dL_drgb,
                    const mb3dgs_gaussian_grads* grads, float* best_ms, mb3dgs_stream_t stream);

/* Debug/test access (device outputs, async): the sorted Gaussian ids of all
 * tile lists d_ids[capacity], per-tile [start, end) d_ranges[n_tiles][2]
 * (tiles of all views, row-major per view), and per (view, Gaussian)
 * integer pixel rectangles d_rects[n_views*P][4] = x0, y0, x1, y1 inclusive
 * (x0 > x1 when culled).  Any output pointer may be NULL. */
int mb3dgs_debug_tile_lists(const mb3dgs_config* cfg, const mb3dgs_camera* cams, int n_views, int64_t P,
                            int64_t pair_capacity, const void* ws, size_t ws_bytes, int32_t* d_ids,
                            int32_t* d_ranges, int32_t* d_rects, mb3dgs_stream_t stream);

/* Total number of CUDA kernels this library has launched in the process
 * (host counter; used to report launches per step). */
int64_t mb3dgs_launch_count(void);

/* Measured ALU throughput of the current device (the denominators of the
 * ALU roofline of the per-pair kernels; not part of the method).  fp32_tflops:
 * FP32 FMA pipe, 2 flop per FFMA; *_tops: MUFU (XU) pipe operations per
 * second, 1e12 units, per instruction kind. */
typedef struct mb3dgs_alu_peaks {
    double fp32_tflops;
    double ex2_tops, rsqrt_tops, rcp_tops, sin_tops;
    int sm_count;
} mb3dgs_alu_peaks;

/* Runs the throughput probes (independent FFMA / MUFU chains on every SM,
 * several waves of full CTAs, best of three CUDA-event-timed launches each)
 * on the stream and fills *out.  Synchronises the stream; takes ~50 ms;
 * allocates no device memory. */
int mb3dgs_probe_alu_peaks(mb3dgs_alu_peaks* out, mb3dgs_stream_t stream);

/* ---------------------------------------------------------------------------
 * Adaptive density control (Sec. 3.4 "Training and Densification"; App. D
 * "Adaptive Density Control"): the per-Gaussian rules a training loop runs
 * between optimiser steps.  All arrays are device, SoA as mb3dgs_gaussians
 * (scales after exp, weights after softplus); all calls are asynchronous on
 * the stream and allocate nothing.
 * ------------------------------------------------------------------------- */
typedef struct mb3dgs_adc_config {
    float grad_threshold;   /* densify when |sum_t |dL/dmean|| / n_visible >= this; 1e-4 (App. D) */
    float prune_opacity;    /* prune a resulting particle whose view-independent opacity is below
                               this; 0.005 (the 3DGS rule the paper keeps) */
    float percent_dense;    /* clone when max(s) <= percent_dense x scene_extent, else split; 0.01 */
    float scene_extent;     /* caller's scene scale (3DGS: camera extent); 1 */
    float big_world;        /* also prune when max(s) > big_world x scene_extent; 0.1; 0 = off */
    float split_gamma;      /* split: the largest scale times gamma; 0.6385502815 (App. D) */
    float split_delta;      /* split: children at mean -/+ delta s_max v; 0.6128153091 (App. D) */
} mb3dgs_adc_config;

/* Mutable Gaussian arrays (outputs of mb3dgs_densify), capacity entries each. */
typedef struct mb3dgs_gaussians_out {
    float* means;
    float* scales;
    float* quats;
    float* weights;
    float* sh;
    int64_t capacity;
} mb3dgs_gaussians_out;

int mb3dgs_adc_config_default(mb3dgs_adc_config* cfg);

/* View-independent opacity (App. D): the opacity of a particle seen along its
 * shortest axis through its centre, o = 1 - exp(-sqrt(2 pi) w min(s)).
 * weights [P], scales [P,3] in; opacity [P] out. */
int mb3dgs_view_independent_opacity(const float* d_weights, const float* d_scales, int64_t P, float* d_opacity,
                                    mb3dgs_stream_t stream);

/* Peak densities from opacities (App. D, with the average scale):
 * w = -log(1 - o) / (sqrt(2 pi) avg(s)).  opacity [P] in [0, 1), scales [P,3]
 * in; weights [P] out.  o >= 1 gives +inf. */
int mb3dgs_init_weights(const float* d_opacity, const float* d_scales, int64_t P, float* d_weights,
                        mb3dgs_stream_t stream);

/* One step of the densification statistics (App. D, after AbsGS): for every
 * visible particle abs_sum[i] += |dL/dmean_i| component-wise (float32) and
 * count[i] += 1.  d_visible [P] (0/1 bytes) may be NULL: a particle is then
 * visible when a component of its mean gradient is non-zero.  abs_sum [P,3]
 * and count [P] are the caller's running buffers (zero them at the start). */
int mb3dgs_accumulate_grad_stats(const float* d_dmeans, const uint8_t* d_visible, int64_t P, float* d_abs_sum,
                                 int32_t* d_count, mb3dgs_stream_t stream);

/* Device workspace bytes of mb3dgs_densify for P input particles. */
int mb3dgs_densify_workspace_size(int64_t P, size_t* bytes);

/* Clone / split / prune (App. D with the 3DGS rules):
 *   grad_i = |abs_sum_i| / count_i (0 when count_i = 0);
 *   grad_i >= grad_threshold and max(s_i) <= percent_dense x extent: clone,
 *     the particle and its copy each with w_i / 2;
 *   grad_i >= grad_threshold otherwise: split into two particles at
 *     mean -/+ split_delta s_max v (v the axis of the largest scale s_max,
 *     the first one on ties), that scale times split_gamma, the rest copied;
 *   every resulting particle is kept unless its view-independent opacity is
 *   below prune_opacity or max(s) > big_world x extent.
 * Threshold tests run in float32 in a fixed operation order (no fused
 * multiply-add), so that decisions are reproducible: the opacity test as
 * sqrt(2 pi) w min(s) >= -log(1 - prune_opacity).
 * Outputs keep the input order, each input's particles contiguous (clone:
 * original then copy; split: minus then plus offset).  out->capacity must be
 * at least 2 g->P; *d_P_out (device int64) receives the new count.
 * d_action [P] (int8, may be NULL) receives 0 kept as is, 1 cloned, 2 split
 * (before pruning); d_first [P] (int32, may be NULL) the index of input i's
 * first output particle (its outputs are d_first[i] .. d_first[i+1] - 1, the
 * last input's end being *d_P_out): the map for carrying per-particle
 * optimiser state over.  P is limited to 2^30.  Errors:
 * MB3DGS_ERR_INVALID_ARG for null arrays, capacity below 2P or a bad config;
 * MB3DGS_ERR_WORKSPACE_TOO_SMALL. */
int mb3dgs_densify(const mb3dgs_adc_config* cfg, const mb3dgs_gaussians* g, const float* d_abs_sum,
                   const int32_t* d_count, void* ws, size_t ws_bytes, const mb3dgs_gaussians_out* out,
                   int64_t* d_P_out, int8_t* d_action, int32_t* d_first, mb3dgs_stream_t stream);

/* Number of tiles (cfg->tile_w x cfg->tile_h pixels) over all views (host only). */
int64_t mb3dgs_num_tiles(const mb3dgs_config* cfg, const mb3dgs_camera* cams, int n_views);

#ifdef __cplusplus
}
#endif
#endif /* MB3DGS_H */
