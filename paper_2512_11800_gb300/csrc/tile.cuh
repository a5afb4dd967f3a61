// Per-tile pass machinery shared by the moment, shading and adjoint passes:
// the work schedule (persistent CTAs over a work-ordered queue, or one CTA
// per tile), the pixel of each thread, and cp.async staging of records --
// per warp for the passes whose warps work on their own 8x4-pixel
// footprints, per CTA (batches of a tile's list) for the moment-adjoint pass,
// whose per-record sums are combined over the whole tile in shared memory.
#pragma once
#include "common.cuh"

namespace mb {

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}

// Stage the records of list[start + b * batch ..) (at most batch <= TPB of
// them) into shared memory: each thread copies up to 8 x 16 B; no multicast.
__device__ __forceinline__ int stage_batch(float* s_rec, const float* __restrict__ rec, const int32_t* __restrict__ ids,
                                           int64_t rec_base, int start, int end, int b, int batch) {
    const int first = start + b * batch;
    const int nb = min(batch, end - first);
#pragma unroll
    for (int j = 0; j < REC / 4; ++j) {
        const int lin = j * TPB + threadIdx.x;
        const int rr = lin >> 3, cc = lin & 7;
        if (rr < nb) cp_async16(s_rec + rr * REC + cc * 4, rec + (rec_base + ids[first + rr]) * REC + cc * 4);
    }
    asm volatile("cp.async.wait_all;\n" ::);
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
    tile_pixel(V, tx, ty, threadIdx.x & 31, threadIdx.x >> 5, c.px, c.py);
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

// Tile schedule of one per-tile launch.
struct TileSched {
    const int* order;   // QUEUE: tiles by decreasing list length; GRID: nullptr
    int* queue;         // QUEUE: this launch's tile counter (zeroed before the launch)
    int64_t n_tiles;
};

// The CTA's next tile, -1 when none is left (block-uniform; barriers inside,
// which also separate one tile's shared-memory use from the next).  GRID:
// tile blockIdx.x once.  QUEUE: the next slot of the ordered queue.
__device__ __forceinline__ int64_t next_tile(const TileSched& ts, int* s_slot, bool first) {
    if (ts.order == nullptr) return first ? (int64_t)blockIdx.x : -1;
    __syncthreads();
    if (threadIdx.x == 0) *s_slot = atomicAdd(ts.queue, 1);
    __syncthreads();
    const int t = *s_slot;
    return t < ts.n_tiles ? (int64_t)ts.order[t] : -1;
}

// Host: grid size and schedule of a per-tile launch of `func` (queue counter
// `q` zeroed on the stream for QUEUE).
struct TileLaunch {
    unsigned grid;
    TileSched ts;
};
TileLaunch tile_launch(const Params& p, const Layout& L, char* ws, int q, const void* func, size_t smem,
                       cudaStream_t st);

// Host: raises a kernel's dynamic shared-memory limit to `smem` once per
// device (outside any later stream capture); false on failure.
bool allow_dynamic_smem(const void* func, size_t smem);

// ---------------------------------------------------------------------------
// Warp-level work of the forward passes.  A work unit is one warp footprint
// (8 x 4 pixels) of one tile; every warp takes units on its own (no barrier
// between the warps of a CTA), walks the tile's Gaussian list in chunks of 32,
// keeps the records whose rectangle overlaps its footprint (ballot, order
// kept) and stages only those into its own shared-memory buffer.  Every pixel
// still visits its Gaussians in ascending id order, so per-pixel sums are the
// same as with whole-tile batches.
// ---------------------------------------------------------------------------
constexpr int WARPS = TPB / 32;
constexpr int WARP_STAGE_FLOATS = 32 * REC + 32;   // 32 records + their ids

// Next unit of this warp: the tile (-1 when none is left) and the footprint
// index in *fp (warp-uniform).  GRID: CTA = tile, warp w = footprint w, once.
// QUEUE: unit u of the ordered queue is footprint u % 8 of tile order[u / 8].
__device__ __forceinline__ int64_t next_unit(const TileSched& ts, bool first, int* fp) {
    if (ts.order == nullptr) {
        *fp = threadIdx.x >> 5;
        return first ? (int64_t)blockIdx.x : -1;
    }
    int u = 0;
    if ((threadIdx.x & 31) == 0) u = atomicAdd(ts.queue, 1);
    u = __shfl_sync(0xffffffffu, u, 0);
    if ((int64_t)u >= ts.n_tiles * WARPS) return -1;
    *fp = u & (WARPS - 1);
    return (int64_t)ts.order[u / WARPS];
}

// Pixel of this lane for footprint fp of `tile`, plus the footprint's pixel
// box [fx0, fx0 + 7] x [fy0, fy0 + 3] (for the record filter).
__device__ __forceinline__ PixelCtx unit_ctx(const ViewTable& vt, const int2* __restrict__ ranges, int64_t P,
                                             int64_t tile, int fp, int* fx0, int* fy0) {
    PixelCtx c;
    c.v = find_view(vt, tile);
    const ViewDesc& V = vt.v[c.v];
    const int lt = (int)(tile - V.tile_base);
    const int tx = lt % V.tiles_x, ty = lt / V.tiles_x;
    const int lane = threadIdx.x & 31;
    tile_pixel(V, tx, ty, lane, fp, c.px, c.py);
    *fx0 = c.px - (lane & 7);
    *fy0 = c.py - (lane >> 3);
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

// Stage the records of list[pos, pos + 32) whose rectangle overlaps the
// footprint box into the warp's buffer (ascending list order); returns how
// many.  All 32 lanes call it; the buffer is ready when it returns.
__device__ __forceinline__ int stage_warp_chunk(float* __restrict__ s_buf, const float* __restrict__ rec,
                                                const int32_t* __restrict__ ids, int64_t rec_base, int pos, int end,
                                                int fx0, int fy0) {
    const int lane = threadIdx.x & 31;
    int* s_ids = reinterpret_cast<int*>(s_buf + 32 * REC);
    bool keep = false;
    int id = 0;
    if (pos + lane < end) {
        id = ids[pos + lane];
        const int* ri = reinterpret_cast<const int*>(rec + (rec_base + id) * REC + R_RECT);
        const int x0 = __ldg(ri + 0), y0 = __ldg(ri + 1), x1 = __ldg(ri + 2), y1 = __ldg(ri + 3);
        keep = x0 <= fx0 + 7 && x1 >= fx0 && y0 <= fy0 + 3 && y1 >= fy0;
    }
    const unsigned mask = __ballot_sync(0xffffffffu, keep);
    const int m = __popc(mask);
    __syncwarp();                 // the previous chunk's records are no longer read
    if (keep) s_ids[__popc(mask & ((1u << lane) - 1u))] = id;
    __syncwarp();
    for (int t = lane; t < m * (REC / 4); t += 32) {
        const int k = t / (REC / 4), part = t % (REC / 4);
        cp_async16(s_buf + k * REC + part * 4, rec + (rec_base + s_ids[k]) * REC + part * 4);
    }
    asm volatile("cp.async.wait_all;\n" ::);
    __syncwarp();
    return m;
}

enum TileQueue { Q_MOMENTS = 0, Q_SHADE = 1, Q_BWD_QUAD = 2, Q_BWD_MOM = 3, N_QUEUES = 4 };

}  // namespace mb
