// Per-tile pass machinery shared by the moment, shading and adjoint passes:
// the tile schedule (persistent CTAs over a work-ordered queue, or one CTA per
// tile), the pixel of each thread, and cp.async staging of record batches.
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

enum TileQueue { Q_MOMENTS = 0, Q_SHADE = 1, Q_BWD_QUAD = 2, Q_BWD_MOM = 3, N_QUEUES = 4 };

}  // namespace mb
