// Tile work order for the persistent per-tile passes: all tiles of all views
// sorted by decreasing Gaussian-list length (32 power-of-two buckets, longest
// first), so that the long tiles start in the first wave and the tail of each
// pass is made of short ones.  Each per-tile launch then takes tiles from
// this order through its own atomic counter (TileSched).
#include <mutex>
#include <vector>

#include "tile.cuh"

namespace mb {

constexpr int NBUCKET = 32;
constexpr int SCHED_COUNTS = 32;    // int offsets inside the sched region
constexpr int SCHED_CURSORS = 64;

__device__ __forceinline__ int tile_bucket(int2 r) {
    const int w = r.y - r.x;
    return w > 0 ? __clz(w) - 1 : NBUCKET - 1;   // longer list -> smaller bucket
}

__global__ void k_tile_hist(const int2* __restrict__ ranges, int64_t n, int* __restrict__ counts) {
    __shared__ int h[NBUCKET];
    if (threadIdx.x < NBUCKET) h[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&h[tile_bucket(ranges[t])], 1);
    __syncthreads();
    if (threadIdx.x < NBUCKET && h[threadIdx.x]) atomicAdd(&counts[threadIdx.x], h[threadIdx.x]);
}

__global__ void k_tile_scatter(const int2* __restrict__ ranges, int64_t n, const int* __restrict__ counts,
                               int* __restrict__ cursors, int* __restrict__ order) {
    __shared__ int base[NBUCKET];
    if (threadIdx.x == 0) {
        int s = 0;
        for (int k = 0; k < NBUCKET; ++k) {
            base[k] = s;
            s += counts[k];
        }
    }
    __syncthreads();
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int k = tile_bucket(ranges[t]);
        order[base[k] + atomicAdd(&cursors[k], 1)] = (int)t;
    }
}

void launch_tile_order(const Layout& L, char* ws, cudaStream_t st) {
    if (L.n_tiles == 0) return;
    int* sched = reinterpret_cast<int*>(ws + L.sched);
    const int2* ranges = reinterpret_cast<const int2*>(ws + L.ranges);
    cudaMemsetAsync(sched, 0, SCHED_BYTES, st);
    const unsigned g = (unsigned)std::min<int64_t>(ceil_div64(L.n_tiles, 256), 608);
    count_launch(2);
    k_tile_hist<<<g, 256, 0, st>>>(ranges, L.n_tiles, sched + SCHED_COUNTS);
    k_tile_scatter<<<g, 256, 0, st>>>(ranges, L.n_tiles, sched + SCHED_COUNTS, sched + SCHED_CURSORS,
                                      reinterpret_cast<int*>(ws + L.order));
}

// CTAs of `func` resident on the whole device (one wave), cached per
// (device, kernel, shared memory).
static int resident_ctas(const void* func, size_t smem) {
    struct Entry {
        int dev;
        const void* func;
        size_t smem;
        int ctas;
    };
    static std::mutex mu;
    static std::vector<Entry> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    std::lock_guard<std::mutex> lock(mu);
    for (const Entry& e : cache)
        if (e.dev == dev && e.func == func && e.smem == smem) return e.ctas;
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, func, TPB, smem) != cudaSuccess)
        return 0;
    const int ctas = sms * std::max(per_sm, 1);
    cache.push_back({dev, func, smem, ctas});
    return ctas;
}

bool allow_dynamic_smem(const void* func, size_t smem) {
    static std::mutex mu;
    static std::vector<std::pair<int, const void*>> done;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    std::lock_guard<std::mutex> lock(mu);
    for (const auto& d : done)
        if (d.first == dev && d.second == func) return true;
    // the largest dynamic size any launch of this kernel uses (batch = TPB)
    if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return false;
    done.push_back({dev, func});
    return true;
}

TileLaunch tile_launch(const Params& p, const Layout& L, char* ws, int q, const void* func, size_t smem,
                       cudaStream_t st) {
    TileLaunch t;
    t.ts.n_tiles = L.n_tiles;
    t.ts.order = nullptr;
    t.ts.queue = nullptr;
    t.grid = (unsigned)L.n_tiles;
    if (p.schedule != MB3DGS_SCHEDULE_QUEUE) return t;
    const int ctas = resident_ctas(func, smem);
    if (ctas <= 0) {            // query failed: one CTA per tile, still in work order
        cudaGetLastError();
        t.grid = (unsigned)L.n_tiles;
    } else {
        t.grid = (unsigned)std::min<int64_t>(L.n_tiles, ctas);
    }
    int* sched = reinterpret_cast<int*>(ws + L.sched);
    cudaMemsetAsync(sched + q, 0, sizeof(int), st);
    t.ts.order = reinterpret_cast<const int*>(ws + L.order);
    t.ts.queue = sched + q;
    return t;
}

}  // namespace mb
