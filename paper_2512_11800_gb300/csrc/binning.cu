// Stage 2: tile binning by tile key only (no depth sort).
//
// counts[(v,i)] (tiles touched by each Gaussian's pixel rectangle) ->
// exclusive scan -> emission of (tile, Gaussian) pairs in (view, Gaussian)
// order -> stable LSD radix sort on the tile key (8-bit digits), which keeps
// each tile's Gaussians in ascending id order -> per-tile [start, end).
// All kernels are sized by the workspace's pair capacity and read the live
// pair count from device memory, so the stage needs no host round trip.
#include "common.cuh"

namespace mb {

constexpr int SCAN_TPB = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_CHUNK = SCAN_TPB * SCAN_ITEMS;  // elements per scan block

constexpr int SORT_TPB = 256;
constexpr int SORT_ROUNDS = 16;
constexpr int SORT_CHUNK = SORT_TPB * SORT_ROUNDS;  // pairs per sort block
constexpr int RADIX = 256;

// ---------------------------------------------------------------- scans
// Exclusive scans of int counts into int (tile pairs, radix histograms) or
// 64-bit (per-pixel offsets of the kept bound queries, whose total can pass
// 2^31) offsets.
template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* s_warp, T* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int nw = blockDim.x >> 5;
        T w = lane < nw ? s_warp[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) s_warp[lane] = w;
    }
    __syncthreads();
    T base = wid > 0 ? s_warp[wid - 1] : T(0);
    if (total) *total = s_warp[(blockDim.x >> 5) - 1];
    __syncthreads();
    return base + x - v;
}

// out[i] = sum_{j<i} in[j] within each block chunk; block sums to sums[b]
template <typename Tin, typename T>
__global__ void k_scan_blocks(const Tin* __restrict__ in, T* __restrict__ out, T* __restrict__ sums, int64_t n) {
    __shared__ T s_warp[32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_ITEMS;
    T vals[SCAN_ITEMS];
    T local = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        vals[k] = (base + k < n) ? (T)in[base + k] : T(0);
        local += vals[k];
    }
    T total;
    T pre = block_exclusive_scan<T>(local, s_warp, &total);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < n) out[base + k] = pre;
        pre += vals[k];
    }
    if (threadIdx.x == 0 && sums) sums[blockIdx.x] = total;
}

template <typename T>
__global__ void k_scan_add(T* __restrict__ out, const T* __restrict__ sums_scanned, int64_t n) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK;
    const T add = sums_scanned[blockIdx.x];
    for (int k = threadIdx.x; k < SCAN_CHUNK; k += blockDim.x)
        if (base + k < n) out[base + k] += add;
}

// Exclusive scan of n values (in may equal out).  tmp holds the block sums of
// every level: sum_l ceil(n / CHUNK^l) elements of T.
template <typename Tin, typename T>
static void exclusive_scan_t(const Tin* in, T* out, int64_t n, T* tmp, cudaStream_t st) {
    if (n <= 0) return;
    const int64_t nb = ceil_div64(n, SCAN_CHUNK);
    if (nb == 1) {
        count_launch();
        k_scan_blocks<Tin, T><<<1, SCAN_TPB, 0, st>>>(in, out, nullptr, n);
        return;
    }
    T* sums = tmp;
    count_launch();
    k_scan_blocks<Tin, T><<<(unsigned)nb, SCAN_TPB, 0, st>>>(in, out, sums, n);
    exclusive_scan_t<T, T>(sums, sums, nb, tmp + nb, st);
    count_launch();
    k_scan_add<T><<<(unsigned)nb, SCAN_TPB, 0, st>>>(out, sums, n);
}

void exclusive_scan(const int* in, int* out, int64_t n, int* tmp, cudaStream_t st) {
    exclusive_scan_t<int, int>(in, out, n, tmp, st);
}

void exclusive_scan64(const int* in, long long* out, int64_t n, long long* tmp, cudaStream_t st) {
    exclusive_scan_t<int, long long>(in, out, n, tmp, st);
}

size_t scan_tmp_elems(int64_t n) {
    size_t tot = 0;
    int64_t m = n;
    while (m > SCAN_CHUNK) {
        m = ceil_div64(m, SCAN_CHUNK);
        tot += (size_t)m;
    }
    return tot + 16;
}

// ---------------------------------------------------------------- pair emission
__global__ void k_pair_total(const int* __restrict__ counts, const int* __restrict__ offsets, int64_t VP, int64_t cap,
                             StatusWords* sw) {
    long long tot = VP > 0 ? (long long)offsets[VP - 1] + counts[VP - 1] : 0;
    sw->n_total = tot;
    if (tot > cap) {
        atomicMin(&sw->status, (int)MB3DGS_ERR_CAPACITY);
        sw->n_valid = 0;
    } else {
        sw->n_valid = tot;
    }
}

// counts are scanned in 64-bit-safe fashion only up to 2^31 pairs; the
// capacity is validated on the host to stay below that.
__global__ void k_emit_pairs(ViewTable vt, const float* __restrict__ rec, const int* __restrict__ counts,
                             const int* __restrict__ offsets, int64_t P, int64_t cap, StatusWords* sw,
                             uint32_t* __restrict__ keys, int32_t* __restrict__ vals) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= P * vt.n_views) return;
    if (sw->n_valid == 0) return;
    const int c = counts[idx];
    if (c == 0) return;
    const int v = (int)(idx / P);
    const int32_t gi = (int32_t)(idx - (int64_t)v * P);
    const int* ri = reinterpret_cast<const int*>(rec + idx * REC + R_RECT);
    const ViewDesc& V = vt.v[v];
    const int tx0 = ri[0] / V.tile_w, ty0 = ri[1] / V.tile_h, tx1 = ri[2] / V.tile_w, ty1 = ri[3] / V.tile_h;
    int64_t o = offsets[idx];
    if (o < 0 || o + c > cap) {       // never write past the pair arrays
        atomicMin(&sw->status, (int)MB3DGS_ERR_CAPACITY);
        return;
    }
    for (int ty = ty0; ty <= ty1; ++ty)
        for (int tx = tx0; tx <= tx1; ++tx) {
            keys[o] = (uint32_t)(V.tile_base + ty * V.tiles_x + tx);
            vals[o] = gi;
            ++o;
        }
}

// ---------------------------------------------------------------- radix sort
__global__ void k_radix_hist(const uint32_t* __restrict__ keys, const StatusWords* sw, int shift, int nb,
                             uint32_t* __restrict__ hist) {
    __shared__ uint32_t s_h[RADIX];
    s_h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t n = sw->n_valid;
    const int64_t base = (int64_t)blockIdx.x * SORT_CHUNK;
    if (base < n) {
        for (int k = 0; k < SORT_ROUNDS; ++k) {
            const int64_t i = base + (int64_t)k * SORT_TPB + threadIdx.x;
            if (i < n) atomicAdd(&s_h[(keys[i] >> shift) & (RADIX - 1)], 1u);
        }
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nb + blockIdx.x] = s_h[threadIdx.x];
}

__global__ void k_radix_scatter(const uint32_t* __restrict__ keys, const int32_t* __restrict__ vals,
                                uint32_t* __restrict__ okeys, int32_t* __restrict__ ovals,
                                const uint32_t* __restrict__ hist_scanned, const StatusWords* sw, int shift, int nb) {
    __shared__ uint32_t s_run[RADIX];
    __shared__ uint32_t s_warp[SORT_TPB / 32][RADIX];
    const int64_t n = sw->n_valid;
    const int64_t base = (int64_t)blockIdx.x * SORT_CHUNK;
    if (base >= n) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    s_run[threadIdx.x] = hist_scanned[(int64_t)threadIdx.x * nb + blockIdx.x];
    const uint32_t lt_mask = (1u << lane) - 1u;
    for (int k = 0; k < SORT_ROUNDS; ++k) {
        const int64_t i = base + (int64_t)k * SORT_TPB + threadIdx.x;
        const bool valid = i < n;
        const uint32_t key = valid ? keys[i] : 0u;
        const int32_t val = valid ? vals[i] : 0;
        const uint32_t digit = valid ? ((key >> shift) & (RADIX - 1)) : RADIX;  // RADIX = "none"
#pragma unroll
        for (int w = 0; w < SORT_TPB / 32; ++w) s_warp[w][threadIdx.x] = 0;
        __syncthreads();
        const uint32_t peers = __match_any_sync(0xffffffffu, digit);
        const uint32_t rank = __popc(peers & lt_mask);
        const int leader = __ffs(peers) - 1;
        if (valid && lane == leader) s_warp[wid][digit] = __popc(peers);
        __syncthreads();
        {
            const int d = threadIdx.x;
            uint32_t run = s_run[d];
#pragma unroll
            for (int w = 0; w < SORT_TPB / 32; ++w) {
                const uint32_t c = s_warp[w][d];
                s_warp[w][d] = run;
                run += c;
            }
            s_run[d] = run;
        }
        __syncthreads();
        if (valid) {
            const uint32_t pos = s_warp[wid][digit] + rank;
            okeys[pos] = key;
            ovals[pos] = val;
        }
        __syncthreads();
    }
}

// scan of the 256 x nb histogram (uint32 viewed as int; totals < 2^31)
void radix_sort(uint32_t* keys0, int32_t* vals0, uint32_t* keys1, int32_t* vals1, uint32_t* hist, int* scan_tmp,
                const StatusWords* sw, int nb, int passes, cudaStream_t st) {
    uint32_t* kin = keys0;
    int32_t* vin = vals0;
    uint32_t* kout = keys1;
    int32_t* vout = vals1;
    for (int ps = 0; ps < passes; ++ps) {
        const int shift = 8 * ps;
        count_launch();
        k_radix_hist<<<nb, RADIX, 0, st>>>(kin, sw, shift, nb, hist);
        exclusive_scan(reinterpret_cast<int*>(hist), reinterpret_cast<int*>(hist), (int64_t)RADIX * nb, scan_tmp, st);
        count_launch();
        k_radix_scatter<<<nb, SORT_TPB, 0, st>>>(kin, vin, kout, vout, hist, sw, shift, nb);
        uint32_t* tk = kin; kin = kout; kout = tk;
        int32_t* tv = vin; vin = vout; vout = tv;
    }
}

__global__ void k_tile_ranges(const uint32_t* __restrict__ keys, const StatusWords* sw, int2* __restrict__ ranges) {
    const int64_t n = sw->n_valid;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t k = keys[i];
    if (i == 0 || keys[i - 1] != k) ranges[k].x = (int)i;
    if (i == n - 1 || keys[i + 1] != k) ranges[k].y = (int)(i + 1);
}

void launch_binning(const ViewTable& vt, const Layout& L, char* ws, cudaStream_t st) {
    const int64_t VP = L.VP;
    int* counts = reinterpret_cast<int*>(ws + L.counts);
    int* offsets = reinterpret_cast<int*>(ws + L.offsets);
    int* tmp = reinterpret_cast<int*>(ws + L.scan_tmp);
    StatusWords* sw = reinterpret_cast<StatusWords*>(ws + L.status);
    float* rec = reinterpret_cast<float*>(ws + L.rec);
    uint32_t* keys0 = reinterpret_cast<uint32_t*>(ws + L.keys[0]);
    uint32_t* keys1 = reinterpret_cast<uint32_t*>(ws + L.keys[1]);
    int32_t* vals0 = reinterpret_cast<int32_t*>(ws + L.vals[0]);
    int32_t* vals1 = reinterpret_cast<int32_t*>(ws + L.vals[1]);
    uint32_t* hist = reinterpret_cast<uint32_t*>(ws + L.hist);
    int2* ranges = reinterpret_cast<int2*>(ws + L.ranges);

    cudaMemsetAsync(ranges, 0, sizeof(int2) * (size_t)L.n_tiles, st);
    if (VP == 0) {
        cudaMemsetAsync(&sw->n_total, 0, 16, st);
        return;
    }
    exclusive_scan(counts, offsets, VP, tmp, st);
    count_launch();
    k_pair_total<<<1, 1, 0, st>>>(counts, offsets, VP, L.cap, sw);
    count_launch();
    k_emit_pairs<<<(unsigned)ceil_div64(VP, 128), 128, 0, st>>>(vt, rec, counts, offsets, L.P, L.cap, sw, keys0,
                                                                vals0);
    if (L.sort_passes > 0)
        radix_sort(keys0, vals0, keys1, vals1, hist, tmp, sw, L.nb_sort, L.sort_passes, st);
    const uint32_t* kf = reinterpret_cast<const uint32_t*>(ws + L.keys[L.final_buf]);
    if (L.cap > 0) {
        count_launch();
        k_tile_ranges<<<(unsigned)ceil_div64(L.cap, 256), 256, 0, st>>>(kf, sw, ranges);
    }
}

}  // namespace mb
