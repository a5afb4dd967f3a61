// Throughput probes of the two ALU pipes that bound the per-pair kernels:
// the FP32 FMA pipe and the MUFU (XU) special-function pipe.  They give the
// measured denominators of the ALU roofline (achieved work / peak), taken on
// the GPU at its current clocks instead of derived from unit counts.
//
// Each probe runs independent dependency chains per thread (enough chains and
// resident warps to hide the pipe latency) over a grid of several waves of
// full CTAs on every SM, timed with CUDA events on the caller's stream after
// one untimed launch.  The chains are kept alive by a store that only runs
// for an impossible value, so nothing is eliminated and nothing is written.
#include <cuda_runtime.h>

#include "common.cuh"

namespace mb {

constexpr int PROBE_CHAINS = 8;
constexpr int PROBE_TPB = 256;

__global__ void __launch_bounds__(PROBE_TPB) k_probe_ffma(float* __restrict__ sink, int iters, float a, float b) {
    float x[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = (float)(threadIdx.x + k) * 1e-3f;
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = fmaf(x[k], a, b);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s += x[k];
    if (s == 1234567.0f && sink) sink[threadIdx.x] = s;
}

// One MUFU instruction per chain step; the operand negation is a free source
// modifier, so x <- 2^-x and x <- rsqrt(x) stay finite and bounded.  The
// reciprocal chain is x <- 1/(x + 1) (an FADD on the FMA pipe beside each
// MUFU): x <- 1/x would let the compiler cancel pairs of reciprocals.
template <int OP>
__device__ __forceinline__ float mufu_op(float x) {
    float y;
    if (OP == 0) asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x));
    else if (OP == 1) asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    else if (OP == 2) asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x + 1.0f));
    else asm volatile("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int OP>
__global__ void __launch_bounds__(PROBE_TPB) k_probe_mufu(float* __restrict__ sink, int iters) {
    float x[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = 0.5f + (float)(threadIdx.x + k) * 1e-3f;
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = mufu_op<OP>(x[k]);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s += x[k];
    if (s == 1234567.0f && sink) sink[threadIdx.x] = s;
}

// Operations per second of one probe kernel: best of `reps` timed launches.
template <typename F>
static int time_probe(F launch, double ops_per_launch, int reps, cudaStream_t st, double* ops_per_s) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return MB3DGS_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return MB3DGS_ERR_CUDA;
    }
    launch();   // untimed: module load, clocks up
    float best = 1e30f;
    int rc = MB3DGS_OK;
    for (int r = 0; r < reps && rc == MB3DGS_OK; ++r) {
        cudaEventRecord(e0, st);
        launch();
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = MB3DGS_ERR_CUDA;
            break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms > 0.0f && ms < best) best = ms;
    }
    if (cudaGetLastError() != cudaSuccess) rc = MB3DGS_ERR_CUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == MB3DGS_OK) *ops_per_s = ops_per_launch / (best * 1e-3);
    return rc;
}

}  // namespace mb

extern "C" int mb3dgs_probe_alu_peaks(mb3dgs_alu_peaks* out, mb3dgs_stream_t stream) {
    using namespace mb;
    if (!out) return MB3DGS_ERR_INVALID_ARG;
    int dev = 0, sms = 0, blocks_per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MB3DGS_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MB3DGS_ERR_CUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_probe_ffma, PROBE_TPB, 0) != cudaSuccess)
        return MB3DGS_ERR_CUDA;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int waves = 4;
    const unsigned grid = (unsigned)(sms * (blocks_per_sm > 0 ? blocks_per_sm : 1) * waves);
    const double threads = (double)grid * PROBE_TPB;
    const int it_f = 512, it_m = 64;
    const double per_thread_f = (double)it_f * 16 * PROBE_CHAINS;
    const double per_thread_m = (double)it_m * 16 * PROBE_CHAINS;
    std::memset(out, 0, sizeof(*out));
    out->sm_count = sms;
    double v = 0.0;
    int rc = time_probe([&] { count_launch(); k_probe_ffma<<<grid, PROBE_TPB, 0, st>>>(nullptr, it_f, 0.999f, 1e-4f); },
                        threads * per_thread_f, 3, st, &v);
    if (rc) return rc;
    out->fp32_tflops = 2.0 * v / 1e12;   // one FFMA = 2 flop
    rc = time_probe([&] { count_launch(); k_probe_mufu<0><<<grid, PROBE_TPB, 0, st>>>(nullptr, it_m); },
                    threads * per_thread_m, 3, st, &v);
    if (rc) return rc;
    out->ex2_tops = v / 1e12;
    rc = time_probe([&] { count_launch(); k_probe_mufu<1><<<grid, PROBE_TPB, 0, st>>>(nullptr, it_m); },
                    threads * per_thread_m, 3, st, &v);
    if (rc) return rc;
    out->rsqrt_tops = v / 1e12;
    rc = time_probe([&] { count_launch(); k_probe_mufu<2><<<grid, PROBE_TPB, 0, st>>>(nullptr, it_m); },
                    threads * per_thread_m, 3, st, &v);
    if (rc) return rc;
    out->rcp_tops = v / 1e12;
    rc = time_probe([&] { count_launch(); k_probe_mufu<3><<<grid, PROBE_TPB, 0, st>>>(nullptr, it_m); },
                    threads * per_thread_m, 3, st, &v);
    if (rc) return rc;
    out->sin_tops = v / 1e12;
    return MB3DGS_OK;
}
