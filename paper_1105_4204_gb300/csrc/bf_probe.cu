// Measured throughput of the FP32 FMA pipe (not part of the filter).
//
// The filter's kernels are bound by plain FP32 arithmetic, not by HBM or the
// tensor cores, so their roofline denominator is the rate at which the SMs
// retire FP32 lane operations.  The nominal figure is SMs x 128 lanes x SM
// clock; this kernel measures what the device actually sustains: every
// resident thread runs kChains independent FMA chains (enough to hide the
// pipe's latency), the scalar form one FFMA per lane operation, the paired
// form one FFMA2 per two.
#include <cuda_runtime.h>

#include "bf_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;   // 2048 resident threads per SM
constexpr int kIters = 2048;      // loop trips per thread
constexpr int kTimedLaunches = 5;

__device__ float g_probe_sink;

__global__ void __launch_bounds__(kThreads, kBlocksPerSm)
    fp32_pipe_scalar(float a, float b, int iters) {
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    // the chains converge to b / (1 - a) per lane; the store keeps them live
    if (s == -1.0f) g_probe_sink = s;
}

__global__ void __launch_bounds__(kThreads, kBlocksPerSm)
    fp32_pipe_paired(float a, float b, int iters) {
    float2 x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k)
        x[k] = make_float2((float)(threadIdx.x + k) * 1e-3f, (float)(threadIdx.x - k) * 1e-3f);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = __ffma2_rn(x[k], a2, b2);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k].x + x[k].y;
    if (s == -1.0f) g_probe_sink = s;
}

}  // namespace

using namespace bf;

extern "C" bf_status bf_fp32_pipe_rate(int paired, double *lane_ops_per_s, cudaStream_t stream) {
    if (!lane_ops_per_s) return fail(BF_EINVAL, "bf_fp32_pipe_rate: lane_ops_per_s is NULL");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_check(e, "bf_fp32_pipe_rate: device query");
    const int grid = sms * kBlocksPerSm;
    auto kern = paired ? fp32_pipe_paired : fp32_pipe_scalar;
    const float a = 0.999f, b = 1e-3f;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {  // warm-up: clocks up, module loaded
        kern<<<grid, kThreads, 0, stream>>>(a, b, kIters);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(t0, stream);
    for (int i = 0; i < kTimedLaunches && e == cudaSuccess; ++i) {
        kern<<<grid, kThreads, 0, stream>>>(a, b, kIters);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(t1, stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (e != cudaSuccess) return cuda_check(e, "bf_fp32_pipe_rate");
    if (!(ms > 0.f)) return fail(BF_ECUDA, "bf_fp32_pipe_rate: zero elapsed time");
    const double ops = (double)kTimedLaunches * grid * kThreads * (double)kIters * kUnroll *
                       kChains * (paired ? 2.0 : 1.0);
    *lane_ops_per_s = ops / (ms * 1e-3);
    return BF_OK;
}
