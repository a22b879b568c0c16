// FP32 FMA throughput of the current device: the denominator of the sweep
// kernel's roofline (the sweep is bound by the FP32 pipe, not by HBM or the
// tensor cores, and no vendor figure for the plain FP32 pipe of this part is
// measured elsewhere).  The paper has no counterpart.
//
// Every thread runs kChains independent chains of packed FP32 FMAs
// (__ffma2_rn, two lanes' worth of FMAs per instruction, the form the sweep
// uses) for a fixed number of rounds; the grid holds the maximum resident
// warps on every SM, so the pipe sees enough independent instructions to stay
// busy.  Each chain is x <- x * a + b with |a| < 1, so values stay bounded.
// The result is written only if it equals an impossible value, which keeps the
// compiler from dropping the chains.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/dd_inpaint.h"
#include "dd_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kRounds = 2048;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) fma2_peak_kernel(float* __restrict__ sink, float a, float b) {
    float2 x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = make_float2(threadIdx.x * 1e-3f + i, blockIdx.x * 1e-3f - i);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll 4
    for (int r = 0; r < kRounds; ++r)
#pragma unroll
        for (int i = 0; i < kChains; ++i) x[i] = __ffma2_rn(x[i], a2, b2);
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i].x + x[i].y;
    if (s == -1234.5f) sink[blockIdx.x] = s;
}

}  // namespace

extern "C" int dd_fp32_fma_peak(int reps, double* tflops, int* sm_count, void* stream) {
    if (reps < 1 || tflops == nullptr) {
        dd::set_last_error("dd_fp32_fma_peak: reps >= 1 and a result pointer are needed");
        return DD_EINVAL;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fma2_peak_kernel, kThreads, 0) != cudaSuccess) {
        dd::set_last_error("dd_fp32_fma_peak: device query failed");
        return DD_ECUDA;
    }
    const int grid = sms * std::max(per, 1);
    float* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = DD_OK;
    if (cudaMalloc(&sink, sizeof(float) * grid) != cudaSuccess) {
        dd::set_last_error("dd_fp32_fma_peak: cudaMalloc failed");
        return DD_ENOMEM;
    }
    float best = 0.f;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = DD_ECUDA;
    } else {
        fma2_peak_kernel<<<grid, kThreads, 0, st>>>(sink, 0.999f, 1e-3f);   // warm-up
        for (int r = 0; r < reps && rc == DD_OK; ++r) {
            float ms = 0.f;
            if (cudaEventRecord(e0, st) != cudaSuccess) { rc = DD_ECUDA; break; }
            fma2_peak_kernel<<<grid, kThreads, 0, st>>>(sink, 0.999f, 1e-3f);
            if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, st) != cudaSuccess ||
                cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                rc = DD_ECUDA;
                break;
            }
            if (ms > 0.f && (best == 0.f || ms < best)) best = ms;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    if (rc != DD_OK || !(best > 0.f)) {
        dd::set_last_error("dd_fp32_fma_peak: launch or timing failed");
        return DD_ECUDA;
    }
    // each __ffma2_rn is two FMAs of two flops each
    const double flops = (double)grid * kThreads * kRounds * kChains * 4.0;
    *tflops = flops / (best * 1e-3) / 1e12;
    if (sm_count) *sm_count = sms;
    return DD_OK;
}
