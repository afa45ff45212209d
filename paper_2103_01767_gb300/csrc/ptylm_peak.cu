// ptylm_peak.cu -- measured FP32 CUDA-core peak of the current device (instrumentation;
// the paper has no counterpart).  The GGN product of the hot path is bound by FP32
// arithmetic (its FFTs), so its roofline needs the rate at which this GPU, at the clocks it
// actually runs, retires FP32 fused multiply-adds.  k_ffma_loop keeps every SM's FP32 pipes
// busy with independent FMA chains; each timed launch counts 2 flops per FMA.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <vector>

#include "../../include/ptylm.h"
#include "kernels.h"

namespace {

// Written only when a chain sum takes a value the recurrence cannot reach, which keeps the
// compiler from removing the loop; device code names it directly.
__device__ float g_peak_sink[1];

constexpr int kChains = 8;      // independent FMA chains per thread (covers the FMA latency)
constexpr int kUnroll = 16;     // FMAs per chain per loop trip
constexpr int kThreads = 256;
constexpr int kCtasPerSm = 8;   // 2048 resident threads per SM

__global__ void __launch_bounds__(kThreads) k_ffma_loop(int iters, float seed) {
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + 1e-3f * (float)(c + threadIdx.x % 7);
    // a <- 0.999 a + 0.001 converges to 1, so the chains stay finite and normal
    const float m = 0.999f, add = 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], m, add);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == -1.0f) g_peak_sink[0] = s;
}

}  // namespace

extern "C" ptylm_status ptylm_fp32_peak(int launches, int iters, double* tflops_host, double* ms_host,
                                        void* stream_ptr) {
    ptylm::set_last_error("");
    if (launches < 1 || iters < 1 || !tflops_host) {
        ptylm::set_last_error("launches and iters must be >= 1 and tflops_host non-NULL");
        return PTYLM_ERR_ARG;
    }
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        ptylm::set_last_error("no usable CUDA device");
        return PTYLM_ERR_CUDA;
    }
    const int grid = sms * kCtasPerSm;
    const double flops = 2.0 * kChains * kUnroll * (double)iters * (double)grid * kThreads;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    std::vector<double> ms;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    // one untimed launch brings the clocks up
    if (e == cudaSuccess) {
        k_ffma_loop<<<grid, kThreads, 0, stream>>>(iters, 0.5f);
        e = cudaGetLastError();
    }
    for (int l = 0; l < launches && e == cudaSuccess; ++l) {
        e = cudaEventRecord(e0, stream);
        if (e == cudaSuccess) {
            k_ffma_loop<<<grid, kThreads, 0, stream>>>(iters, 0.5f + 1e-3f * l);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float t = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (e == cudaSuccess) ms.push_back(t);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        char msg[160];
        snprintf(msg, sizeof msg, "FFMA loop: %s", cudaGetErrorString(e));
        ptylm::set_last_error(msg);
        return PTYLM_ERR_CUDA;
    }
    std::sort(ms.begin(), ms.end());
    const double med = ms[ms.size() / 2];
    *tflops_host = flops / (med * 1e-3) / 1e12;
    if (ms_host) *ms_host = med;
    return PTYLM_OK;
}
