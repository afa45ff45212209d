// ptylm_noalloc.cu -- ptylm_forward_loss_noalloc: the error metric f and ||grad_zeta l||^2
// at (O, P) without a context and without allocating device memory.
//
// Some callers must not allocate device memory: serving or real-time loops that reserve
// all their memory at start-up (cudaMalloc and cudaFree can synchronise the device and take
// unbounded time), plug-ins inside a host framework whose memory pool already holds nearly
// all of the device memory, and code whose device bytes must all be accounted to another
// allocator.  This entry point takes inputs and outputs from the caller and keeps its only
// scratch -- twiddle tables, one FP64 partial pair per CTA, the reduction counter, an error
// flag and two result slots -- in the file-scope device array g_noalloc_scratch below,
// which every GPU that loads the library holds until the process exits.  All calls share
// it: calls whose work overlaps on the GPU race.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <cstdint>

#include "../../include/ptylm.h"
#include "kernels.h"
#include "ptycho_device.cuh"
#include "reduce.cuh"
#include "team_fft.cuh"

// Scratch layout (bytes): see kTwOffset ... kResultOffset below.  File scope, static: one copy
// per GPU that loads the library, alive until process exit.  Host code must not use its
// name as an address (it is a host-side stand-in); it uses cudaGetSymbolAddress instead.
static __device__ __align__(256) unsigned char g_noalloc_scratch[PTYLM_NOALLOC_SCRATCH_BYTES];

namespace {

using namespace ptylm;

// Scratch layout (bytes): twiddles for sides 32, 64, 128 | partials | counter, flag | result.
constexpr int kMaxCtas = PTYLM_NOALLOC_MAX_CTAS;
constexpr size_t kTwOffset = 0;                                   // 224 float2
constexpr size_t kTwBytes = sizeof(float2) * (32 + 64 + 128);
constexpr size_t kPartOffset = 2048;
constexpr size_t kPartBytes = sizeof(double) * 2 * kMaxCtas;
constexpr size_t kCounterOffset = kPartOffset + kPartBytes;      // unsigned counter, int flag
constexpr size_t kResultOffset = kCounterOffset + 256;            // double[2]
constexpr size_t kScratchBytes = kResultOffset + 256;
static_assert(kScratchBytes == PTYLM_NOALLOC_SCRATCH_BYTES, "header constant out of date");
static_assert(kTwBytes <= kPartOffset, "twiddle tables overflow their slot");

size_t tw_offset(int LS) {  // tables for 32, 64, 128 back to back
    return kTwOffset + sizeof(float2) * (LS == 5 ? 0 : LS == 6 ? 32 : 96);
}

// Error metric of one position set, natural-order measurements; out-of-range positions set
// the flag and are skipped (the check is uniform across a team, so barriers stay matched).
template <int LS>
__global__ void __launch_bounds__(Geo<LS>::THREADS, 512 / Geo<LS>::THREADS)
k_loss_noalloc(const float2* __restrict__ O, const float2* __restrict__ P, const int2* __restrict__ pos,
               const float* __restrict__ y, int K, int ny, int nx, float b, int loss, const float2* tw_g,
               double* partials, unsigned* counter, int* flag, double* result) {
    using G = Geo<LS>;
    TeamCtx<G> c = team_setup<G>(tw_g);
    const float invS = 1.0f / G::S;
    const int ky = freq_ky<G>(c.tid);
    double acc_l = 0.0, acc_d = 0.0;
    float2 v[32];
    for (int k = blockIdx.x * G::TEAMS + c.team; k < K; k += gridDim.x * G::TEAMS) {
        const int2 rc = pos[k];
        if (rc.x < 0 || rc.y < 0 || rc.x > ny - G::S || rc.y > nx - G::S) {
            if (c.tid == 0) atomicOr(flag, 1);
            continue;
        }
        gather_times_probe<G>(v, O, P, nx, rc.x, rc.y, c.tid);
        team_fft_fwd<G>(v, c.sm, c.tw, c.tid);
        const float* yk = y + (size_t)k * G::M + ky * G::S;
        float sl = 0.0f, sd = 0.0f;
#pragma unroll
        for (int e = 0; e < 32; ++e) {
            const float2 ps = v[e] * invS;
            const float h = ps.x * ps.x + ps.y * ps.y + b;
            const float yv = __ldg(yk + freq_kx<G>(c.tid, e));
            const PixelTerms t = pixel_terms<true>(loss, h, loss == 0 ? sqrtf(yv) : yv);
            sl += t.l;
            sd += t.dl * t.dl;
        }
        acc_l += (double)sl;
        acc_d += (double)sd;
        team_sync<G>();
    }
    double sums[2] = {acc_l, acc_d};
    grid_reduce<2>(sums, partials, counter, result, 0, OP_STORE, 1.0);
}

const void* kernel_for(int LS) {
    switch (LS) {
        case 5: return (const void*)k_loss_noalloc<5>;
        case 6: return (const void*)k_loss_noalloc<6>;
        case 7: return (const void*)k_loss_noalloc<7>;
    }
    return nullptr;
}

size_t smem_bytes(int LS) {
    switch (LS) {
        case 5: return sizeof(float2) * (Geo<5>::TW_WORDS + Geo<5>::TEAMS * Geo<5>::EXW);
        case 6: return sizeof(float2) * (Geo<6>::TW_WORDS + Geo<6>::TEAMS * Geo<6>::EXW);
        case 7: return sizeof(float2) * (Geo<7>::TW_WORDS + Geo<7>::TEAMS * Geo<7>::EXW);
    }
    return 0;
}

int threads_for(int LS) {
    switch (LS) {
        case 5: return Geo<5>::THREADS;
        case 6: return Geo<6>::THREADS;
        case 7: return Geo<7>::THREADS;
    }
    return 0;
}

int teams_for(int LS) {
    switch (LS) {
        case 5: return Geo<5>::TEAMS;
        case 6: return Geo<6>::TEAMS;
        case 7: return Geo<7>::TEAMS;
    }
    return 0;
}

// Per-device state, set up by the first call on that device.
constexpr int kMaxDevices = 64;
struct DeviceState {
    bool ready = false;
    unsigned char* base = nullptr;  // device address of g_noalloc_scratch
    int num_sms = 0;
    int ctas_per_sm[3] = {0, 0, 0};
};
DeviceState g_dev[kMaxDevices];
std::mutex g_mutex;
ptylm_status fail(ptylm_status s, const char* fmt, ...) {
    char msg[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof msg, fmt, ap);
    va_end(ap);
    set_last_error(msg);
    return s;
}

// Once per device, with that device current: the scratch's device address, the twiddle
// tables W_S^j = exp(-2 pi i j / S) (FP64, rounded once), kernel attributes and occupancy.
ptylm_status setup_device(int dev, DeviceState** out) {
    std::lock_guard<std::mutex> lock(g_mutex);
    DeviceState& d = g_dev[dev];
    if (!d.ready) {
        void* base = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&base, g_noalloc_scratch);
        if (e != cudaSuccess) return fail(PTYLM_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        float2 tw[32 + 64 + 128];
        int o = 0;
        for (int S : {32, 64, 128})
            for (int j = 0; j < S; ++j, ++o) {
                const double ang = 2.0 * M_PI * (double)j / (double)S;
                tw[o] = make_float2((float)std::cos(ang), (float)-std::sin(ang));
            }
        e = cudaMemcpy(static_cast<unsigned char*>(base) + kTwOffset, tw, kTwBytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail(PTYLM_ERR_CUDA, "uploading twiddles: %s", cudaGetErrorString(e));
        e = cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return fail(PTYLM_ERR_CUDA, "device attribute: %s", cudaGetErrorString(e));
        for (int LS = 5; LS <= 7; ++LS) {
            const void* fn = kernel_for(LS);
            e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(LS));
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d.ctas_per_sm[LS - 5], fn, threads_for(LS),
                                                                  smem_bytes(LS));
            if (e != cudaSuccess || d.ctas_per_sm[LS - 5] <= 0)
                return fail(PTYLM_ERR_CUDA, "kernel for side %d cannot launch: %s", 1 << LS,
                            e != cudaSuccess ? cudaGetErrorString(e) : "zero occupancy");
        }
        d.base = static_cast<unsigned char*>(base);
        d.ready = true;
    }
    *out = &d;
    return PTYLM_OK;
}

}  // namespace

extern "C" ptylm_status ptylm_forward_loss_noalloc(int ny, int nx, int m, int K, int loss, float background,
                                                   const ptylm_c64* O, const ptylm_c64* P,
                                                   const int32_t* positions, const float* y, double* out_dev,
                                                   void* stream_ptr) {
    set_last_error("");
    int LS = 0;
    if (m == 32) LS = 5;
    else if (m == 64) LS = 6;
    else if (m == 128) LS = 7;
    else return fail(PTYLM_ERR_ARG, "probe side %d beyond the allocation-free path (32, 64 or 128)", m);
    if (ny < m || nx < m || K < 0) return fail(PTYLM_ERR_ARG, "object %dx%d, probe %d, K=%d invalid", ny, nx, m, K);
    if ((long)ny * nx > (1L << 31)) return fail(PTYLM_ERR_ARG, "object too large");
    if (loss != PTYLM_LOSS_GAUSSIAN && loss != PTYLM_LOSS_POISSON) return fail(PTYLM_ERR_ARG, "unknown loss %d", loss);
    if (!(background > 0.0f) || !std::isfinite(background)) return fail(PTYLM_ERR_ARG, "background must be > 0");
    if (!out_dev || (K > 0 && (!O || !P || !positions || !y))) return fail(PTYLM_ERR_ARG, "NULL array");
    if (reinterpret_cast<uintptr_t>(positions) % 8 != 0) return fail(PTYLM_ERR_ARG, "positions must be 8-byte aligned");
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return fail(PTYLM_ERR_CUDA, "no usable CUDA device");
    }
    DeviceState* d = nullptr;
    ptylm_status s = setup_device(dev, &d);
    if (s != PTYLM_OK) return s;
    unsigned* counter = reinterpret_cast<unsigned*>(d->base + kCounterOffset);
    int* flag = reinterpret_cast<int*>(d->base + kCounterOffset + sizeof(unsigned));
    double* result = reinterpret_cast<double*>(d->base + kResultOffset);
    // counter and flag must start at zero (the result and partials are fully overwritten)
    cudaError_t e = cudaMemsetAsync(d->base + kCounterOffset, 0, 2 * sizeof(unsigned), stream);
    if (e != cudaSuccess) return fail(PTYLM_ERR_CUDA, "clearing scratch: %s", cudaGetErrorString(e));
    if (K == 0) {
        e = cudaMemsetAsync(out_dev, 0, 2 * sizeof(double), stream);
        if (e != cudaSuccess) return fail(PTYLM_ERR_CUDA, "%s", cudaGetErrorString(e));
        return PTYLM_OK;
    }
    const int teams = teams_for(LS);
    const int grid = std::min({d->ctas_per_sm[LS - 5] * d->num_sms, (K + teams - 1) / teams, kMaxCtas});
    const float2* Od = reinterpret_cast<const float2*>(O);
    const float2* Pd = reinterpret_cast<const float2*>(P);
    const int2* posd = reinterpret_cast<const int2*>(positions);
    const float2* tw = reinterpret_cast<const float2*>(d->base + tw_offset(LS));
    double* partials = reinterpret_cast<double*>(d->base + kPartOffset);
    void* args[] = {&Od, &Pd, &posd, &y, &K, &ny, &nx, &background, &loss, &tw, &partials, &counter, &flag, &result};
    e = cudaLaunchKernel(kernel_for(LS), dim3(grid), dim3(threads_for(LS)), args, smem_bytes(LS), stream);
    if (e != cudaSuccess) return fail(PTYLM_ERR_CUDA, "launch: %s", cudaGetErrorString(e));
    e = cudaMemcpyAsync(out_dev, result, 2 * sizeof(double), cudaMemcpyDeviceToDevice, stream);
    int host_flag = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&host_flag, flag, sizeof(int), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return fail(PTYLM_ERR_CUDA, "%s", cudaGetErrorString(e));
    if (host_flag) return fail(PTYLM_ERR_ARG, "a position lies outside [0, %d] x [0, %d]", ny - m, nx - m);
    return PTYLM_OK;
}
