// learned_kernels.cu -- kernels of the learned initialisation besides the convolutions
// (see learned.h; the tensor-core convolutions are in conv_tc.cu): Adam, the probe-support
// mask, the physics input and training pairs, and the overlap stitching.
//
// The physics input and the training pairs run the team FFT of the GGN product on one
// 128 x 128 pattern per 512-thread CTA.
#include <cuda_bf16.h>

#include <algorithm>

#include "learned.h"
#include "ptycho_device.cuh"
#include "team_fft.cuh"

namespace ptylm {

namespace {

__global__ void k_adam(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v, const float* __restrict__ g,
                       long n, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

__global__ void k_support(const float2* __restrict__ P, float* __restrict__ mask, int M) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x)
        mask[i] = (P[i].x != 0.0f || P[i].y != 0.0f) ? 1.0f : 0.0f;
}

using G7 = Geo<7>;

// u = F(P) / max(|F(P)|, 1e-3 max|F(P)|) in team-register order (element e of thread t at
// e*T + t).
__global__ void __launch_bounds__(G7::THREADS) k_probe_phasor(const float2* __restrict__ P, const float2* tw,
                                                              float2* __restrict__ u) {
    using G = G7;
    TeamCtx<G> c = team_setup<G>(tw);
    const int x = c.tid & (G::S - 1), b = c.tid >> G::LOG_S;
    float2 v[32];
#pragma unroll
    for (int a = 0; a < 32; ++a) v[a] = P[(G::BX * a + b) * G::S + x];
    team_fft_fwd<G>(v, c.sm, c.tw, c.tid);
    float mx = 0.0f;
#pragma unroll
    for (int e = 0; e < 32; ++e) mx = fmaxf(mx, v[e].x * v[e].x + v[e].y * v[e].y);
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    __shared__ float red[G::T / 32];
    if ((c.tid & 31) == 0) red[c.tid >> 5] = mx;
    __syncthreads();
    mx = 0.0f;
    for (int q = 0; q < G::T / 32; ++q) mx = fmaxf(mx, red[q]);
    const float floor_mag = 1e-3f * sqrtf(mx);   // u fades where F(P) nearly vanishes
#pragma unroll
    for (int e = 0; e < 32; ++e) {
        const float r = fmaxf(sqrtf(v[e].x * v[e].x + v[e].y * v[e].y), floor_mag);
        u[e * G::T + c.tid] = make_float2(v[e].x / r, v[e].y / r);
    }
}

// Object estimate from the back-propagated field e (pass-1 layout) into channel planes.
__device__ __forceinline__ void write_estimate(const float2* v, const float2* __restrict__ P, float eps_abs,
                                               float* __restrict__ X, int tid) {
    using G = G7;
    const int x = tid & (G::S - 1), b = tid >> G::LOG_S;
#pragma unroll
    for (int a = 0; a < 32; ++a) {
        const int yy = G::BX * a + b;
        const float2 p = P[yy * G::S + x];
        const float inv = 1.0f / (p.x * p.x + p.y * p.y + eps_abs);
        const float2 est = cmulc(v[a], p);   // e conj(P)
        X[yy * G::S + x] = est.x * inv;
        X[G::M + yy * G::S + x] = est.y * inv;
    }
}

__global__ void __launch_bounds__(G7::THREADS) k_learn_pairs(const float2* __restrict__ pool, int side,
                                                             const int4* __restrict__ samples, const float2* __restrict__ P,
                                                             const float2* __restrict__ u, const float2* tw, float eps_abs,
                                                             float* __restrict__ X, float* __restrict__ T) {
    using G = G7;
    TeamCtx<G> c = team_setup<G>(tw);
    const int4 smp = samples[blockIdx.x];
    const float2* O = pool + (size_t)smp.x * side * side;
    float2 v[32];
    gather_times_probe<G>(v, O, P, side, smp.y, smp.z, c.tid);   // psi = P . O patch
    const float invM = 1.0f / G::M;
    team_fft_roundtrip<G>(v, c.sm, c.tw, c.tid, [&](float2* g, int j) {
#pragma unroll
        for (int k2y = 0; k2y < G::BY; ++k2y) {
            const int e = j * G::BY + k2y;
            const float mag = sqrtf(g[k2y].x * g[k2y].x + g[k2y].y * g[k2y].y) * invM;
            g[k2y] = u[e * G::T + c.tid] * mag;   // |F psi| with the probe's far-field phase
        }
    });
    write_estimate(v, P, eps_abs, X + (size_t)blockIdx.x * 2 * G::M, c.tid);
    const int x = c.tid & (G::S - 1), b = c.tid >> G::LOG_S;
    float* Tk = T + (size_t)blockIdx.x * 2 * G::M;
#pragma unroll 4
    for (int a = 0; a < 32; ++a) {
        const int yy = G::BX * a + b;
        const float2 o = O[(size_t)(smp.y + yy) * side + smp.z + x];
        Tk[yy * G::S + x] = o.x;
        Tk[G::M + yy * G::S + x] = o.y;
    }
}

__global__ void __launch_bounds__(G7::THREADS) k_physics_inputs(const float* __restrict__ y, int take_sqrt,
                                                                const int* __restrict__ idx, const float2* __restrict__ P,
                                                                const float2* __restrict__ u, const float2* tw,
                                                                float eps_abs, float* __restrict__ X) {
    using G = G7;
    TeamCtx<G> c = team_setup<G>(tw);
    const int k = idx[blockIdx.x];
    const float* yk = y + (size_t)k * G::M + c.tid;
    const float invS = 1.0f / G::S;
    float2 v[32];
#pragma unroll
    for (int e = 0; e < 32; ++e) {
        const float ym = __ldg(yk + e * G::T);
        const float mag = take_sqrt ? sqrtf(fmaxf(ym, 0.0f)) : ym;
        v[e] = u[e * G::T + c.tid] * (mag * invS);
    }
    team_fft_inv<G>(v, c.sm, c.tw, c.tid);
    write_estimate(v, P, eps_abs, X + (size_t)blockIdx.x * 2 * G::M, c.tid);
}

__global__ void __launch_bounds__(256) k_stitch_acc(const float* __restrict__ est, const int* __restrict__ idx,
                                                    const int2* __restrict__ pos, const float2* __restrict__ P, int S,
                                                    int nx, float2* num, float* den) {
    const int i = blockIdx.x;
    const int2 rc = pos[idx[i]];
    const int M = S * S;
    const float* E = est + (size_t)i * 2 * M;
    for (int p = threadIdx.x; p < M; p += blockDim.x) {
        const float2 q = P[p];
        const float w = q.x * q.x + q.y * q.y;
        if (w == 0.0f) continue;
        const size_t o = (size_t)(rc.x + p / S) * nx + rc.y + p % S;
        atomicAdd(&num[o].x, w * E[p]);
        atomicAdd(&num[o].y, w * E[M + p]);
        atomicAdd(&den[o], w);
    }
}

__global__ void k_stitch_fin(const float2* __restrict__ num, const float* __restrict__ den, long N, float2* __restrict__ O) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
        const float d = den[i];
        O[i] = d > 0.0f ? make_float2(num[i].x / d, num[i].y / d) : make_float2(1.0f, 0.0f);
    }
}

int blocks_for(long n) { return (int)std::min<long>(4096, std::max<long>(1, (n + 255) / 256)); }

bool team_smem_ready = false;
cudaError_t prepare_team_kernels() {
    if (team_smem_ready) return cudaSuccess;
    const int smem = (int)(sizeof(float2) * (G7::TW_WORDS + G7::EXW));
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_probe_phasor, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_learn_pairs, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_physics_inputs, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess) return e;
    team_smem_ready = true;
    return cudaSuccess;
}
size_t team_smem() { return sizeof(float2) * (G7::TW_WORDS + G7::EXW); }

}  // namespace

cudaError_t adam_step(float* w, float* m, float* v, const float* g, long n, float lr, float b1, float b2, float eps,
                      int t, cudaStream_t st) {
    const float c1 = 1.0f / (1.0f - powf(b1, (float)t)), c2 = 1.0f / (1.0f - powf(b2, (float)t));
    k_adam<<<blocks_for(n), 256, 0, st>>>(w, m, v, g, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t support_mask(const float2* P, float* mask, int M, cudaStream_t st) {
    k_support<<<blocks_for(M), 256, 0, st>>>(P, mask, M);
    return cudaGetLastError();
}

cudaError_t probe_phasor(const float2* P, const float2* tw, float2* u, cudaStream_t st) {
    cudaError_t e = prepare_team_kernels();
    if (e != cudaSuccess) return e;
    k_probe_phasor<<<1, G7::THREADS, team_smem(), st>>>(P, tw, u);
    return cudaGetLastError();
}

cudaError_t learn_pairs(const float2* pool, int side, const int4* samples, int N, const float2* P, const float2* u,
                        const float2* tw, float eps_abs, float* X, float* T, cudaStream_t st) {
    cudaError_t e = prepare_team_kernels();
    if (e != cudaSuccess) return e;
    if (N <= 0) return cudaSuccess;
    k_learn_pairs<<<N, G7::THREADS, team_smem(), st>>>(pool, side, samples, P, u, tw, eps_abs, X, T);
    return cudaGetLastError();
}

cudaError_t physics_inputs(const float* y_team, int take_sqrt, const int* idx, int n, const float2* P, const float2* u,
                           const float2* tw, float eps_abs, float* X, cudaStream_t st) {
    cudaError_t e = prepare_team_kernels();
    if (e != cudaSuccess) return e;
    if (n <= 0) return cudaSuccess;
    k_physics_inputs<<<n, G7::THREADS, team_smem(), st>>>(y_team, take_sqrt, idx, P, u, tw, eps_abs, X);
    return cudaGetLastError();
}

cudaError_t stitch_accumulate(const float* est, const int* idx, int n, const int2* pos, const float2* P, int nx,
                              float2* num, float* den, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_stitch_acc<<<n, 256, 0, st>>>(est, idx, pos, P, G7::S, nx, num, den);
    return cudaGetLastError();
}

cudaError_t stitch_finish(const float2* num, const float* den, long N, float2* O, cudaStream_t st) {
    k_stitch_fin<<<blocks_for(N), 256, 0, st>>>(num, den, N, O);
    return cudaGetLastError();
}

}  // namespace ptylm
