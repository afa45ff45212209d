// learned_kernels.cu -- kernels of the learned initialisation (see learned.h).
//
// Convolutions are direct 3x3 correlations on 16 x 16 output tiles: each CTA stages an
// input tile (with halo; upsampled coordinates read the low-resolution input at half the
// index) and the bfloat16 weights of 8 input channels in shared memory, and every thread
// accumulates COT output channels of one pixel in FP32 registers.  The backward pass uses
// the same kernel on the transposed, flipped weights (stride-1 layers, followed by a 2 x 2
// sum for the upsampling), a gather kernel for the stride-2 layers, and a per-(out, in)
// channel reduction with FP32 atomics for the weight gradients.
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

constexpr int TS = 16;   // output tile side
constexpr int CIT = 8;   // input channels staged per round

template <int COT, int STRIDE, bool UP>
__global__ void __launch_bounds__(256) k_conv_fwd(ConvShape s, const float* __restrict__ x,
                                                  const __nv_bfloat16* __restrict__ w, const float* __restrict__ bias,
                                                  float* __restrict__ y) {
    constexpr int IT = (TS - 1) * STRIDE + 3;
    __shared__ float sx[CIT][IT][IT + 1];
    __shared__ float sw[CIT][9][COT];
    const int Hu = UP ? 2 * s.Hin : s.Hin, Wu = UP ? 2 * s.Win : s.Win;
    const int Ho = Hu / STRIDE, Wo = Wu / STRIDE;
    const int tiles_x = (Wo + TS - 1) / TS;
    const int oy0 = (blockIdx.x / tiles_x) * TS, ox0 = (blockIdx.x % tiles_x) * TS;
    const int co0 = blockIdx.y * COT, n = blockIdx.z;
    const int tx = threadIdx.x % TS, ty = threadIdx.x / TS;
    float acc[COT];
#pragma unroll
    for (int co = 0; co < COT; ++co) acc[co] = bias ? bias[co0 + co] : 0.0f;
    const int iy0 = oy0 * STRIDE - 1, ix0 = ox0 * STRIDE - 1;
    for (int c0 = 0; c0 < s.Ci; c0 += CIT) {
        const int nc = min(CIT, s.Ci - c0);
        for (int i = threadIdx.x; i < nc * IT * IT; i += blockDim.x) {
            const int c = i / (IT * IT), r = (i / IT) % IT, q = i % IT;
            const int iy = iy0 + r, ix = ix0 + q;
            float val = 0.0f;
            if (iy >= 0 && iy < Hu && ix >= 0 && ix < Wu) {
                const int ly = UP ? (iy >> 1) : iy, lx = UP ? (ix >> 1) : ix;
                val = x[(((size_t)n * s.Ci + c0 + c) * s.Hin + ly) * s.Win + lx];
            }
            sx[c][r][q] = val;
        }
        for (int i = threadIdx.x; i < nc * 9 * COT; i += blockDim.x) {
            const int co = i % COT, t = (i / COT) % 9, c = i / (9 * COT);
            sw[c][t][co] = __bfloat162float(w[((size_t)(co0 + co) * s.Ci + c0 + c) * 9 + t]);
        }
        __syncthreads();
        for (int c = 0; c < nc; ++c) {
#pragma unroll
            for (int u = 0; u < 3; ++u)
#pragma unroll
                for (int v = 0; v < 3; ++v) {
                    const float xv = sx[c][ty * STRIDE + u][tx * STRIDE + v];
#pragma unroll
                    for (int co = 0; co < COT; ++co) acc[co] = fmaf(sw[c][u * 3 + v][co], xv, acc[co]);
                }
        }
        __syncthreads();
    }
    const int oy = oy0 + ty, ox = ox0 + tx;
    if (oy < Ho && ox < Wo) {
#pragma unroll
        for (int co = 0; co < COT; ++co) {
            const float r = s.relu ? fmaxf(acc[co], 0.0f) : acc[co];
            y[(((size_t)n * s.Co + co0 + co) * Ho + oy) * Wo + ox] = r;
        }
    }
}

// dx of a stride-2 layer: dx[c][y][x] = sum_{o,u,v} w[o][c][u][v] dy[o][(y+1-u)/2][(x+1-v)/2]
// over the taps where y+1-u and x+1-v are even and in range.
template <int CT>
__global__ void __launch_bounds__(256) k_conv_bwd_data_s2(ConvShape s, const float* __restrict__ dy,
                                                          const __nv_bfloat16* __restrict__ w, float* __restrict__ dx) {
    constexpr int GT = TS / 2 + 2;   // dy rows / columns a 16 x 16 input tile needs
    __shared__ float sg[CIT][GT][GT + 1];
    __shared__ float sw[CIT][9][CT];
    const int Ho = s.Hin / 2, Wo = s.Win / 2;
    const int tiles_x = (s.Win + TS - 1) / TS;
    const int y0 = (blockIdx.x / tiles_x) * TS, x0 = (blockIdx.x % tiles_x) * TS;
    const int c0 = blockIdx.y * CT, n = blockIdx.z;
    const int tx = threadIdx.x % TS, ty = threadIdx.x / TS;
    const int gy0 = y0 / 2 - 1, gx0 = x0 / 2 - 1;
    float acc[CT];
#pragma unroll
    for (int c = 0; c < CT; ++c) acc[c] = 0.0f;
    const int yy = y0 + ty, xx = x0 + tx;
    for (int o0 = 0; o0 < s.Co; o0 += CIT) {
        const int no = min(CIT, s.Co - o0);
        for (int i = threadIdx.x; i < no * GT * GT; i += blockDim.x) {
            const int o = i / (GT * GT), r = (i / GT) % GT, q = i % GT;
            const int gy = gy0 + r, gx = gx0 + q;
            sg[o][r][q] = (gy >= 0 && gy < Ho && gx >= 0 && gx < Wo)
                              ? dy[(((size_t)n * s.Co + o0 + o) * Ho + gy) * Wo + gx] : 0.0f;
        }
        for (int i = threadIdx.x; i < no * 9 * CT; i += blockDim.x) {
            const int c = i % CT, t = (i / CT) % 9, o = i / (9 * CT);
            sw[o][t][c] = __bfloat162float(w[((size_t)(o0 + o) * s.Ci + c0 + c) * 9 + t]);
        }
        __syncthreads();
        for (int o = 0; o < no; ++o) {
#pragma unroll
            for (int u = 0; u < 3; ++u) {
                const int ny2 = yy + 1 - u;
                if (ny2 & 1) continue;
                const int r = ny2 / 2 - gy0;
#pragma unroll
                for (int v = 0; v < 3; ++v) {
                    const int nx2 = xx + 1 - v;
                    if (nx2 & 1) continue;
                    const float g = sg[o][r][nx2 / 2 - gx0];
#pragma unroll
                    for (int c = 0; c < CT; ++c) acc[c] = fmaf(sw[o][u * 3 + v][c], g, acc[c]);
                }
            }
        }
        __syncthreads();
    }
    if (yy < s.Hin && xx < s.Win) {
#pragma unroll
        for (int c = 0; c < CT; ++c) dx[(((size_t)n * s.Ci + c0 + c) * s.Hin + yy) * s.Win + xx] = acc[c];
    }
}

// dx[n][c][y][x] = sum of the 2 x 2 block of the high-resolution gradient
__global__ void k_pool2_sum(const float* __restrict__ hi, float* __restrict__ lo, long n_lo, int H, int W) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n_lo; i += (long)gridDim.x * blockDim.x) {
        const int x = i % W, y = (i / W) % H;
        const long plane = i / ((long)H * W);
        const float* h = hi + plane * 4L * H * W;
        const int W2 = 2 * W;
        lo[i] = h[(2 * y) * W2 + 2 * x] + h[(2 * y) * W2 + 2 * x + 1] + h[(2 * y + 1) * W2 + 2 * x] +
                h[(2 * y + 1) * W2 + 2 * x + 1];
    }
}

template <int STRIDE, bool UP>
__global__ void __launch_bounds__(256) k_conv_wgrad(ConvShape s, const float* __restrict__ x,
                                                    const float* __restrict__ dy, float* __restrict__ dw) {
    const int o = blockIdx.x / s.Ci, c = blockIdx.x % s.Ci;
    const int Hu = UP ? 2 * s.Hin : s.Hin, Wu = UP ? 2 * s.Win : s.Win;
    const int Ho = Hu / STRIDE, Wo = Wu / STRIDE;
    float acc[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) acc[t] = 0.0f;
    const long plane = (long)Ho * Wo, total = (long)s.N * plane;
    for (long e = blockIdx.y * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.y * blockDim.x) {
        const int n = (int)(e / plane);
        const int i = (int)((e % plane) / Wo), j = (int)(e % Wo);
        const float g = dy[((size_t)n * s.Co + o) * plane + (size_t)i * Wo + j];
        const float* xc = x + ((size_t)n * s.Ci + c) * s.Hin * s.Win;
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            const int iy = i * STRIDE + u - 1;
            if (iy < 0 || iy >= Hu) continue;
            const int ly = UP ? (iy >> 1) : iy;
#pragma unroll
            for (int v = 0; v < 3; ++v) {
                const int ix = j * STRIDE + v - 1;
                if (ix < 0 || ix >= Wu) continue;
                acc[u * 3 + v] = fmaf(g, xc[ly * s.Win + (UP ? (ix >> 1) : ix)], acc[u * 3 + v]);
            }
        }
    }
    __shared__ float red[9][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int t = 0; t < 9; ++t) {
        float vsum = acc[t];
        for (int off = 16; off > 0; off >>= 1) vsum += __shfl_xor_sync(0xffffffffu, vsum, off);
        if (lane == 0) red[t][warp] = vsum;
    }
    __syncthreads();
    if (threadIdx.x < 9) {
        float tsum = 0.0f;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) tsum += red[threadIdx.x][q];
        atomicAdd(dw + ((size_t)o * s.Ci + c) * 9 + threadIdx.x, tsum);
    }
}

__global__ void __launch_bounds__(256) k_bias_grad(const float* __restrict__ dy, int N, int Co, long plane,
                                                   float* __restrict__ db) {
    const int o = blockIdx.x;
    float acc = 0.0f;
    for (long e = threadIdx.x; e < (long)N * plane; e += blockDim.x) {
        const long n = e / plane, p = e % plane;
        acc += dy[((size_t)n * Co + o) * plane + p];
    }
    __shared__ float red[8];
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
        db[o] = t;
    }
}

__global__ void k_to_bf16(const float* __restrict__ w32, __nv_bfloat16* __restrict__ w16, __nv_bfloat16* __restrict__ wt,
                          int Co, int Ci) {
    const int n = Co * Ci * 9;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const __nv_bfloat16 h = __float2bfloat16_rn(w32[i]);
        w16[i] = h;
        const int t = i % 9, c = (i / 9) % Ci, o = i / (9 * Ci);
        if (wt) wt[((size_t)c * Co + o) * 9 + (8 - t)] = h;
    }
}

__global__ void k_relu_bwd(float* __restrict__ g, const float* __restrict__ a, long n) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        if (!(a[i] > 0.0f)) g[i] = 0.0f;
}

__global__ void __launch_bounds__(256) k_mse(const float* __restrict__ out, const float* __restrict__ t,
                                             const float* __restrict__ mask, long n, int HW, float inv_terms,
                                             float* __restrict__ g, double* loss) {
    double acc = 0.0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float d = (out[i] - t[i]) * mask[i % HW];
        g[i] = 2.0f * d * inv_terms;
        acc += (double)d * d;
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    __shared__ double red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q];
        atomicAdd(loss, s * inv_terms);
    }
}

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
    const int smem = (int)(sizeof(float2) * (G7::S + G7::M));
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_probe_phasor, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_learn_pairs, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_physics_inputs, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess) return e;
    team_smem_ready = true;
    return cudaSuccess;
}
size_t team_smem() { return sizeof(float2) * (G7::S + G7::M); }

template <int COT>
cudaError_t conv_fwd_dispatch(const ConvShape& s, const float* x, const __nv_bfloat16* w, const float* b, float* y,
                              cudaStream_t st) {
    const int Ho = s.Ho(), Wo = s.Wo();
    const dim3 grid(((Ho + TS - 1) / TS) * ((Wo + TS - 1) / TS), s.Co / COT, s.N);
    if (s.stride == 2 && !s.up) k_conv_fwd<COT, 2, false><<<grid, 256, 0, st>>>(s, x, w, b, y);
    else if (s.stride == 1 && s.up) k_conv_fwd<COT, 1, true><<<grid, 256, 0, st>>>(s, x, w, b, y);
    else if (s.stride == 1 && !s.up) k_conv_fwd<COT, 1, false><<<grid, 256, 0, st>>>(s, x, w, b, y);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace

cudaError_t conv_forward(const ConvShape& s, const float* x, const __nv_bfloat16* w, const float* bias, float* y,
                         cudaStream_t st) {
    if (s.Co % 16 == 0) return conv_fwd_dispatch<16>(s, x, w, bias, y, st);
    if (s.Co % 2 == 0) return conv_fwd_dispatch<2>(s, x, w, bias, y, st);
    return cudaErrorInvalidValue;
}

cudaError_t conv_backward_data(const ConvShape& s, const float* dy, const __nv_bfloat16* w, const __nv_bfloat16* wt,
                               float* dx, float* scratch, cudaStream_t st) {
    if (s.stride == 2 && !s.up) {
        if (s.Ci % 16) return cudaErrorInvalidValue;
        const dim3 grid(((s.Hin + TS - 1) / TS) * ((s.Win + TS - 1) / TS), s.Ci / 16, s.N);
        k_conv_bwd_data_s2<16><<<grid, 256, 0, st>>>(s, dy, w, dx);
        return cudaGetLastError();
    }
    if (s.stride == 1 && s.up) {
        // gradient w.r.t. the upsampled input: a stride-1 correlation of dy with wt
        ConvShape t{s.N, s.Co, s.Ci, s.Ho(), s.Wo(), 1, 0, 0};
        cudaError_t e = conv_forward(t, dy, wt, nullptr, scratch, st);
        if (e != cudaSuccess) return e;
        const long n_lo = (long)s.N * s.Ci * s.Hin * s.Win;
        k_pool2_sum<<<blocks_for(n_lo), 256, 0, st>>>(scratch, dx, n_lo, s.Hin, s.Win);
        return cudaGetLastError();
    }
    return cudaErrorInvalidValue;
}

cudaError_t conv_backward_weights(const ConvShape& s, const float* x, const float* dy, float* dw, float* db, int num_sms,
                                  cudaStream_t st) {
    const long work = (long)s.N * s.Ho() * s.Wo();
    const int pairs = s.Co * s.Ci;
    const int split = (int)std::max<long>(1, std::min<long>((4L * num_sms + pairs - 1) / pairs, (work + 255) / 256));
    const dim3 grid(pairs, split);
    if (s.stride == 2 && !s.up) k_conv_wgrad<2, false><<<grid, 256, 0, st>>>(s, x, dy, dw);
    else if (s.stride == 1 && s.up) k_conv_wgrad<1, true><<<grid, 256, 0, st>>>(s, x, dy, dw);
    else if (s.stride == 1 && !s.up) k_conv_wgrad<1, false><<<grid, 256, 0, st>>>(s, x, dy, dw);
    else return cudaErrorInvalidValue;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_bias_grad<<<s.Co, 256, 0, st>>>(dy, s.N, s.Co, (long)s.Ho() * s.Wo(), db);
    return cudaGetLastError();
}

cudaError_t weights_to_bf16(const ConvShape& s, const float* w32, __nv_bfloat16* w16, __nv_bfloat16* wt, cudaStream_t st) {
    k_to_bf16<<<blocks_for((long)s.Co * s.Ci * 9), 256, 0, st>>>(w32, w16, wt, s.Co, s.Ci);
    return cudaGetLastError();
}

cudaError_t relu_backward(float* g, const float* a, long n, cudaStream_t st) {
    k_relu_bwd<<<blocks_for(n), 256, 0, st>>>(g, a, n);
    return cudaGetLastError();
}

cudaError_t mse_loss(const float* out, const float* t, const float* mask, int N, int HW, double n_terms, float* g,
                     double* loss, cudaStream_t st) {
    const long n = (long)N * 2 * HW;
    k_mse<<<blocks_for(n), 256, 0, st>>>(out, t, mask, n, HW, (float)(1.0 / n_terms), g, loss);
    return cudaGetLastError();
}

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
