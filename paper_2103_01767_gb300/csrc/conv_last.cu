// conv_last.cu -- the decoder's last layer (x2 nearest upsampling, then a 3x3 convolution to
// Co <= 2 output channels) on the CUDA cores: forward, input gradient, weight gradient.
//
// On the tensor cores this layer is the slowest of the network: its N = 16 MMAs carry 2 useful
// columns, and each 8 x 16 tile of its 128 x 128 output runs a whole pipeline for four
// 16-channel K steps.  Here each thread owns one pixel (a, b) of the low-resolution input
// and the 2 x 2 block of output pixels (2a + py, 2b + px) it feeds.  With nearest
// upsampling, output phase (py, px) sees source rows a + py - 1 + jy (jy = 0, 1) and
// columns b + px - 1 + jx: a 2 x 2 kernel whose weights are sums of the 3 x 3 taps
//   Weff[py][px][jy][jx][o][c] = sum over taps (u, v) with floor((py + u - 1) / 2) = py - 1 + jy
//                                and floor((px + v - 1) / 2) = px - 1 + jx of w[o][c][u][v],
// formed in shared memory from the same bfloat16 weight copy (wf) the tensor-core layers use.
// Activations are the (hi, lo) pairs of the other layers, added in FP32.
#include "conv_tc.h"

#include "tc_common.cuh"

namespace ptylm {

namespace {

using namespace tc;

constexpr int kMaxCo = 2;
constexpr int kMaxCi = 256;
constexpr int kThreads = 256;

// floor((p + u - 1) / 2) - (p - 1): which of the two source rows (0, 1) tap u of phase p reads
__device__ __forceinline__ int tap_src(int p, int u) { return ((p + u + 1) >> 1) - p; }

// weff[((c * 4 + ph) * 4 + 2 * jy + jx) * kMaxCo + o]; wf[t][c/8][Co][c%8] (bfloat16)
__device__ void build_weff(const __nv_bfloat16* __restrict__ wf, int Co, int Ci, int Ci_pad, float* weff) {
    for (int i = threadIdx.x; i < Ci * 16 * kMaxCo; i += blockDim.x) {
        const int o = i % kMaxCo, j = (i / kMaxCo) % 4, ph = (i / kMaxCo / 4) % 4, c = i / kMaxCo / 16;
        const int py = ph >> 1, px = ph & 1, jy = j >> 1, jx = j & 1;
        float s = 0.0f;
        if (o < Co)
            for (int u = 0; u < 3; ++u)
                for (int v = 0; v < 3; ++v)
                    if (tap_src(py, u) == jy && tap_src(px, v) == jx)
                        s += __bfloat162float(wf[(((size_t)(3 * u + v) * (Ci_pad >> 3) + (c >> 3)) * Co + o) * 8 + (c & 7)]);
        weff[i] = s;
    }
}

// y32[n][o][2a + py][2b + px] = bias[o] + sum Weff x, one thread per input pixel (n, a, b)
__global__ void __launch_bounds__(kThreads) k_last_forward(const __nv_bfloat16* __restrict__ xhi,
                                                          const __nv_bfloat16* __restrict__ xlo, int N, int H, int W,
                                                          int Ci, int Ci_pad, int Co, const __nv_bfloat16* __restrict__ wf,
                                                          const float* __restrict__ bias, float* __restrict__ y32) {
    __shared__ __align__(16) float weff[kMaxCi * 16 * kMaxCo];
    build_weff(wf, Co, Ci, Ci_pad, weff);
    __syncthreads();
    const long p = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (long)N * H * W) return;
    const int n = (int)(p / ((long)H * W)), a = (int)((p / W) % H), b = (int)(p % W);
    const int C8 = Ci >> 3;
    float acc[4][kMaxCo];
#pragma unroll
    for (int ph = 0; ph < 4; ++ph)
#pragma unroll
        for (int o = 0; o < kMaxCo; ++o) acc[ph][o] = o < Co ? bias[o] : 0.0f;
    for (int q = 0; q < C8; ++q) {
        float xv[3][3][8];   // source rows a - 1 .. a + 1, columns b - 1 .. b + 1, 8 channels
#pragma unroll
        for (int dy = 0; dy < 3; ++dy)
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
                const int y = a + dy - 1, x = b + dx - 1;
                if (y >= 0 && y < H && x >= 0 && x < W) {
                    load_pair8(xhi, xlo, chunk_at(0, C8, H, W, n, y, x, q), xv[dy][dx]);
                } else {
#pragma unroll
                    for (int j = 0; j < 8; ++j) xv[dy][dx][j] = 0.0f;
                }
            }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float4* wc = reinterpret_cast<const float4*>(weff + (size_t)(8 * q + j) * 16 * kMaxCo);
#pragma unroll
            for (int ph = 0; ph < 4; ++ph) {
                const int py = ph >> 1, px = ph & 1;
                const float4 w01 = wc[2 * ph], w23 = wc[2 * ph + 1];   // (jy, jx) = 00, 01, 10, 11 x (o0, o1)
                const float s00 = xv[py][px][j], s01 = xv[py][px + 1][j];
                const float s10 = xv[py + 1][px][j], s11 = xv[py + 1][px + 1][j];
                acc[ph][0] = fmaf(w01.x, s00, fmaf(w01.z, s01, fmaf(w23.x, s10, fmaf(w23.z, s11, acc[ph][0]))));
                acc[ph][1] = fmaf(w01.y, s00, fmaf(w01.w, s01, fmaf(w23.y, s10, fmaf(w23.w, s11, acc[ph][1]))));
            }
        }
    }
    const int Ho = 2 * H, Wo = 2 * W;
    for (int o = 0; o < Co; ++o)
#pragma unroll
        for (int py = 0; py < 2; ++py)
            *reinterpret_cast<float2*>(y32 + (((size_t)n * Co + o) * Ho + 2 * a + py) * Wo + 2 * b) =
                make_float2(acc[2 * py][o], acc[2 * py + 1][o]);
}

// dx = (d conv / d x)^T dy, masked by act > 0, written as the pair dx (and its parity copy);
// db_part[block][c] = sum over the block's pixels of dx.  One thread per input pixel.
__global__ void __launch_bounds__(kThreads) k_last_backward_data(
    const __nv_bfloat16* __restrict__ ghi, const __nv_bfloat16* __restrict__ glo, int N, int H, int W, int Ci, int Ci_pad,
    int Co, const __nv_bfloat16* __restrict__ wf, const __nv_bfloat16* __restrict__ ahi,
    const __nv_bfloat16* __restrict__ alo, __nv_bfloat16* __restrict__ dhi, __nv_bfloat16* __restrict__ dlo,
    __nv_bfloat16* __restrict__ dphi, __nv_bfloat16* __restrict__ dplo, float* __restrict__ db_part) {
    __shared__ __align__(16) float weff[kMaxCi * 16 * kMaxCo];
    __shared__ float dbs[kThreads / 32][kMaxCi];
    build_weff(wf, Co, Ci, Ci_pad, weff);
    __syncthreads();
    const long p = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = p < (long)N * H * W;
    const int n = valid ? (int)(p / ((long)H * W)) : 0, a = (int)((p / W) % H), b = (int)(p % W);
    const int Ho = 2 * H, Wo = 2 * W, C8 = Ci >> 3;
    // dy at the output pixels this input feeds: rows 2a - 1 .. 2a + 2, columns 2b - 1 .. 2b + 2
    // (output row 2a' + py with a' = a + 1 - py - jy)
    float g[4][4][kMaxCo];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int Y = 2 * a - 1 + r, X = 2 * b - 1 + s;
            float v[8];
            if (valid && Y >= 0 && Y < Ho && X >= 0 && X < Wo) {
                load_pair8(ghi, glo, chunk_at(0, 1, Ho, Wo, n, Y, X, 0), v);
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = 0.0f;
            }
#pragma unroll
            for (int o = 0; o < kMaxCo; ++o) g[r][s][o] = o < Co ? v[o] : 0.0f;
        }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int q = 0; q < C8; ++q) {
        float d[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float4* wc = reinterpret_cast<const float4*>(weff + (size_t)(8 * q + j) * 16 * kMaxCo);
            float s = 0.0f;
#pragma unroll
            for (int ph = 0; ph < 4; ++ph) {
                const int py = ph >> 1, px = ph & 1;
                const float4 w01 = wc[2 * ph], w23 = wc[2 * ph + 1];
                // (jy, jx) feeds output (2a' + py, 2b' + px) with a' = a + 1 - py - jy: row index
                // r = 2a' + py - (2a - 1) = 3 - py - 2 jy
                const int r0 = 3 - py, r1 = 1 - py, c0 = 3 - px, c1 = 1 - px;
                s = fmaf(w01.x, g[r0][c0][0], fmaf(w01.y, g[r0][c0][1], s));
                s = fmaf(w01.z, g[r0][c1][0], fmaf(w01.w, g[r0][c1][1], s));
                s = fmaf(w23.x, g[r1][c0][0], fmaf(w23.y, g[r1][c0][1], s));
                s = fmaf(w23.z, g[r1][c1][0], fmaf(w23.w, g[r1][c1][1], s));
            }
            d[j] = s;
        }
        if (valid) {
            float av[8];
            load_pair8(ahi, alo, chunk_at(0, C8, H, W, n, a, b, q), av);
#pragma unroll
            for (int j = 0; j < 8; ++j) d[j] = av[j] > 0.0f ? d[j] : 0.0f;
            store_pair8(dhi, dlo, chunk_at(0, C8, H, W, n, a, b, q), d);
            if (dphi) store_pair8(dphi, dplo, chunk_at(1, C8, H, W, n, a, b, q), d);
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) d[j] = 0.0f;
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float t = d[j];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
            if (lane == 0) dbs[warp][8 * q + j] = t;
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < Ci; c += blockDim.x) {
        float t = 0.0f;
        for (int w = 0; w < kThreads / 32; ++w) t += dbs[w][c];
        db_part[(size_t)blockIdx.x * Ci + c] = t;
    }
}

// Partial weight gradients ws[block][(o * Ci + c) * 9 + t] over the input rows
// [row0, row0 + rows) of image n: thread (c, group) with c < Ci runs along the rows
// row0 + group, row0 + group + groups, ..., keeping its 3 x 3 input window in registers.
constexpr int kWgRows = 16;
__global__ void __launch_bounds__(kThreads) k_last_wgrad(const __nv_bfloat16* __restrict__ xhi,
                                                        const __nv_bfloat16* __restrict__ xlo,
                                                        const __nv_bfloat16* __restrict__ ghi,
                                                        const __nv_bfloat16* __restrict__ glo, int H, int W, int Ci,
                                                        int Co, float* __restrict__ ws) {
    const int groups = kThreads / Ci;   // Ci divides kThreads
    const int c = threadIdx.x % Ci, grp = threadIdx.x / Ci;
    const int n = blockIdx.x / (H / kWgRows), row0 = (blockIdx.x % (H / kWgRows)) * kWgRows;
    const int Ho = 2 * H, Wo = 2 * W, C8 = Ci >> 3;
    extern __shared__ float sm[];        // [groups][2 output rows][Wo][kMaxCo] dy, then reduction space
    float acc[kMaxCo][9];
#pragma unroll
    for (int o = 0; o < kMaxCo; ++o)
#pragma unroll
        for (int t = 0; t < 9; ++t) acc[o][t] = 0.0f;
    float* gs = sm + (size_t)grp * 2 * Wo * kMaxCo;
    const __nv_bfloat16* xh = xhi + chunk_at(0, C8, H, W, n, 0, 0, c >> 3) + (c & 7);
    const __nv_bfloat16* xl = xlo + chunk_at(0, C8, H, W, n, 0, 0, c >> 3) + (c & 7);
    auto xat = [&](int y, int x) -> float {
        if (y < 0 || y >= H || x < 0 || x >= W) return 0.0f;
        const size_t o = ((size_t)y * W + x) * 8;
        return __bfloat162float(xh[o]) + __bfloat162float(xl[o]);
    };
    for (int it = 0; it < kWgRows / groups; ++it) {
        const int a = row0 + grp + groups * it;
        __syncthreads();   // the previous row's dy is no longer read
        // dy of output rows 2a, 2a + 1 into this group's slice: gs[(py * Wo + X) * kMaxCo + o]
        for (int i = c; i < 2 * Wo; i += Ci) {
            const int py = i / Wo, X = i % Wo;
            float v[8];
            load_pair8(ghi, glo, chunk_at(0, 1, Ho, Wo, n, 2 * a + py, X, 0), v);
#pragma unroll
            for (int o = 0; o < kMaxCo; ++o) gs[(py * Wo + X) * kMaxCo + o] = o < Co ? v[o] : 0.0f;
        }
        __syncthreads();
        // window of input rows a - 1 .. a + 1 and columns b - 1 .. b + 1, slid along b
        float win[3][3];
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
            win[dy][1] = xat(a + dy - 1, -1);
            win[dy][2] = xat(a + dy - 1, 0);
        }
        for (int b = 0; b < W; ++b) {
#pragma unroll
            for (int dy = 0; dy < 3; ++dy) {
                win[dy][0] = win[dy][1];
                win[dy][1] = win[dy][2];
                win[dy][2] = xat(a + dy - 1, b + 1);
            }
#pragma unroll
            for (int py = 0; py < 2; ++py)
#pragma unroll
                for (int px = 0; px < 2; ++px) {
                    const float2 gv = *reinterpret_cast<const float2*>(gs + (py * Wo + 2 * b + px) * kMaxCo);
#pragma unroll
                    for (int u = 0; u < 3; ++u)
#pragma unroll
                        for (int v = 0; v < 3; ++v) {
                            const float xs = win[py + tap_src(py, u)][px + tap_src(px, v)];
                            acc[0][3 * u + v] = fmaf(gv.x, xs, acc[0][3 * u + v]);
                            acc[1][3 * u + v] = fmaf(gv.y, xs, acc[1][3 * u + v]);
                        }
                }
        }
    }
    // sum the groups in a fixed order
    __syncthreads();
    float* red = sm;   // [groups][Ci][kMaxCo * 9]
#pragma unroll
    for (int o = 0; o < kMaxCo; ++o)
#pragma unroll
        for (int t = 0; t < 9; ++t) red[((size_t)grp * Ci + c) * kMaxCo * 9 + o * 9 + t] = acc[o][t];
    __syncthreads();
    for (int i = threadIdx.x; i < Ci * Co * 9; i += blockDim.x) {
        const int cc = (i / 9) % Ci, o = i / 9 / Ci, t = i % 9;
        float s = 0.0f;
        for (int q = 0; q < groups; ++q) s += red[((size_t)q * Ci + cc) * kMaxCo * 9 + o * 9 + t];
        ws[(size_t)blockIdx.x * Co * Ci * 9 + i] = s;   // i = (o * Ci + c) * 9 + t
    }
}

// dw[i] = sum over blocks q of ws[q][i]: warp w of a block sums the rows q = w (mod 8) for
// 32 consecutive i (coalesced), then the eight warp sums are added in warp order
__global__ void __launch_bounds__(256) k_last_wgrad_sum(const float* __restrict__ ws, int blocks, int count,
                                                        float* __restrict__ dw) {
    __shared__ float part[8][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int i = blockIdx.x * 32 + lane;
    float s = 0.0f;
    if (i < count)
        for (int q = w; q < blocks; q += 8) s += ws[(size_t)q * count + i];
    part[w][lane] = s;
    __syncthreads();
    if (w == 0 && i < count) {
        float t = 0.0f;
        for (int k = 0; k < 8; ++k) t += part[k][lane];
        dw[i] = t;
    }
}

bool last_layer_shape_ok(const TcLayer& L, int H) {
    return L.up && L.Co >= 1 && L.Co <= kMaxCo && L.Ci % 8 == 0 && L.Ci <= kMaxCi && kThreads % L.Ci == 0 &&
           H % kWgRows == 0 && (kWgRows % (kThreads / L.Ci)) == 0;
}

size_t wgrad_smem(const TcLayer& L, int W) {
    const int groups = kThreads / L.Ci;
    const size_t dy = (size_t)groups * 2 * (2 * W) * kMaxCo, red = (size_t)groups * L.Ci * kMaxCo * 9;
    return sizeof(float) * (dy > red ? dy : red);
}

}  // namespace

bool tc_last_supported(const TcLayer& L) { return last_layer_shape_ok(L, L.Hin); }

cudaError_t tc_last_forward(const TcLayer& L, const Act2& x, const __nv_bfloat16* wf, const float* bias, float* y32,
                            cudaStream_t st) {
    if (!last_layer_shape_ok(L, x.H) || x.par || x.C != L.Ci || x.H != L.Hin || x.W != L.Hin) return cudaErrorInvalidValue;
    const long total = (long)x.N * x.H * x.W;
    if (total == 0) return cudaSuccess;
    k_last_forward<<<(unsigned)((total + kThreads - 1) / kThreads), kThreads, 0, st>>>(x.hi, x.lo, x.N, x.H, x.W, L.Ci,
                                                                                      L.Ci_pad, L.Co, wf, bias, y32);
    return cudaGetLastError();
}

int tc_last_bias_parts(const TcLayer& L, int N) { return (int)(((long)N * L.Hin * L.Hin + kThreads - 1) / kThreads); }

cudaError_t tc_last_backward_data(const TcLayer& L, const Act2& dy, const __nv_bfloat16* wf, const Act2& act,
                                  const Act2& dx, float* db_part, int* n_part, cudaStream_t st) {
    if (!last_layer_shape_ok(L, act.H) || act.par || dx.par || dy.par || dy.C != 8 || act.C != L.Ci || dx.C != L.Ci ||
        dy.H != 2 * act.H)
        return cudaErrorInvalidValue;
    const long total = (long)act.N * act.H * act.W;
    const int blocks = (int)((total + kThreads - 1) / kThreads);
    *n_part = blocks;
    if (total == 0) return cudaSuccess;
    k_last_backward_data<<<blocks, kThreads, 0, st>>>(dy.hi, dy.lo, act.N, act.H, act.W, L.Ci, L.Ci_pad, L.Co, wf,
                                                      act.hi, act.lo, dx.hi, dx.lo, dx.phi, dx.plo, db_part);
    return cudaGetLastError();
}

size_t tc_last_wgrad_workspace(const TcLayer& L, int N) { return (size_t)N * (L.Hin / kWgRows) * L.Co * L.Ci * 9; }

cudaError_t tc_last_wgrad(const TcLayer& L, const Act2& x, const Act2& dy, float* ws, float* dw, cudaStream_t st) {
    if (!last_layer_shape_ok(L, x.H) || x.par || dy.par || dy.C != 8 || x.C != L.Ci || dy.H != 2 * x.H)
        return cudaErrorInvalidValue;
    const int blocks = x.N * (x.H / kWgRows), count = L.Co * L.Ci * 9;
    if (blocks == 0) return cudaMemsetAsync(dw, 0, sizeof(float) * count, st);
    const size_t smem = wgrad_smem(L, x.W);
    if (smem > 48 * 1024) return cudaErrorInvalidValue;
    k_last_wgrad<<<blocks, kThreads, smem, st>>>(x.hi, x.lo, dy.hi, dy.lo, x.H, x.W, L.Ci, L.Co, ws);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_last_wgrad_sum<<<(count + 31) / 32, 256, 0, st>>>(ws, blocks, count, dw);
    return cudaGetLastError();
}

}  // namespace ptylm
