// conv_tc.cu -- tensor-core 3x3 convolutions of the learned initialisation (see conv_tc.h).
//
// Implicit GEMM.  A CTA owns a tile of 8 x 16 points of an output sub-lattice (the output
// grid itself, or one parity class of it), i.e. 128 GEMM rows = 128 TMEM lanes, and up to four
// such accumulators ("phases") of N columns each.  The K loop runs over input channels, 16 per
// pipeline stage.  Per stage a TMA producer thread loads
//   * a few "copies" of the input: boxes of (8 channels) x (16 columns) x (rows) from the map or
//     one of its parity planes, each with its own column shift (every box row is 256
//     contiguous bytes of the chunk-major layout); a tap's
//     operand is a copy started `row` rows down (the canonical no-swizzle K-major layout makes
//     a row shift a plain descriptor offset, so one copy serves the three taps of a column);
//     out-of-range coordinates fill zeros, which is the convolution's zero padding;
//   * the bfloat16 weights of all nine taps for those 16 channels (18 contiguous bulk copies);
// and one MMA thread issues, per (phase, tap) group and per split (hi, lo), a 128 x N x 16
// tcgen05.mma into the phase's accumulator.  Mbarrier rings (full / empty) pipeline the stages.
//
// Layer forms (s: stride-2 layer, u: upsampling layer):
//   forward s:  output (a, b) reads input (2a+u-1, 2b+v-1): six copies from the four parity
//               views of the input (column shift 0 or -1);
//   forward u:  four phases (py, px) of the output (2a+py, 2b+px) read the low-resolution
//               input at (a + floor((py+u-1)/2), b + floor((px+v-1)/2)): three copies;
//   input gradient s: four phases (qy, qx) of the input grid, (2a'+qy, 2b'+qx), collect dy at
//               (a' + e, b' + f), e, f in {0, 1}, from the taps with matching parity;
//   input gradient u: a stride-1 correlation of dy at full resolution whose 2 x 2 sums (taken
//               with warp shuffles: a warp holds two full rows of the tile) give the gradient
//               of the low-resolution input.
// The weight gradient is a GEMM over pixels with MN-major operands (k_wgrad_tc).
#include "conv_tc.h"

#include <cuda.h>

#include <algorithm>
#include <cstring>

#include "tc_common.cuh"

namespace ptylm {

namespace {

using namespace tc;

constexpr int kThreads = 128;
constexpr int kMaxStage = 8;
constexpr int kMaxCopy = 8;
constexpr int kMaxGroup = 36;
constexpr int kSmemLimit = 232448;    // shared memory a CTA may use (static + dynamic)
constexpr int kOneCtaPerSm = 120 * 1024;  // dynamic request that leaves no room for a second CTA

enum { EPI_HIDDEN = 0, EPI_LAST = 1, EPI_BWD = 2, EPI_POOL = 3 };

struct Copy {
    int8_t row0, col;  // box start relative to the tile origin (sub-lattice units)
    int8_t par;        // parity plane of a parity-split map, -1 for a plain map
};
struct Group {
    uint8_t phase, copy, row, tap;
};

struct ConvArgs {
    int tiles_x, tiles_y;  // 8 x 16 tiles per image
    int n_copy, split, rows, ksteps, N, P, tmem_cols, n_stage;
    int a_slot;       // bytes of one (copy, chunk) box: rows * 256
    int a_bytes;      // A bytes of a stage: split * n_copy * 2 * a_slot
    int stage_bytes;  // a_bytes + 2 * 9 * N * 16
    int gstart[5];    // groups sorted by phase: phase p owns [gstart[p], gstart[p+1])
    unsigned cmask[4];  // copies used per phase group
    Copy copy[kMaxCopy];
    Group group[kMaxGroup];
    int mode, osy, osx;
    int8_t opy[4], opx[4];
    int oH, oW, oC;  // output tensor (chunk-major pair, or FP32 planes for the last layer)
    int out_par;     // layout of (out_hi, out_lo)
    __nv_bfloat16* out_hi;
    __nv_bfloat16* out_lo;
    __nv_bfloat16* out_phi;  // optional parity-split copy of the output
    __nv_bfloat16* out_plo;
    float* out32;
    const __nv_bfloat16* wts;  // weights [9][K/8][R][8]
    int wK8, wR;
    const float* bias;
    int relu;
    const __nv_bfloat16* m_hi;
    const __nv_bfloat16* m_lo;
    int m_par;
    float* db_part;
    unsigned* err;
    unsigned spin;
};

struct ConvParams {
    CUtensorMap amap[2];  // the input tensor: hi, lo
    ConvArgs a;
};

__device__ __forceinline__ unsigned char* align1024(unsigned char* p) {
    return reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// 16 channels from ch0 of pixel (y, x) into the output pair (and its parity copy)
__device__ __forceinline__ void store_out16(const ConvArgs& a, int n, int y, int x, int ch0, const float* v) {
    const int C8 = a.oC >> 3;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        store_pair8(a.out_hi, a.out_lo, chunk_at(a.out_par, C8, a.oH, a.oW, n, y, x, (ch0 >> 3) + q), v + 8 * q);
        if (a.out_phi) store_pair8(a.out_phi, a.out_plo, chunk_at(1, C8, a.oH, a.oW, n, y, x, (ch0 >> 3) + q), v + 8 * q);
    }
}

__global__ void __launch_bounds__(kThreads, 1) k_conv_tc(const __grid_constant__ ConvParams p) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = align1024(smem_raw);
    __shared__ uint64_t full[kMaxStage], empty[kMaxStage], done;
    __shared__ uint32_t tbase;
    __shared__ int abort_flag, issued, consumed;
    __shared__ float red[4][256];
    const ConvArgs& a = p.a;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int per_img = a.tiles_x * a.tiles_y;
    const int n = blockIdx.x / per_img, t = blockIdx.x % per_img;
    const int a0 = (t / a.tiles_x) * 8, b0 = (t % a.tiles_x) * 16;
    const int pg = blockIdx.y, o0 = blockIdx.z * a.N;
    const int S = a.n_stage;

    if (warp == 0) tmem_alloc(smem_u32(&tbase), a.tmem_cols);
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            bar_init(smem_u32(&full[s]), 1);
            bar_init(smem_u32(&empty[s]), 1);
        }
        bar_init(smem_u32(&done), 1);
        bar_fence_init();
        abort_flag = 0;
        issued = 0;
        consumed = 0;
    }
    for (int i = threadIdx.x; i < 4 * 256; i += kThreads) (&red[0][0])[i] = 0.0f;
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tbase;
    const uint32_t sbase = smem_u32(smem);
    const unsigned cmask = a.cmask[pg];

    if (warp == 0) {
        // TMA producer: lane 0 issues, the other lanes wait at the warp barrier
        if (lane == 0) {
            const int nb = min(a.N, a.wR - o0);   // weight rows present (the rest is never read into D)
            uint32_t bytes = 18u * (uint32_t)nb * 16u;
            for (int j = 0; j < a.n_copy; ++j)
                if (cmask >> j & 1) bytes += (uint32_t)(a.split * 2 * a.a_slot);
            int ks = 0;
            for (; ks < a.ksteps; ++ks) {
                const int s = ks % S, use = ks / S;
                if (use > 0 && !bar_wait(smem_u32(&empty[s]), (use - 1) & 1, a.spin)) {
                    atomicOr(a.err, 1u);
                    abort_flag = 1;
                    break;
                }
                if (*(volatile int*)&abort_flag) break;
                const uint32_t st = sbase + s * a.stage_bytes;
                const uint32_t fb = smem_u32(&full[s]);
                bar_expect_tx(fb, bytes);
                for (int sp = 0; sp < a.split; ++sp)
                    for (int j = 0; j < a.n_copy; ++j) {
                        if (!(cmask >> j & 1)) continue;
                        const uint32_t dst = st + (uint32_t)((sp * a.n_copy + j) * 2 * a.a_slot);
                        const Copy cp = a.copy[j];
                        const int x = (b0 + cp.col) * 8, y = a0 + cp.row0;
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
                            const int chunk = 2 * ks + q;
                            tma_load_4d(dst + q * a.a_slot, &p.amap[sp], x, y, cp.par < 0 ? chunk : 4 * chunk + cp.par, n, fb);
                        }
                    }
                const uint32_t bdst = st + a.a_bytes;
                for (int q = 0; q < 2; ++q)
                    for (int t = 0; t < 9; ++t) {
                        const __nv_bfloat16* src = a.wts + (((size_t)t * a.wK8 + 2 * ks + q) * a.wR + o0) * 8;
                        bulk_load(bdst + (uint32_t)((q * 9 + t) * a.N * 16), src, (uint32_t)nb * 16u, fb);
                    }
            }
            issued = ks;
        }
        __syncwarp();
    } else if (warp == 1) {
        // MMA issuer: lane 0 issues, the other lanes wait at the warp barrier
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(128, a.N, 0, 0);
            const int g0 = a.gstart[pg * a.P], g1 = a.gstart[pg * a.P + a.P];
            unsigned started = 0;
            int ks = 0;
            for (; ks < a.ksteps; ++ks) {
                const int s = ks % S, use = ks / S;
                if (!bar_wait(smem_u32(&full[s]), use & 1, a.spin)) {
                    atomicOr(a.err, 2u);
                    abort_flag = 1;
                    break;
                }
                fence_after();
                const uint32_t st = sbase + s * a.stage_bytes;
                const uint64_t bd0 = sdesc(st + a.a_bytes, 9u * a.N * 16u, 128u);
                for (int g = g0; g < g1; ++g) {
                    const Group gr = a.group[g];
                    const int ph = gr.phase - pg * a.P;
                    const uint64_t bd = bd0 + (uint64_t)((gr.tap * a.N * 16) >> 4);
                    const uint32_t d = tmem + (uint32_t)(ph * a.N);
                    for (int sp = 0; sp < a.split; ++sp) {
                        const uint32_t aaddr = st + (uint32_t)((sp * a.n_copy + gr.copy) * 2 * a.a_slot + gr.row * 256);
                        const uint64_t ad = sdesc(aaddr, (uint32_t)a.a_slot, 128u);
                        mma_bf16(d, ad, bd, idesc, (started >> ph) & 1u);
                        started |= 1u << ph;
                    }
                }
                mma_commit(smem_u32(&empty[s]));
            }
            consumed = ks;
            mma_commit(smem_u32(&done));
        }
        __syncwarp();
    }
    const bool ok = bar_wait(smem_u32(&done), 0, a.spin);
    if (!ok && lane == 0) atomicOr(a.err, 4u);
    fence_after();
    __syncthreads();
    const bool abort = *(volatile int*)&abort_flag || !ok;
    if (abort && threadIdx.x == 0) {
        // let the copies still in flight land before the CTA's shared memory is released
        for (int ks = consumed; ks < issued; ++ks) bar_wait(smem_u32(&full[ks % S]), (ks / S) & 1, a.spin);
    }

    if (!abort) {
        const int i = 32 * warp + lane;
        const int r = i >> 4, c = i & 15;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);
        for (int ph = 0; ph < a.P; ++ph) {
            const int phase = pg * a.P + ph;
            const int oy = a.osy * (a0 + r) + a.opy[phase], ox = a.osx * (b0 + c) + a.opx[phase];
            for (int cb = 0; cb < a.N; cb += 16) {
                float v[16];
                tmem_ld16(lane_base + (uint32_t)(ph * a.N + cb), v);
                const int ch0 = o0 + cb;
                if (a.mode == EPI_HIDDEN) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        v[j] += a.bias[ch0 + j];
                        if (a.relu) v[j] = fmaxf(v[j], 0.0f);
                    }
                    store_out16(a, n, oy, ox, ch0, v);
                } else if (a.mode == EPI_LAST) {
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (ch0 + j < a.oC)
                            a.out32[(((size_t)n * a.oC + ch0 + j) * a.oH + oy) * a.oW + ox] = v[j] + a.bias[ch0 + j];
                } else {
                    int py = oy, px = ox;
                    bool writer = true;
                    if (a.mode == EPI_POOL) {
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            v[j] += __shfl_xor_sync(0xffffffffu, v[j], 1);
                            v[j] += __shfl_xor_sync(0xffffffffu, v[j], 16);
                        }
                        writer = ((r | c) & 1) == 0;
                        py = (a0 + r) >> 1;
                        px = (b0 + c) >> 1;
                    }
                    if (writer) {
                        bool m[16];
#pragma unroll
                        for (int q = 0; q < 2; ++q)
                            load_mask8(a.m_hi, a.m_lo, chunk_at(a.m_par, a.oC >> 3, a.oH, a.oW, n, py, px, (ch0 >> 3) + q),
                                       m + 8 * q);
#pragma unroll
                        for (int j = 0; j < 16; ++j) v[j] = m[j] ? v[j] : 0.0f;
                        store_out16(a, n, py, px, ch0, v);
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j) v[j] = 0.0f;
                    }
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float sum = warp_sum(v[j]);
                        if (lane == 0) red[warp][cb + j] += sum;
                    }
                }
            }
        }
        if (a.mode >= EPI_BWD) {
            __syncthreads();
            const size_t part = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
            for (int ch = threadIdx.x; ch < a.N; ch += kThreads)
                a.db_part[part * a.oC + o0 + ch] = red[0][ch] + red[1][ch] + red[2][ch] + red[3][ch];
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, a.tmem_cols);
}

// ---------------------------------------------------------------------------------------
// Weight gradient: D_t[row][col] = sum over pixels p of A_t[row][p] B_t[col][p], one TMEM
// accumulator per tap t.  One operand is the output gradient dy at the forward pass's output
// pixels (shared by all taps), the other the tap-shifted input (copies as in the forward
// pass).  Both are stored pixel-major with channels contiguous, i.e. MN-major operands; K is
// the pixel index, 16 pixels (one row of the tile) per MMA.  A CTA runs over a strided
// subset of the pixel tiles and writes its partial sums; k_wgrad_reduce adds them in a fixed
// order.  Rows (or columns) beyond the real channel count read whatever lies next in shared
// memory and are discarded.

struct WgArgs {
    int tiles_x, tiles_y, phases, n_tiles, rows_px;
    int w2;           // 0: A = dy (rows = output channels), B = input copies; 1: swapped
    int g_real;       // dy chunk boxes per split
    int x_real;       // input chunk boxes per copy and split
    int n_copy, rows, N, c_tiles, Nc, tmem_cols, n_stage;
    int g_slot, x_slot, g_bytes, x_bytes, stage_bytes;
    int n_split;      // gridDim.x
    int g_parity;     // 1: dy is read from its parity copy, plane = phase
    Copy copy[6];
    uint8_t grp[4][9][2];  // phase, tap -> copy, row offset
    unsigned cmask[4];
    float* part;
    unsigned* err;
    unsigned spin;
};

struct WgParams {
    CUtensorMap gmap[2];  // dy (or its parity copy): hi, lo
    CUtensorMap xmap[2];  // the layer input: hi, lo
    WgArgs a;
};

__global__ void __launch_bounds__(kThreads, 1) k_wgrad_tc(const __grid_constant__ WgParams p) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = align1024(smem_raw);
    __shared__ uint64_t full[kMaxStage], empty[kMaxStage], done;
    __shared__ uint32_t tbase;
    __shared__ int abort_flag, issued, consumed;
    const WgArgs& a = p.a;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int split = blockIdx.x, kind = blockIdx.y;
    const int S = a.n_stage;
    int o0, c0;
    if (a.w2) {
        c0 = kind * 128;
        o0 = 0;
    } else {
        o0 = (kind / a.c_tiles) * 128;
        c0 = (kind % a.c_tiles) * a.Nc;
    }
    const int per_phase = a.tiles_x * a.tiles_y;

    if (warp == 0) tmem_alloc(smem_u32(&tbase), a.tmem_cols);
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            bar_init(smem_u32(&full[s]), 1);
            bar_init(smem_u32(&empty[s]), 1);
        }
        bar_init(smem_u32(&done), 1);
        bar_fence_init();
        abort_flag = 0;
        issued = 0;
        consumed = 0;
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tbase;
    const uint32_t sbase = smem_u32(smem);
    const int my_tiles = split < a.n_tiles ? (a.n_tiles - 1 - split) / a.n_split + 1 : 0;

    if (warp == 0) {
        // TMA producer: lane 0 issues, the other lanes wait at the warp barrier
        if (lane == 0) {
            int it = 0;
            for (; it < my_tiles; ++it) {
                const int tile = split + it * a.n_split;
                const int nimg = tile / (a.phases * per_phase), rem = tile % (a.phases * per_phase);
                const int ph = rem / per_phase, tt = rem % per_phase;
                const int a0 = (tt / a.tiles_x) * a.rows_px, b0 = (tt % a.tiles_x) * 16;
                const int s = it % S, use = it / S;
                if (use > 0 && !bar_wait(smem_u32(&empty[s]), (use - 1) & 1, a.spin)) {
                    atomicOr(a.err, 8u);
                    abort_flag = 1;
                    break;
                }
                if (*(volatile int*)&abort_flag) break;
                const unsigned cm = a.cmask[ph];
                uint32_t bytes = (uint32_t)(2 * a.g_real * a.g_slot);
                for (int j = 0; j < a.n_copy; ++j)
                    if (cm >> j & 1) bytes += (uint32_t)(2 * a.x_real * a.x_slot);
                const uint32_t st = sbase + s * a.stage_bytes;
                const uint32_t fb = smem_u32(&full[s]);
                bar_expect_tx(fb, bytes);
                for (int sp = 0; sp < 2; ++sp) {
                    for (int q = 0; q < a.g_real; ++q) {
                        const int chunk = (o0 >> 3) + q;
                        tma_load_4d(st + (uint32_t)((sp * a.g_real + q) * a.g_slot), &p.gmap[sp], b0 * 8, a0,
                                    a.g_parity ? 4 * chunk + ph : chunk, nimg, fb);
                    }
                    for (int j = 0; j < a.n_copy; ++j) {
                        if (!(cm >> j & 1)) continue;
                        const Copy cp = a.copy[j];
                        const uint32_t xb = st + (uint32_t)(a.g_bytes + ((sp * a.n_copy + j) * a.x_real) * a.x_slot);
                        for (int q = 0; q < a.x_real; ++q) {
                            const int chunk = (c0 >> 3) + q;
                            tma_load_4d(xb + (uint32_t)(q * a.x_slot), &p.xmap[sp], (b0 + cp.col) * 8, a0 + cp.row0,
                                        cp.par < 0 ? chunk : 4 * chunk + cp.par, nimg, fb);
                        }
                    }
                }
            }
            issued = it;
        }
        __syncwarp();
    } else if (warp == 1) {
        // MMA issuer: lane 0 issues, the other lanes wait at the warp barrier
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(128, a.N, 1, 1);
            int it = 0;
            for (; it < my_tiles; ++it) {
                const int tile = split + it * a.n_split;
                const int ph = (tile % (a.phases * per_phase)) / per_phase;
                const int s = it % S, use = it / S;
                if (!bar_wait(smem_u32(&full[s]), use & 1, a.spin)) {
                    atomicOr(a.err, 16u);
                    abort_flag = 1;
                    break;
                }
                fence_after();
                const uint32_t st = sbase + s * a.stage_bytes;
                for (int tap = 0; tap < 9; ++tap) {
                    const int cp = a.grp[ph][tap][0], ro = a.grp[ph][tap][1];
                    const uint32_t d = tmem + (uint32_t)(tap * a.N);
                    const uint32_t x0 = st + (uint32_t)(a.g_bytes + cp * a.x_real * a.x_slot + ro * 256);
                    const uint32_t xstride = (uint32_t)(a.n_copy * a.x_real * a.x_slot);  // split 0 -> 1
                    const uint32_t gstride = (uint32_t)(a.g_real * a.g_slot);
                    for (int k = 0; k < a.rows_px; ++k) {
    #pragma unroll
                        for (int combo = 0; combo < 3; ++combo) {
                            const int sg = combo == 2 ? 1 : 0, sx = combo == 1 ? 1 : 0;   // hi.hi, hi.lo, lo.hi
                            const uint64_t gd = sdesc(st + sg * gstride + k * 256, 128u, (uint32_t)a.g_slot);
                            const uint64_t xd = sdesc(x0 + sx * xstride + k * 256, 128u, (uint32_t)a.x_slot);
                            const uint32_t acc = (it > 0 || k > 0 || combo > 0) ? 1u : 0u;
                            if (a.w2) mma_bf16(d, xd, gd, idesc, acc);
                            else mma_bf16(d, gd, xd, idesc, acc);
                        }
                    }
                }
                mma_commit(smem_u32(&empty[s]));
            }
            consumed = it;
            mma_commit(smem_u32(&done));
        }
        __syncwarp();
    }
    const bool ok = bar_wait(smem_u32(&done), 0, a.spin);
    if (!ok && lane == 0) atomicOr(a.err, 32u);
    fence_after();
    __syncthreads();
    const bool abort = *(volatile int*)&abort_flag || !ok;
    if (abort && threadIdx.x == 0)
        for (int it = consumed; it < issued; ++it) bar_wait(smem_u32(&full[it % S]), (it / S) & 1, a.spin);
    if (!abort) {
        const int row = 32 * warp + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);
        const size_t blk = (size_t)kind * a.n_split + split;
        for (int tap = 0; tap < 9; ++tap)
            for (int cb = 0; cb < a.N; cb += 16) {
                float v[16];
                tmem_ld16(lane_base + (uint32_t)(tap * a.N + cb), v);
                if (my_tiles == 0)
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] = 0.0f;
                float4* dst = reinterpret_cast<float4*>(a.part + (((blk * 9 + tap) * 128 + row) * a.N + cb));
#pragma unroll
                for (int q = 0; q < 4; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            }
    }
    fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, a.tmem_cols);
}

// dw[o][c][t] = sum_s part[kind][s][t][row][col] in split order
__global__ void k_wgrad_reduce(const float* __restrict__ part, int Co, int Ci, int w2, int c_tiles, int Nc, int N,
                               int n_split, float* __restrict__ dw) {
    const int total = Co * Ci * 9;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int t = i % 9, c = (i / 9) % Ci, o = i / (9 * Ci);
        int kind, row, col;
        if (w2) {
            kind = c / 128;
            row = c % 128;
            col = o;
        } else {
            kind = (o / 128) * c_tiles + c / Nc;
            row = o % 128;
            col = c % Nc;
        }
        float s = 0.0f;
        for (int q = 0; q < n_split; ++q) s += part[((((size_t)kind * n_split + q) * 9 + t) * 128 + row) * N + col];
        dw[i] = s;
    }
}

// bias gradient: slice sums of the partial rows (32 channels x 8 rows of parts per block),
// then the slices in order; both steps in a fixed order
__global__ void __launch_bounds__(256) k_bias_slices(const float* __restrict__ part, int n_part, int C, int per_slice,
                                                     float* __restrict__ tmp) {
    const int tx = threadIdx.x & 31, r = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + tx;
    const int q0 = blockIdx.y * per_slice, q1 = min(n_part, q0 + per_slice);
    float s = 0.0f;
    if (c < C)
        for (int q = q0 + r; q < q1; q += 8) s += part[(size_t)q * C + c];
    __shared__ float red[8][32];
    red[r][tx] = s;
    __syncthreads();
    if (r == 0 && c < C) {
        float t = 0.0f;
        for (int k = 0; k < 8; ++k) t += red[k][tx];
        tmp[(size_t)blockIdx.y * C + c] = t;
    }
}

__global__ void k_bias_final(const float* __restrict__ tmp, int slices, int C, float* __restrict__ db) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    float s = 0.0f;
    for (int q = 0; q < slices; ++q) s += tmp[(size_t)q * C + c];
    db[c] = s;
}

// wf[t][c/8][o][c%8] = w[o][c][t] (c < Ci_pad), wb[t][o/8][c][o%8] = w[o][c][t] (o < Co_pad)
__global__ void k_weights_tc(const float* __restrict__ w, int Co, int Ci, int Ci_pad, int Co_pad,
                             __nv_bfloat16* __restrict__ wf, __nv_bfloat16* __restrict__ wb) {
    const int total = 9 * Co * Ci_pad + 9 * Ci * Co_pad;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        if (i < 9 * Co * Ci_pad) {
            const int e = i & 7, r = i >> 3, o = r % Co, q = (r / Co) % (Ci_pad >> 3), t = r / Co / (Ci_pad >> 3);
            const int c = 8 * q + e;
            wf[i] = __float2bfloat16_rn(c < Ci ? w[((size_t)o * Ci + c) * 9 + t] : 0.0f);
        } else {
            const int j = i - 9 * Co * Ci_pad;
            const int e = j & 7, r = j >> 3, c = r % Ci, q = (r / Ci) % (Co_pad >> 3), t = r / Ci / (Co_pad >> 3);
            const int o = 8 * q + e;
            wb[j] = __float2bfloat16_rn(o < Co ? w[((size_t)o * Ci + c) * 9 + t] : 0.0f);
        }
    }
}

__global__ void k_pack_input(const float* __restrict__ X, int N, int H, int W, int par, __nv_bfloat16* __restrict__ hi,
                             __nv_bfloat16* __restrict__ lo) {
    const long HW = (long)H * W, total = (long)N * HW;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        const int n = (int)(i / HW), y = (int)((i % HW) / W), x = (int)(i % W);
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = j < 2 ? X[((size_t)n * 2 + j) * HW + (i % HW)] : 0.0f;
        store_pair8(hi, lo, chunk_at(par, 1, H, W, n, y, x, 0), v);
    }
}

// out[n][c][y][x] = hi + lo of channel c < C_real of the pair a (any layout)
__global__ void k_unpack_act(const __nv_bfloat16* __restrict__ hi, const __nv_bfloat16* __restrict__ lo, int N, int H,
                             int W, int C8, int par, int C_real, float* __restrict__ out) {
    const long HW = (long)H * W, total = (long)N * C_real * HW;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        const int n = (int)(i / (C_real * HW)), c = (int)((i / HW) % C_real), y = (int)((i % HW) / W), x = (int)(i % W);
        const size_t o = chunk_at(par, C8, H, W, n, y, x, c >> 3) + (c & 7);
        out[i] = __bfloat162float(hi[o]) + __bfloat162float(lo[o]);
    }
}

__global__ void __launch_bounds__(256) k_mse_tc(const float* __restrict__ out, const float* __restrict__ t,
                                                const float* __restrict__ mask, int N, int H, int W, float inv_terms,
                                                __nv_bfloat16* __restrict__ ghi, __nv_bfloat16* __restrict__ glo,
                                                __nv_bfloat16* __restrict__ gphi, __nv_bfloat16* __restrict__ gplo,
                                                float* __restrict__ db_part, double* loss) {
    double acc = 0.0;
    float d0 = 0.0f, d1 = 0.0f;
    const long HW = (long)H * W, total = (long)N * HW;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        const int n = (int)(i / HW), p = (int)(i % HW), y = p / W, x = p % W;
        const float mk = mask[p];
        float g[8];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const long k = ((long)n * 2 + c) * HW + p;
            const float d = (out[k] - t[k]) * mk;
            acc += (double)d * d;
            g[c] = 2.0f * d * inv_terms;
        }
#pragma unroll
        for (int c = 2; c < 8; ++c) g[c] = 0.0f;
        d0 += g[0];
        d1 += g[1];
        store_pair8(ghi, glo, chunk_at(0, 1, H, W, n, y, x, 0), g);
        if (gphi) store_pair8(gphi, gplo, chunk_at(1, 1, H, W, n, y, x, 0), g);
    }
    __shared__ double rl[8];
    __shared__ float r0[8], r1[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
        d0 += __shfl_xor_sync(0xffffffffu, d0, o);
        d1 += __shfl_xor_sync(0xffffffffu, d1, o);
    }
    if ((threadIdx.x & 31) == 0) {
        rl[threadIdx.x >> 5] = acc;
        r0[threadIdx.x >> 5] = d0;
        r1[threadIdx.x >> 5] = d1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        float s0 = 0.0f, s1 = 0.0f;
        for (int q = 0; q < 8; ++q) {
            s += rl[q];
            s0 += r0[q];
            s1 += r1[q];
        }
        atomicAdd(loss, s * inv_terms);
        db_part[blockIdx.x * 2] = s0;
        db_part[blockIdx.x * 2 + 1] = s1;
    }
}

// ---------------------------------------------------------------------------------------
// host side

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn g_encode = nullptr;
bool g_ready = false;
int g_conv_dyn = 0, g_wg_dyn = 0;   // dynamic shared memory the two kernels may request

// map of one half (hi or lo) of a chunk-major tensor; box = 16 pixels x 8 channels x `rows`
// rows of one chunk (one parity plane of a parity-split tensor: chunk coordinate 4 q + plane)
bool enc_act(CUtensorMap* m, const __nv_bfloat16* base, const Act2& t, bool parity, int rows) {
    const size_t es = sizeof(__nv_bfloat16);
    const int C8 = t.C / 8, H = parity ? t.H / 2 : t.H, W = parity ? t.W / 2 : t.W, planes = parity ? 4 : 1;
    cuuint64_t dims[4] = {(cuuint64_t)W * 8, (cuuint64_t)H, (cuuint64_t)C8 * planes, (cuuint64_t)t.N};
    cuuint64_t strides[3] = {(cuuint64_t)W * 8 * es, (cuuint64_t)H * W * 8 * es, (cuuint64_t)C8 * planes * H * W * 8 * es};
    cuuint32_t box[4] = {128, (cuuint32_t)rows, 1, 1}, estr[4] = {1, 1, 1, 1};
    return g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int pow2_cols(int c) {
    int r = 32;
    while (r < c) r <<= 1;
    return r;
}

// floor((p + u - 1) / 2) for p, u in {0, 1} x {0, 1, 2}
int half_shift(int p, int u) { return (p + u - 1) >= 0 ? (p + u - 1) / 2 : -1; }

struct ConvPlan {
    ConvParams prm;
    dim3 grid;
    int smem;
};

void sort_groups(ConvArgs& a, const Group* g, int ng, int phases) {
    int k = 0;
    for (int ph = 0; ph < phases; ++ph) {
        a.gstart[ph] = k;
        for (int i = 0; i < ng; ++i)
            if (g[i].phase == ph) a.group[k++] = g[i];
    }
    for (int ph = phases; ph <= 4; ++ph) a.gstart[ph] = k;
}

// stages and tile sizes for a given N; returns false when not even one stage fits
bool fit_stages(ConvArgs& a) {
    a.a_slot = a.rows * 256;
    a.a_bytes = a.split * a.n_copy * 2 * a.a_slot;
    a.stage_bytes = a.a_bytes + 2 * 9 * a.N * 16;
    const int budget = g_conv_dyn - 1024;
    a.n_stage = std::min(kMaxStage, std::min(a.ksteps, budget / a.stage_bytes));
    return a.n_stage >= 1;
}

cudaError_t finish_plan(ConvPlan& pl, int n_img, int num_sms, int phases, int Ntot) {
    ConvArgs& a = pl.prm.a;
    // N: largest divisor of Ntot (<= 256) for which two stages fit, else one
    int best = 0;
    for (int N = std::min(256, Ntot); N >= 16; N -= 16) {
        if (Ntot % N) continue;
        a.N = N;
        if (!fit_stages(a)) continue;
        if (a.n_stage >= std::min(2, a.ksteps)) {
            best = N;
            break;
        }
        if (!best) best = N;
    }
    if (!best) return cudaErrorInvalidConfiguration;
    a.N = best;
    fit_stages(a);
    // phases per CTA: all of them if TMEM allows and the grid still covers the SMs
    const int tiles = a.tiles_x * a.tiles_y * n_img * (Ntot / a.N);
    a.P = phases;
    while (a.P > 1 && (a.P * a.N > 512 || tiles * (phases / a.P) < num_sms)) a.P >>= 1;
    if (a.P * a.N > 512) return cudaErrorInvalidConfiguration;
    a.tmem_cols = pow2_cols(a.P * a.N);
    for (int pg = 0; pg < 4; ++pg) {
        unsigned m = 0;
        if (pg < phases / a.P)
            for (int g = a.gstart[pg * a.P]; g < a.gstart[pg * a.P + a.P]; ++g) m |= 1u << a.group[g].copy;
        a.cmask[pg] = m;
    }
    pl.grid = dim3(a.tiles_x * a.tiles_y * n_img, phases / a.P, Ntot / a.N);
    int smem = a.n_stage * a.stage_bytes + 1024;
    // more than 256 TMEM columns: keep one CTA per SM so the allocation never waits
    if (a.tmem_cols > 256) smem = std::max(smem, kOneCtaPerSm);
    if (smem > g_conv_dyn) return cudaErrorInvalidConfiguration;
    pl.smem = smem;
    return cudaSuccess;
}

}  // namespace

cudaError_t tc_prepare() {
    if (g_ready) return cudaSuccess;
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return e != cudaSuccess ? e : cudaErrorNotSupported;
    g_encode = reinterpret_cast<EncodeTiledFn>(fn);
    int dev = 0, optin = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, k_conv_tc)) != cudaSuccess) return e;
    g_conv_dyn = std::min(kSmemLimit, optin - (int)fa.sharedSizeBytes);
    if ((e = cudaFuncGetAttributes(&fa, k_wgrad_tc)) != cudaSuccess) return e;
    g_wg_dyn = std::min(kSmemLimit, optin - (int)fa.sharedSizeBytes);
    if ((e = cudaFuncSetAttribute(k_conv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, g_conv_dyn)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, g_wg_dyn)) != cudaSuccess) return e;
    g_ready = true;
    return cudaSuccess;
}

cudaError_t tc_conv_forward(const TcLayer& L, const Act2& x, const __nv_bfloat16* wf, const float* bias, const Act2* y,
                            float* y32, unsigned* err, unsigned spin, int num_sms, cudaStream_t st) {
    cudaError_t e = tc_prepare();
    if (e != cudaSuccess) return e;
    static ConvPlan pl;
    std::memset(&pl, 0, sizeof pl);
    ConvArgs& a = pl.prm.a;
    const int Ho = L.Hout();
    Group g[kMaxGroup];
    int ng = 0, phases;
    a.split = 2;
    a.ksteps = L.Ci_pad / 16;
    if (!L.up) {
        // the input is read by parity planes: it must be stored split by parity
        if (!x.par) return cudaErrorInvalidValue;
        phases = 1;
        a.tiles_y = Ho / 8;
        a.tiles_x = Ho / 16;
        a.rows = 9;
        a.n_copy = 6;
        const int qx[3] = {0, 1, 1}, dx[3] = {0, -1, 0};
        for (int qy = 0; qy < 2; ++qy)
            for (int var = 0; var < 3; ++var) a.copy[qy * 3 + var] = Copy{-1, (int8_t)dx[var], (int8_t)(2 * qy + qx[var])};
        for (int u = 0; u < 3; ++u)
            for (int v = 0; v < 3; ++v) {
                const int qy = u == 1 ? 0 : 1, dy = u == 0 ? -1 : 0, var = v == 1 ? 0 : (v == 0 ? 1 : 2);
                g[ng++] = Group{0, (uint8_t)(qy * 3 + var), (uint8_t)(dy + 1), (uint8_t)(3 * u + v)};
            }
        a.osy = a.osx = 1;
    } else {
        phases = 4;
        a.tiles_y = L.Hin / 8;
        a.tiles_x = L.Hin / 16;
        if (x.par) return cudaErrorInvalidValue;
        a.rows = 10;
        a.n_copy = 3;
        for (int j = 0; j < 3; ++j) a.copy[j] = Copy{-1, (int8_t)(j - 1), -1};
        for (int py = 0; py < 2; ++py)
            for (int px = 0; px < 2; ++px)
                for (int u = 0; u < 3; ++u)
                    for (int v = 0; v < 3; ++v)
                        g[ng++] = Group{(uint8_t)(2 * py + px), (uint8_t)(half_shift(px, v) + 1),
                                        (uint8_t)(half_shift(py, u) + 1), (uint8_t)(3 * u + v)};
        a.osy = a.osx = 2;
        for (int ph = 0; ph < 4; ++ph) {
            a.opy[ph] = (int8_t)(ph >> 1);
            a.opx[ph] = (int8_t)(ph & 1);
        }
    }
    sort_groups(a, g, ng, phases);
    const bool last = y == nullptr;
    const int Ntot = (L.Co + 15) / 16 * 16;
    if ((e = finish_plan(pl, x.N, num_sms, phases, Ntot)) != cudaSuccess) return e;
    if (!enc_act(&pl.prm.amap[0], x.hi, x, x.par != 0, a.rows) || !enc_act(&pl.prm.amap[1], x.lo, x, x.par != 0, a.rows))
        return cudaErrorInvalidValue;
    a.wts = wf;
    a.wK8 = L.Ci_pad / 8;
    a.wR = L.Co;
    a.mode = last ? EPI_LAST : EPI_HIDDEN;
    a.oH = Ho;
    a.oW = Ho;
    a.oC = L.Co;
    a.out_par = last ? 0 : y->par;
    a.out_hi = last ? nullptr : y->hi;
    a.out_lo = last ? nullptr : y->lo;
    a.out_phi = last ? nullptr : y->phi;
    a.out_plo = last ? nullptr : y->plo;
    a.out32 = y32;
    a.bias = bias;
    a.relu = L.relu;
    a.err = err;
    a.spin = spin;
    k_conv_tc<<<pl.grid, kThreads, pl.smem, st>>>(pl.prm);
    return cudaGetLastError();
}

int tc_bias_parts(const TcLayer& L, int N, int num_sms) {
    // upper bound: one part per (tile, phase group)
    const int S = L.up ? L.Hout() : L.Hin / 2;   // sub-lattice side of the output gradient tiles
    (void)num_sms;
    return (S / 8) * (S / 16) * N * 4;
}

cudaError_t tc_conv_backward_data(const TcLayer& L, const Act2& dy, const __nv_bfloat16* wb, const Act2& act,
                                  const Act2& dx, float* db_part, int* n_part, unsigned* err, unsigned spin, int num_sms,
                                  cudaStream_t st) {
    cudaError_t e = tc_prepare();
    if (e != cudaSuccess) return e;
    static ConvPlan pl;
    std::memset(&pl, 0, sizeof pl);
    ConvArgs& a = pl.prm.a;
    Group g[kMaxGroup];
    int ng = 0, phases;
    a.split = 2;
    a.ksteps = L.Co_pad / 16;
    if (!L.up) {
        // dx on the input grid in four parity phases; dy rows a'+e, columns b'+f
        phases = 4;
        const int Sd = L.Hin / 2;
        a.tiles_y = Sd / 8;
        a.tiles_x = Sd / 16;
        a.rows = 9;
        a.n_copy = 2;
        for (int j = 0; j < 2; ++j) a.copy[j] = Copy{0, (int8_t)j, -1};
        for (int qy = 0; qy < 2; ++qy)
            for (int qx = 0; qx < 2; ++qx)
                for (int u = 0; u < 3; ++u)
                    for (int v = 0; v < 3; ++v) {
                        if ((qy == 0) != (u == 1) || (qx == 0) != (v == 1)) continue;
                        const int ey = (qy == 1 && u == 0) ? 1 : 0, ex = (qx == 1 && v == 0) ? 1 : 0;
                        g[ng++] = Group{(uint8_t)(2 * qy + qx), (uint8_t)ex, (uint8_t)ey, (uint8_t)(3 * u + v)};
                    }
        a.osy = a.osx = 2;
        for (int ph = 0; ph < 4; ++ph) {
            a.opy[ph] = (int8_t)(ph >> 1);
            a.opx[ph] = (int8_t)(ph & 1);
        }
        a.mode = EPI_BWD;
    } else {
        // stride-1 correlation of dy with the transposed weights, then 2 x 2 sums
        phases = 1;
        const int Sd = L.Hout();
        a.tiles_y = Sd / 8;
        a.tiles_x = Sd / 16;
        a.rows = 10;
        a.n_copy = 3;
        for (int j = 0; j < 3; ++j) a.copy[j] = Copy{-1, (int8_t)(j - 1), -1};
        for (int u = 0; u < 3; ++u)
            for (int v = 0; v < 3; ++v) g[ng++] = Group{0, (uint8_t)(2 - v), (uint8_t)(2 - u), (uint8_t)(3 * u + v)};
        a.osy = a.osx = 1;
        a.mode = EPI_POOL;
    }
    sort_groups(a, g, ng, phases);
    if (dy.par) return cudaErrorInvalidValue;   // both forms read dy by plain rows
    if ((e = finish_plan(pl, dy.N, num_sms, phases, L.Ci)) != cudaSuccess) return e;
    if (!enc_act(&pl.prm.amap[0], dy.hi, dy, false, a.rows) || !enc_act(&pl.prm.amap[1], dy.lo, dy, false, a.rows))
        return cudaErrorInvalidValue;
    a.wts = wb;
    a.wK8 = L.Co_pad / 8;
    a.wR = L.Ci;
    a.oH = L.Hin;
    a.oW = L.Hin;
    a.oC = L.Ci;
    a.out_par = dx.par;
    a.out_hi = dx.hi;
    a.out_lo = dx.lo;
    a.out_phi = dx.phi;
    a.out_plo = dx.plo;
    a.m_par = act.par;
    a.m_hi = act.hi;
    a.m_lo = act.lo;
    a.db_part = db_part;
    a.err = err;
    a.spin = spin;
    *n_part = (int)(pl.grid.x * pl.grid.y);
    k_conv_tc<<<pl.grid, kThreads, pl.smem, st>>>(pl.prm);
    return cudaGetLastError();
}

namespace {

struct WgPlan {
    WgParams prm;
    dim3 grid;
    int smem;
};

cudaError_t plan_wgrad(WgPlan& pl, const TcLayer& L, const Act2* x, const Act2* dy, int n_img, int num_sms) {
    std::memset(&pl, 0, sizeof pl);
    WgArgs& a = pl.prm.a;
    a.w2 = L.Co <= 16 ? 1 : 0;
    a.phases = L.up ? 4 : 1;
    const int S = L.up ? L.Hin : L.Hout();   // per-phase output sub-lattice side
    a.n_copy = L.up ? 3 : 6;
    if (a.w2) {
        a.N = (L.Co + 15) / 16 * 16;
        a.g_real = (L.Co + 7) / 8;
        a.x_real = std::min(16, L.Ci / 8);
        a.c_tiles = 1;
        a.Nc = 0;
    } else {
        a.Nc = L.Ci_pad >= 32 ? 32 : 16;
        a.N = a.Nc;
        a.g_real = std::min(16, L.Co / 8);
        a.x_real = a.Nc / 8;
        a.c_tiles = L.Ci_pad / a.Nc;
    }
    const int kinds = a.w2 ? (L.Ci + 127) / 128 : ((L.Co + 127) / 128) * a.c_tiles;
    if (9 * a.N > 512) return cudaErrorInvalidConfiguration;
    a.tmem_cols = pow2_cols(9 * a.N);
    // pixel rows per stage: 8 if two stages fit, else 4
    const int budget = g_wg_dyn - 1024;
    for (int rp = 8; rp >= 4; rp -= 4) {
        a.rows_px = rp;
        a.rows = rp + (L.up ? 2 : 1);
        a.g_slot = rp * 16 * 16;
        a.x_slot = a.rows * 256;
        a.g_bytes = 2 * a.g_real * a.g_slot;
        a.x_bytes = 2 * a.n_copy * a.x_real * a.x_slot;
        a.stage_bytes = a.g_bytes + a.x_bytes;
        // rows / columns beyond the real channels read on into the next 16 slots at most
        const int tail = 16 * std::max(a.g_slot, a.x_slot);
        a.n_stage = std::min(kMaxStage, (budget - tail) / a.stage_bytes);
        if (a.n_stage >= 2 || rp == 4) break;
    }
    if (a.n_stage < 1) return cudaErrorInvalidConfiguration;
    a.tiles_y = S / a.rows_px;
    a.tiles_x = S / 16;
    a.n_tiles = n_img * a.phases * a.tiles_x * a.tiles_y;
    a.n_split = std::max(1, std::min(a.n_tiles, num_sms / kinds));
    for (int j = 0; j < a.n_copy; ++j) {
        if (L.up) a.copy[j] = Copy{-1, (int8_t)(j - 1), -1};
        else {
            const int dxv[3] = {0, -1, 0}, qxv[3] = {0, 1, 1};
            a.copy[j] = Copy{-1, (int8_t)dxv[j % 3], (int8_t)(2 * (j / 3) + qxv[j % 3])};
        }
    }
    a.g_parity = L.up ? 1 : 0;
    for (int ph = 0; ph < a.phases; ++ph) {
        unsigned m = 0;
        for (int u = 0; u < 3; ++u)
            for (int v = 0; v < 3; ++v) {
                int cp, ro;
                if (L.up) {
                    cp = half_shift(ph & 1, v) + 1;
                    ro = half_shift(ph >> 1, u) + 1;
                } else {
                    const int qy = u == 1 ? 0 : 1, dyv = u == 0 ? -1 : 0, var = v == 1 ? 0 : (v == 0 ? 1 : 2);
                    cp = qy * 3 + var;
                    ro = dyv + 1;
                }
                a.grp[ph][3 * u + v][0] = (uint8_t)cp;
                a.grp[ph][3 * u + v][1] = (uint8_t)ro;
                m |= 1u << cp;
            }
        a.cmask[ph] = m;
    }
    if (x && dy) {
        // up layers read dy by parity planes (its parity copy), stride-2 layers by plain rows;
        // the input x of a stride-2 layer is read by parity planes, of an up layer by plain rows
        if (L.up ? (!dy->phi || x->par) : (dy->par || !x->par)) return cudaErrorInvalidValue;
        const __nv_bfloat16* ghi = L.up ? dy->phi : dy->hi;
        const __nv_bfloat16* glo = L.up ? dy->plo : dy->lo;
        if (!enc_act(&pl.prm.gmap[0], ghi, *dy, L.up != 0, a.rows_px) || !enc_act(&pl.prm.gmap[1], glo, *dy, L.up != 0, a.rows_px) ||
            !enc_act(&pl.prm.xmap[0], x->hi, *x, x->par != 0, a.rows) || !enc_act(&pl.prm.xmap[1], x->lo, *x, x->par != 0, a.rows))
            return cudaErrorInvalidValue;
    }
    pl.grid = dim3(a.n_split, kinds, 1);
    pl.smem = a.n_stage * a.stage_bytes + 16 * std::max(a.g_slot, a.x_slot) + 1024;
    if (a.tmem_cols > 256) pl.smem = std::max(pl.smem, kOneCtaPerSm);
    if (pl.smem > g_wg_dyn) return cudaErrorInvalidConfiguration;
    return cudaSuccess;
}

}  // namespace

size_t tc_wgrad_workspace(const TcLayer& L, int N, int num_sms) {
    if (tc_prepare() != cudaSuccess) return 0;
    static WgPlan pl;
    if (plan_wgrad(pl, L, nullptr, nullptr, N, num_sms) != cudaSuccess) return 0;
    return (size_t)pl.grid.x * pl.grid.y * 9 * 128 * pl.prm.a.N;
}

cudaError_t tc_conv_wgrad(const TcLayer& L, const Act2& x, const Act2& dy, float* ws, float* dw, unsigned* err,
                          unsigned spin, int num_sms, cudaStream_t st) {
    cudaError_t e = tc_prepare();
    if (e != cudaSuccess) return e;
    static WgPlan pl;
    if ((e = plan_wgrad(pl, L, &x, &dy, x.N, num_sms)) != cudaSuccess) return e;
    WgArgs& a = pl.prm.a;
    a.part = ws;
    a.err = err;
    a.spin = spin;
    k_wgrad_tc<<<pl.grid, kThreads, pl.smem, st>>>(pl.prm);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int total = L.Co * L.Ci * 9;
    k_wgrad_reduce<<<std::max(1, std::min(4 * num_sms, (total + 255) / 256)), 256, 0, st>>>(
        ws, L.Co, L.Ci, a.w2, a.c_tiles, a.Nc, a.N, a.n_split, dw);
    return cudaGetLastError();
}

cudaError_t tc_bias_reduce(const float* part, int n_part, int C, float* tmp, float* db, cudaStream_t st) {
    if (n_part < 1 || C < 1) return cudaErrorInvalidValue;
    const int slices = std::min(kBiasSlices, n_part), per = (n_part + slices - 1) / slices;
    k_bias_slices<<<dim3((C + 31) / 32, slices), 256, 0, st>>>(part, n_part, C, per, tmp);
    k_bias_final<<<(C + 127) / 128, 128, 0, st>>>(tmp, slices, C, db);
    return cudaGetLastError();
}

cudaError_t tc_weights(const TcLayer& L, const float* w32, __nv_bfloat16* wf, __nv_bfloat16* wb, cudaStream_t st) {
    const int total = 9 * L.Co * L.Ci_pad + 9 * L.Ci * L.Co_pad;
    k_weights_tc<<<std::max(1, std::min(1024, (total + 255) / 256)), 256, 0, st>>>(w32, L.Co, L.Ci, L.Ci_pad, L.Co_pad, wf,
                                                                                  wb);
    return cudaGetLastError();
}

cudaError_t tc_pack_input(const float* X, const Act2& x0, cudaStream_t st) {
    const long total = (long)x0.N * x0.H * x0.W;
    k_pack_input<<<(int)std::min<long>(2048, (total + 255) / 256), 256, 0, st>>>(X, x0.N, x0.H, x0.W, x0.par, x0.hi, x0.lo);
    return cudaGetLastError();
}

cudaError_t tc_unpack(const Act2& a, int C_real, float* out, cudaStream_t st) {
    if (C_real < 1 || C_real > a.C) return cudaErrorInvalidValue;
    const long total = (long)a.N * C_real * a.H * a.W;
    if (total == 0) return cudaSuccess;
    const int blocks = (int)std::min<long>((total + 255) / 256, 4096);
    k_unpack_act<<<blocks, 256, 0, st>>>(a.hi, a.lo, a.N, a.H, a.W, a.C >> 3, a.par, C_real, out);
    return cudaGetLastError();
}

cudaError_t tc_mse(const float* out, const float* t, const float* mask, const Act2& g, double n_terms, float* db_part,
                   int* n_part, double* loss, cudaStream_t st) {
    if (g.par) return cudaErrorInvalidValue;
    k_mse_tc<<<kMseBlocks, 256, 0, st>>>(out, t, mask, g.N, g.H, g.W, (float)(1.0 / n_terms), g.hi, g.lo, g.phi, g.plo,
                                         db_part, loss);
    *n_part = kMseBlocks;
    return cudaGetLastError();
}

}  // namespace ptylm
