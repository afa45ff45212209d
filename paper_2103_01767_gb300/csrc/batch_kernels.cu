// batch_kernels.cu -- the per-position operators over a batch of independent problems with
// uneven object sizes, probe sides (32, 64, 128), scans and losses, each operator as ONE
// persistent launch.
//
// Every CTA has 512 threads and 128 KB of exchange buffers.  A problem's FFT tile is its
// probe side S with E values per thread (Geo<LS, LE>): E = 32 gives teams of S^2/32 threads
// (16 teams per CTA for a 32 x 32 probe, 4 for 64 x 64, one for 128 x 128); E = 16, an
// autotuner choice for sides 32 and 64, gives teams of S^2/16 threads (8 and 2 per CTA),
// with twice the threads and half the registers per patch.  A work item is one problem's
// positions for all teams of the CTA.  CTAs take items from a device counter (largest
// patches first in the default order), branch once per item on the problem's tile and run
// the same team code as the single-problem kernels (gather x probe, team 2D FFT, frequency
// stage, inverse FFT, x conj(probe) and overlap scatter-add; App. A steps 1-4).  Positions beyond
// a problem's K in its last item run the FFT on zeros (the team barriers are CTA-wide) and
// touch no memory.  The last CTA to finish restores the counters, so the launch can be
// replayed inside a CUDA graph.
#include <type_traits>

#include "batch.h"
#include "ptycho_device.cuh"
#include "team_fft.cuh"
#include "reduce.cuh"

namespace ptylm {

// Shared-memory twiddles of the five tiles back to back (fill_twiddles: 2S entries each),
// built from the S-entry tables of sides 32, 64, 128 (a.tw, at 0, 32, 96).
template <class G>
__device__ __forceinline__ constexpr int batch_tw_offset() {
    return G::LOG_S == 5 ? (G::LOG_E == 5 ? 0 : 64) : G::LOG_S == 6 ? (G::LOG_E == 5 ? 128 : 256) : 384;
}
constexpr int kBatchTwWords = 640;
__device__ __forceinline__ void batch_fill_twiddles(float2* tw, const float2* w_all) {
    fill_twiddles<Geo<5, 5>>(tw + batch_tw_offset<Geo<5, 5>>(), w_all, threadIdx.x, blockDim.x);
    fill_twiddles<Geo<5, 4>>(tw + batch_tw_offset<Geo<5, 4>>(), w_all, threadIdx.x, blockDim.x);
    fill_twiddles<Geo<6, 5>>(tw + batch_tw_offset<Geo<6, 5>>(), w_all + 32, threadIdx.x, blockDim.x);
    fill_twiddles<Geo<6, 4>>(tw + batch_tw_offset<Geo<6, 4>>(), w_all + 32, threadIdx.x, blockDim.x);
    fill_twiddles<Geo<7, 5>>(tw + batch_tw_offset<Geo<7, 5>>(), w_all + 96, threadIdx.x, blockDim.x);
}

// Sum two per-thread doubles over the warp and add them to f[0], f[1].
__device__ __forceinline__ void warp_add_to(double* f, double x, double y) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_xor_sync(0xffffffffu, x, o);
        y += __shfl_xor_sync(0xffffffffu, y, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(f, x);
        atomicAdd(f + 1, y);
    }
}

// Forward model, error metric and (CACHE) cache a and gradient for one item.
template <class G, bool CACHE>
__device__ __forceinline__ void batch_forward_item(const BatchArgs& a, const BatchProblem& p, const BatchItem& it,
                                                   float2* smem, const float2* tw_all) {
    constexpr int TEAMS = BATCH_THREADS / G::T;
    const int team = threadIdx.x / G::T, tid = threadIdx.x % G::T;
    float2* sm = smem + team * G::EXW;
    const float2* tw = tw_all + batch_tw_offset<G>();
    const float invS = 1.0f / G::S;
    const float2* O = a.V + p.z_off;
    float2* gout = a.out + p.z_off;
    double acc_l = 0.0, acc_d = 0.0;
    float2 v[G::E];
    for (int j = 0; j < it.per_team; ++j) {
        const int k = it.k0 + team + TEAMS * j;
        const bool valid = k < p.K;
        const int2 rc = valid ? p.pos[k] : make_int2(0, 0);
        const float* yk = p.y + (size_t)(valid ? k : 0) * G::M + tid;
        if (valid) {
            gather_times_probe<G>(v, O, p.P, p.nx, rc.x, rc.y, tid);   // its loads first, then the prefetch
            prefetch_tile_l2(p.y + (size_t)k * G::M, sizeof(float) * G::M, tid);
        } else {
#pragma unroll
            for (int e = 0; e < G::E; ++e) v[e] = make_float2(0.0f, 0.0f);
        }
        float sl = 0.0f, sd = 0.0f, s2;
        LossSums ls;  // loss_pixel: h = |g / S|^2 + b (Eq. expected_count), constant factors at the end
        if constexpr (CACHE) {
            float2* ak = p.a_cache + (size_t)(valid ? k : 0) * G::M;
            auto group = [&](auto loss_c, float2* g, int jj) {
                constexpr int LOSS = decltype(loss_c)::value;
                float2 av[G::BY];
#pragma unroll
                for (int k2y = 0; k2y < G::BY; ++k2y) {
                    const int e = jj * G::BY + k2y;
                    float ca, cg;
                    loss_pixel<LOSS, true>(g[k2y], valid ? __ldg(yk + e * G::T) : 0.0f, p.b, invS, ls, ca, cg);
                    av[k2y] = g[k2y] * ca;
                    g[k2y] = g[k2y] * cg;
                }
                if (valid) store_cache_group<G>(ak, av, jj);
            };
            team_fft_roundtrip<G>(v, sm, tw, tid, [&](float2* g, int jj) {
                if (p.loss == 0) group(std::integral_constant<int, 0>{}, g, jj);
                else group(std::integral_constant<int, 1>{}, g, jj);
            });
            if (valid) scatter_times_conj_probe<G>(v, gout, p.P, p.nx, rc.x, rc.y, tid);
        } else {
            team_fft_fwd<G>(v, sm, tw, tid);
            auto pixels = [&](auto loss_c) {
                constexpr int LOSS = decltype(loss_c)::value;
#pragma unroll
                for (int e = 0; e < G::E; ++e) {
                    float ca, cg;
                    loss_pixel<LOSS, false>(v[e], valid ? __ldg(yk + e * G::T) : 0.0f, p.b, invS, ls, ca, cg);
                }
            };
            if (p.loss == 0) pixels(std::integral_constant<int, 0>{});
            else pixels(std::integral_constant<int, 1>{});
        }
        if (p.loss == 0) ls.finish<0>(G::E, sl, sd, s2);
        else ls.finish<1>(G::E, sl, sd, s2);
        if (valid) {
            acc_l += (double)sl;
            acc_d += (double)sd;
            if constexpr (CACHE) p.trp[(size_t)k * G::T + tid] = s2;   // for the closed-form diagonal
        }
        team_sync<G>();
    }
    warp_add_to(a.f + 2 * it.prob, acc_l, acc_d);
}

// out += J^T (Hess l . J v) for one item (App. A steps 2-4 with the cache a).
template <class G>
__device__ __forceinline__ void batch_matvec_item(const BatchArgs& a, const BatchProblem& p, const BatchItem& it,
                                                  float2* smem, const float2* tw_all) {
    constexpr int TEAMS = BATCH_THREADS / G::T;
    const int team = threadIdx.x / G::T, tid = threadIdx.x % G::T;
    float2* sm = smem + team * G::EXW;
    const float2* tw = tw_all + batch_tw_offset<G>();
    const float invM = 1.0f / G::M;
    const float2* V = a.V + p.z_off;
    float2* out = a.out + p.z_off;
    float2 v[G::E];
    for (int j = 0; j < it.per_team; ++j) {
        const int k = it.k0 + team + TEAMS * j;
        const bool valid = k < p.K;
        const int2 rc = valid ? p.pos[k] : make_int2(0, 0);
        const float2* ak = p.a_cache + (size_t)(valid ? k : 0) * G::M;
        if (valid) {
            gather_times_probe<G>(v, V, p.P, p.nx, rc.x, rc.y, tid);   // its loads first, then the prefetch
            prefetch_tile_l2(ak, sizeof(float2) * G::M, tid);
        } else {
#pragma unroll
            for (int e = 0; e < G::E; ++e) v[e] = make_float2(0.0f, 0.0f);
        }
        team_fft_roundtrip<G>(v, sm, tw, tid, [&](float2* g, int jj) {
            float2 av[G::BY];
            if (valid) {
                load_cache_group<G>(ak, av, jj, tid);
            } else {
#pragma unroll
                for (int k2y = 0; k2y < G::BY; ++k2y) av[k2y] = make_float2(0.0f, 0.0f);
            }
#pragma unroll
            for (int k2y = 0; k2y < G::BY; ++k2y) {
                const float t = (av[k2y].x * g[k2y].x + av[k2y].y * g[k2y].y) * invM;
                g[k2y] = av[k2y] * t;
            }
        });
        if (valid) scatter_times_conj_probe<G>(v, out, p.P, p.nx, rc.x, rc.y, tid);
        team_sync<G>();
    }
}

template <int KIND, class G>
__device__ __forceinline__ void batch_item(const BatchArgs& a, const BatchProblem& p, const BatchItem& it,
                                           float2* smem, const float2* tw) {
    if constexpr (KIND == BK_MATVEC) batch_matvec_item<G>(a, p, it, smem, tw);
    else batch_forward_item<G, KIND == BK_FWD_CACHE>(a, p, it, smem, tw);
}

// The persistent scheduler: take items until none are left, then let the last CTA reset
// the counters.
template <int KIND>
__global__ void __launch_bounds__(BATCH_THREADS, 1) k_batch(BatchArgs a) {
    extern __shared__ float4 dyn_smem_f4[];
    float2* tw = reinterpret_cast<float2*>(dyn_smem_f4);
    float2* smem = tw + kBatchTwWords;
    __shared__ int s_item;
    batch_fill_twiddles(tw, a.tw);
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(a.work, 1u);
        __syncthreads();  // also orders the twiddle stores before the first item
        const int idx = s_item;
        __syncthreads();
        if (idx >= a.n_items) break;
        const BatchItem it = a.items[idx];
        if (a.active && !a.active[it.prob]) continue;
        const BatchProblem p = a.probs[it.prob];
        switch (p.LS * 8 + p.LE) {
            case 5 * 8 + 5: batch_item<KIND, Geo<5, 5>>(a, p, it, smem, tw); break;
            case 5 * 8 + 4: batch_item<KIND, Geo<5, 4>>(a, p, it, smem, tw); break;
            case 6 * 8 + 5: batch_item<KIND, Geo<6, 5>>(a, p, it, smem, tw); break;
            case 6 * 8 + 4: batch_item<KIND, Geo<6, 4>>(a, p, it, smem, tw); break;
            default: batch_item<KIND, Geo<7, 5>>(a, p, it, smem, tw); break;
        }
        __syncthreads();  // the next item may lay its teams out differently in shared memory
    }
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(a.done, 1u) == gridDim.x - 1) {
            atomicExch(a.work, 0u);
            atomicExch(a.done, 0u);
            __threadfence();
        }
    }
}

// Measurements from the team-register order of one FFT tile to that of another (same side):
// dst[k][e*T + t] = src[k][e'*T' + t'] where (e', t') holds, in the source tile, the
// frequency (ky, kx) that (e, t) holds in the destination tile (freq_place).
template <int LS, int LF, int LT>
__global__ void k_batch_relayout(const float* __restrict__ src, float* __restrict__ dst, long total) {
    using GF = Geo<LS, LF>;
    using GT = Geo<LS, LT>;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        const long k = i / GT::M;
        const int r = (int)(i - k * GT::M);
        const int e = r / GT::T, t = r % GT::T;
        int tf, ef;
        freq_place<GF>(freq_ky<GT>(t), freq_kx<GT>(t, e), tf, ef);
        dst[i] = src[k * GF::M + ef * GF::T + tf];
    }
}

cudaError_t batch_relayout_measurements(int LS, int le_from, int le_to, const float* src, float* dst, int K, int blocks,
                                        cudaStream_t stream) {
    const long total = (long)K << (2 * LS);
    if (total == 0 || le_from == le_to) return cudaSuccess;
    switch (LS * 8 + le_to) {
        case 5 * 8 + 4: k_batch_relayout<5, 5, 4><<<blocks, 256, 0, stream>>>(src, dst, total); break;
        case 5 * 8 + 5: k_batch_relayout<5, 4, 5><<<blocks, 256, 0, stream>>>(src, dst, total); break;
        case 6 * 8 + 4: k_batch_relayout<6, 5, 4><<<blocks, 256, 0, stream>>>(src, dst, total); break;
        case 6 * 8 + 5: k_batch_relayout<6, 4, 5><<<blocks, 256, 0, stream>>>(src, dst, total); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// The closed-form diagonal (see batch.h): block g handles the g-th position of the batch.
__global__ void __launch_bounds__(256) k_batch_diag(const BatchProblem* __restrict__ probs,
                                                    const int* __restrict__ pos_first, int B,
                                                    const int* __restrict__ mask, float* D) {
    const int g = blockIdx.x;
    int lo = 0, hi = B;   // the problem b with pos_first[b] <= g < pos_first[b + 1]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pos_first[mid] <= g) lo = mid;
        else hi = mid;
    }
    const int b = lo;
    if (mask && !mask[b]) return;
    const BatchProblem p = probs[b];
    const int k = g - pos_first[b];
    const int S = 1 << p.LS, M = S * S, T = M >> p.LE;
    double s[1] = {0.0};
    for (int t = threadIdx.x; t < T; t += blockDim.x) s[0] += (double)p.trp[(size_t)k * T + t];
    block_sum<1>(s);
    __shared__ float scale;
    if (threadIdx.x == 0) scale = (float)s[0] / (2.0f * (float)M);
    __syncthreads();
    const int2 rc = p.pos[k];
    float* Db = D + p.z_off;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        const int y = m >> p.LS, x = m & (S - 1);
        const float2 pv = p.P[m];
        atomicAdd(Db + (size_t)(rc.x + y) * p.nx + rc.y + x, (pv.x * pv.x + pv.y * pv.y) * scale);
    }
}

cudaError_t batch_diag_launch(const BatchProblem* probs, const int* pos_first, int B, int total_positions,
                              const int* mask, float* D, cudaStream_t stream) {
    if (total_positions <= 0) return cudaSuccess;
    k_batch_diag<<<total_positions, 256, 0, stream>>>(probs, pos_first, B, mask, D);
    return cudaGetLastError();
}

// exchange words of a CTA: BATCH_THREADS / T teams of the widest tile's padded buffer
template <class G>
constexpr int batch_ex_words() { return (BATCH_THREADS / G::T) * G::EXW; }
constexpr int cmax(int a, int b) { return a > b ? a : b; }
constexpr int kBatchExWords = cmax(cmax(cmax(batch_ex_words<Geo<5, 5>>(), batch_ex_words<Geo<5, 4>>()),
                                        cmax(batch_ex_words<Geo<6, 5>>(), batch_ex_words<Geo<6, 4>>())),
                                   batch_ex_words<Geo<7, 5>>());
static size_t batch_smem_bytes() { return sizeof(float2) * (kBatchTwWords + kBatchExWords); }

static const void* batch_kernel_ptr(int kernel) {
    switch (kernel) {
        case BK_FWD_LOSS: return (const void*)k_batch<BK_FWD_LOSS>;
        case BK_FWD_CACHE: return (const void*)k_batch<BK_FWD_CACHE>;
        case BK_MATVEC: return (const void*)k_batch<BK_MATVEC>;
    }
    return nullptr;
}

cudaError_t batch_prepare(int* ctas_per_sm) {
    int best = 1 << 30;
    for (int k = 0; k < BK_COUNT; ++k) {
        const void* fn = batch_kernel_ptr(k);
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batch_smem_bytes());
        if (e != cudaSuccess) return e;
        int n = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, BATCH_THREADS, batch_smem_bytes());
        if (e != cudaSuccess) return e;
        best = n < best ? n : best;
    }
    *ctas_per_sm = best;
    return cudaSuccess;
}

cudaError_t batch_launch(int kernel, const BatchArgs& a, int grid, cudaStream_t stream) {
    const void* fn = batch_kernel_ptr(kernel);
    if (!fn || grid <= 0) return cudaErrorInvalidValue;
    BatchArgs arg = a;
    void* args[] = {&arg};
    return cudaLaunchKernel(fn, dim3(grid), dim3(BATCH_THREADS), args, batch_smem_bytes(), stream);
}

}  // namespace ptylm
