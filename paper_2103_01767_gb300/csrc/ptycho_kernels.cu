// ptycho_kernels.cu -- per-scan-position kernels of the far-field ptychography model and
// its matrix-free derivatives (arXiv 2103.01767), for sm_103a.
//
// Every kernel is persistent over scan positions: a team of T = S*S/32 threads owns one
// position at a time, gathers its S x S object patch straight into registers, runs the
// team FFT of team_fft.cuh, applies an elementwise frequency-domain stage in registers
// and (except the loss-only kernel) runs the inverse FFT and scatter-adds the conj(P)
// weighted result into an object-sized array with vector float2 reductions in L2.
//
//   KID_FWD_LOSS   f = sum l(zeta, y)                        (Sec. 4.1, Eq. ell_magnitude)
//   KID_FWD_INTENSITY  h = |psihat|^2 + b in natural order   (Sec. 2, Eq. expected_count)
//   KID_FWD_CACHE  f, ||grad_zeta l||^2, the cache a = psihat (d2l)^(1/2) / zeta and
//                  grad f = J^T grad_zeta l                  (App. A step 1)
//   KID_MATVEC     J^T( Hess l . J v )  with the cache a     (App. A steps 2-4)
//   KID_JTVP       J^T w                                     (App. A Eq. arbitrary_jtvp_sequence)
//   KID_JVP        J v                                       (App. B Eq. jac_ampl, forward mode)
#include "kernels.h"
#include "reduce.cuh"
#include "team_fft.cuh"

namespace ptylm {

__device__ __forceinline__ void red_add_c64(float2* addr, float2 v) {
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(addr), "f"(v.x), "f"(v.y) : "memory");
}

// Asynchronous bulk prefetch of `bytes` (multiple of 16, 16-byte aligned) into L2.
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Threads 0, 1, ... each start pulling one 16 KB chunk of a position's tile (`bytes`, a
// multiple of 16) toward L2, so the spectral stage later finds it there instead of waiting
// on DRAM.
__device__ __forceinline__ void prefetch_tile_l2(const void* tile, unsigned bytes, int tid) {
    constexpr unsigned kChunk = 16384;
    const unsigned off = (unsigned)tid * kChunk;
    if (off < bytes) prefetch_l2(reinterpret_cast<const char*>(tile) + off, min(kChunk, bytes - off));
}

// Per-pixel error-metric terms of Sec. 4.1 Eq. ell_magnitude, from h = |psihat|^2 + b and
// the stored measurement term ym (sqrt(y) for the Gaussian metric, y for Poisson):
//   Gaussian  l = (zeta - sqrt y)^2 / 2,   dl = zeta - sqrt y,     d2l = 1
//   Poisson   l = zeta^2 - y log zeta^2,   dl = 2 zeta - 2 y/zeta, d2l = 2 + 2 y/zeta^2
// returned as the combinations the kernels use: l, dl, dl/zeta and sqrt(d2l)/zeta.  With
// r = h^(-1/2) (so zeta = h r, 1/zeta = r) the Poisson ratios are dl/zeta = 2 (h - y) r^2
// and sqrt(d2l)/zeta = sqrt(2 (h + y)) r^2: no division or IEEE square root per pixel.
struct PixelTerms {
    float l, dl, dl_over_zeta, sqrt_d2l_over_zeta;
};
template <bool WANT_L>
__device__ __forceinline__ PixelTerms pixel_terms(int loss, float h, float ym) {
    PixelTerms t;
    const float r = rsqrtf(h);
    const float zeta = h * r;
    if (loss == 0) {
        const float d = zeta - ym;
        t.l = WANT_L ? 0.5f * d * d : 0.0f;
        t.dl = d;
        t.dl_over_zeta = d * r;
        t.sqrt_d2l_over_zeta = r;
    } else {
        t.l = WANT_L ? h - (ym > 0.0f ? ym * logf(h) : 0.0f) : 0.0f;
        const float hy = h - ym;
        t.dl = 2.0f * hy * r;
        t.dl_over_zeta = 2.0f * hy * r * r;
        const float s = 2.0f * (h + ym);
        t.sqrt_d2l_over_zeta = s * rsqrtf(s) * r * r;
    }
    return t;
}

// Common prologue: twiddles into shared memory, team and thread indices.
template <class G>
struct TeamCtx {
    float2* tw;
    float2* sm;
    int team, tid;
};

template <class G>
__device__ __forceinline__ TeamCtx<G> team_setup(const float2* tw_g) {
    extern __shared__ float4 dyn_smem_f4[];
    float2* dyn = reinterpret_cast<float2*>(dyn_smem_f4);
    TeamCtx<G> c;
    c.tw = dyn;
    for (int i = threadIdx.x; i < G::S; i += blockDim.x) c.tw[i] = tw_g[i];
    c.team = threadIdx.x / G::T;
    c.tid = threadIdx.x % G::T;
    c.sm = dyn + G::S + c.team * G::M;
    __syncthreads();
    return c;
}

// Pass-1 gather: thread t = x + S*b holds rows y = BX*a + b of column x:
//   v[a] = P[y][x] * A[r0 + y][c0 + x].
// Lanes are consecutive columns: each warp load reads 256 contiguous bytes of one row.
template <class G>
__device__ __forceinline__ void gather_times_probe(float2* v, const float2* __restrict__ A,
                                                   const float2* __restrict__ P, int nx, int r0,
                                                   int c0, int tid) {
    const int x = tid & (G::S - 1), b = tid >> G::LOG_S;
    const float2* src = A + (size_t)(r0 + b) * nx + c0 + x;
    const float2* pr = P + b * G::S + x;
    const size_t row_step = (size_t)G::BX * nx;
#pragma unroll
    for (int a0 = 0; a0 < 32; a0 += 8) {
        float2 pv[8], av[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            pv[i] = pr[G::BX * G::S * (a0 + i)];  // plain load: an __ldg is hoisted out of the position loop
            av[i] = __ldg(src + row_step * (a0 + i));
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) v[a0 + i] = cmul(pv[i], av[i]);
        sched_fence();
    }
}

// Pass-1 scatter: out[r0 + y][c0 + x] += conj(P[y][x]) * v[a], same thread layout.
template <class G>
__device__ __forceinline__ void scatter_times_conj_probe(const float2* v, float2* out,
                                                         const float2* __restrict__ P, int nx,
                                                         int r0, int c0, int tid) {
    const int x = tid & (G::S - 1), b = tid >> G::LOG_S;
    float2* dst = out + (size_t)(r0 + b) * nx + c0 + x;
    const float2* pr = P + b * G::S + x;
    const size_t row_step = (size_t)G::BX * nx;
#pragma unroll
    for (int a0 = 0; a0 < 32; a0 += 8) {
        float2 pv[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) pv[i] = pr[G::BX * G::S * (a0 + i)];
#pragma unroll
        for (int i = 0; i < 8; ++i) red_add_c64(dst + row_step * (a0 + i), cmulc(v[a0 + i], pv[i]));
        sched_fence();
    }
}

// ---------------------------------------------------------------------------------------
// Forward model + error metric (+ cache and gradient when CACHE; intensities only when
// INTENSITY).
// ---------------------------------------------------------------------------------------
template <int LS, bool CACHE, bool INTENSITY = false>
__global__ void __launch_bounds__(Geo<LS>::THREADS, 512 / Geo<LS>::THREADS)
k_forward(PtyArgs a) {
    using G = Geo<LS>;
    TeamCtx<G> c = team_setup<G>(a.tw);
    const float invS = 1.0f / G::S;
    double acc_l = 0.0, acc_d = 0.0;
    const int ky = freq_ky<G>(c.tid);
    float2 v[32];
    for (int k = blockIdx.x * G::TEAMS + c.team; k < a.K; k += gridDim.x * G::TEAMS) {
        const int2 rc = a.pos[k];
        const float* yk = a.y + (size_t)k * G::M + c.tid;  // measurements in team-register order
        if constexpr (!INTENSITY) prefetch_tile_l2(a.y + (size_t)k * G::M, sizeof(float) * G::M, c.tid);
        float sl = 0.0f, sd = 0.0f;
        gather_times_probe<G>(v, a.O, a.P, a.nx, rc.x, rc.y, c.tid);
        if constexpr (CACHE) {
            float2* ak = a.a_cache + (size_t)k * G::M + c.tid;
            team_fft_roundtrip<G>(v, c.sm, c.tw, c.tid, [&](float2* g, int j) {
#pragma unroll
                for (int k2y = 0; k2y < G::BY; ++k2y) {
                    const int e = j * G::BY + k2y;
                    const float2 ps = g[k2y] * invS;                    // orthonormal psihat
                    const float h = ps.x * ps.x + ps.y * ps.y + a.b;    // Eq. expected_count
                    const PixelTerms t = pixel_terms<true>(a.loss, h, __ldg(yk + e * G::T));
                    sl += t.l;
                    sd += t.dl * t.dl;
                    ak[e * G::T] = ps * t.sqrt_d2l_over_zeta;
                    g[k2y] = ps * (t.dl_over_zeta * invS);  // psihat grad l / zeta, inverse 1/S folded in
                }
            });
            scatter_times_conj_probe<G>(v, a.out, a.P, a.nx, rc.x, rc.y, c.tid);
        } else {
            team_fft_fwd<G>(v, c.sm, c.tw, c.tid);
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                const float2 ps = v[e] * invS;
                const float h = ps.x * ps.x + ps.y * ps.y + a.b;
                if constexpr (INTENSITY) {
                    a.out_real[(size_t)k * G::M + ky * G::S + freq_kx<G>(c.tid, e)] = h;
                } else {
                    sl += pixel_terms<true>(a.loss, h, __ldg(yk + e * G::T)).l;
                }
            }
        }
        acc_l += (double)sl;
        acc_d += (double)sd;
        team_sync<G>();
    }
    double sums[2] = {acc_l, acc_d};
    if constexpr (!INTENSITY) grid_reduce<2>(sums, a.partials, a.counter, a.scal, S_F, OP_STORE, 1.0);
}

// ---------------------------------------------------------------------------------------
// GGN-vector product: out += J^T (Hess l . J v), with t = Re(conj(a) F(P S_k v)),
// chihat = a t (App. A steps 2-4; the closed-form diagonal Hessian of step 3(ii) is folded
// into a).  out must hold lambda D v (or zero) on entry.
// ---------------------------------------------------------------------------------------
template <int LS>
__global__ void __launch_bounds__(Geo<LS>::THREADS, 512 / Geo<LS>::THREADS)
k_ggn_matvec(PtyArgs a) {
    using G = Geo<LS>;
    TeamCtx<G> c = team_setup<G>(a.tw);
    const float invM = 1.0f / G::M;
    float2 v[32];
    for (int k = blockIdx.x * G::TEAMS + c.team; k < a.K; k += gridDim.x * G::TEAMS) {
        const int2 rc = a.pos[k];
        prefetch_tile_l2(a.a_cache + (size_t)k * G::M, sizeof(float2) * G::M, c.tid);
        gather_times_probe<G>(v, a.O, a.P, a.nx, rc.x, rc.y, c.tid);
        const float2* ak = a.a_cache + (size_t)k * G::M + c.tid;
        team_fft_roundtrip<G>(v, c.sm, c.tw, c.tid, [&](float2* g, int j) {
            float2 av[G::BY];
#pragma unroll
            for (int k2y = 0; k2y < G::BY; ++k2y) av[k2y] = __ldcs(ak + (j * G::BY + k2y) * G::T);
#pragma unroll
            for (int k2y = 0; k2y < G::BY; ++k2y) {
                const float t = (av[k2y].x * g[k2y].x + av[k2y].y * g[k2y].y) * invM;
                g[k2y] = av[k2y] * t;
            }
        });
        scatter_times_conj_probe<G>(v, a.out, a.P, a.nx, rc.x, rc.y, c.tid);
        // No barrier before the next position: its first shared-memory writes go to the
        // slots this same thread read last (team_fft_roundtrip).
    }
}

// ---------------------------------------------------------------------------------------
// J^T w: chihat = psihat w / zeta, recomputing psihat from (O, P).  out += result.
// ---------------------------------------------------------------------------------------
template <int LS>
__global__ void __launch_bounds__(Geo<LS>::THREADS, 512 / Geo<LS>::THREADS)
k_jtvp(PtyArgs a) {
    using G = Geo<LS>;
    TeamCtx<G> c = team_setup<G>(a.tw);
    const float invS = 1.0f / G::S;
    const int ky = freq_ky<G>(c.tid);
    float2 v[32];
    for (int k = blockIdx.x * G::TEAMS + c.team; k < a.K; k += gridDim.x * G::TEAMS) {
        const int2 rc = a.pos[k];
        gather_times_probe<G>(v, a.O, a.P, a.nx, rc.x, rc.y, c.tid);
        const float* wk = a.w + (size_t)k * G::M + ky * G::S;
        team_fft_roundtrip<G>(v, c.sm, c.tw, c.tid, [&](float2* g, int j) {
#pragma unroll
            for (int k2y = 0; k2y < G::BY; ++k2y) {
                const int kx = freq_kx<G>(c.tid, j * G::BY + k2y);
                const float2 ps = g[k2y] * invS;
                const float inv_zeta = rsqrtf(ps.x * ps.x + ps.y * ps.y + a.b);
                g[k2y] = ps * (__ldg(wk + kx) * inv_zeta * invS);
            }
        });
        scatter_times_conj_probe<G>(v, a.out, a.P, a.nx, rc.x, rc.y, c.tid);
        // No barrier before the next position: its first shared-memory writes go to the
        // slots this same thread read last (team_fft_roundtrip).
    }
}

// ---------------------------------------------------------------------------------------
// J v = Re(conj(psihat) F(P S_k v)) / zeta, written in natural [K][S][S] order.  psihat is
// recomputed and parked in a per-team global scratch slot while the direction is transformed.
// ---------------------------------------------------------------------------------------
template <int LS>
__global__ void __launch_bounds__(Geo<LS>::THREADS, 512 / Geo<LS>::THREADS)
k_jvp(PtyArgs a) {
    using G = Geo<LS>;
    TeamCtx<G> c = team_setup<G>(a.tw);
    const float invS = 1.0f / G::S;
    float2* slot = a.scratch + (size_t)(blockIdx.x * G::TEAMS + c.team) * G::M + c.tid;
    float2 v[32];
    for (int k = blockIdx.x * G::TEAMS + c.team; k < a.K; k += gridDim.x * G::TEAMS) {
        const int2 rc = a.pos[k];
        gather_times_probe<G>(v, a.O, a.P, a.nx, rc.x, rc.y, c.tid);
        team_fft_fwd<G>(v, c.sm, c.tw, c.tid);
#pragma unroll
        for (int e = 0; e < 32; ++e) slot[e * G::T] = v[e];
        team_sync<G>();
        gather_times_probe<G>(v, a.V, a.P, a.nx, rc.x, rc.y, c.tid);
        team_fft_fwd<G>(v, c.sm, c.tw, c.tid);
        float* ok = a.out_real + (size_t)k * G::M + freq_ky<G>(c.tid) * G::S;
#pragma unroll
        for (int e = 0; e < 32; ++e) {
            const int kx = freq_kx<G>(c.tid, e);
            const float2 ps = slot[e * G::T] * invS;
            const float2 dps = v[e] * invS;
            const float inv_zeta = rsqrtf(ps.x * ps.x + ps.y * ps.y + a.b);
            ok[kx] = (ps.x * dps.x + ps.y * dps.y) * inv_zeta;
        }
        team_sync<G>();
    }
}

// ---------------------------------------------------------------------------------------
// Measurements from natural [K][S][S] order to the kernels' team-register order
// y_perm[k][e*T + t] = y[k][ky(t)][kx(t, e)] (its square root for the Gaussian metric,
// whose terms only use sqrt(y)).
// ---------------------------------------------------------------------------------------
template <int LS>
__global__ void k_permute_measurements(const float* __restrict__ y, float* __restrict__ y_perm, long total,
                                       int take_sqrt) {
    using G = Geo<LS>;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        const long k = i / G::M;
        const int r = (int)(i - k * G::M);
        const int e = r / G::T, t = r % G::T;
        const float v = y[k * G::M + freq_ky<G>(t) * G::S + freq_kx<G>(t, e)];
        y_perm[i] = take_sqrt ? sqrtf(v) : v;
    }
}

cudaError_t permute_measurements(int LS, const float* y, float* y_perm, int K, int take_sqrt, int blocks,
                                 cudaStream_t stream) {
    const long total = (long)K << (2 * LS);
    if (total == 0) return cudaSuccess;
    switch (LS) {
        case 5: k_permute_measurements<5><<<blocks, 256, 0, stream>>>(y, y_perm, total, take_sqrt); break;
        case 6: k_permute_measurements<6><<<blocks, 256, 0, stream>>>(y, y_perm, total, take_sqrt); break;
        case 7: k_permute_measurements<7><<<blocks, 256, 0, stream>>>(y, y_perm, total, take_sqrt); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Host-side dispatch.
// ---------------------------------------------------------------------------------------
int cta_threads(int LS) {
    switch (LS) {
        case 5: return Geo<5>::THREADS;
        case 6: return Geo<6>::THREADS;
        case 7: return Geo<7>::THREADS;
    }
    return 0;
}

int cta_teams(int LS) {
    switch (LS) {
        case 5: return Geo<5>::TEAMS;
        case 6: return Geo<6>::TEAMS;
        case 7: return Geo<7>::TEAMS;
    }
    return 0;
}

size_t cta_smem_bytes(int LS) {
    switch (LS) {
        case 5: return sizeof(float2) * (Geo<5>::S + Geo<5>::TEAMS * Geo<5>::M);
        case 6: return sizeof(float2) * (Geo<6>::S + Geo<6>::TEAMS * Geo<6>::M);
        case 7: return sizeof(float2) * (Geo<7>::S + Geo<7>::TEAMS * Geo<7>::M);
    }
    return 0;
}

template <int LS>
static const void* kernel_ptr(int kid) {
    switch (kid) {
        case KID_FWD_LOSS: return (const void*)k_forward<LS, false>;
        case KID_FWD_CACHE: return (const void*)k_forward<LS, true>;
        case KID_MATVEC: return (const void*)k_ggn_matvec<LS>;
        case KID_JTVP: return (const void*)k_jtvp<LS>;
        case KID_JVP: return (const void*)k_jvp<LS>;
        case KID_FWD_INTENSITY: return (const void*)k_forward<LS, false, true>;
    }
    return nullptr;
}

static const void* kernel_for(int LS, int kid) {
    switch (LS) {
        case 5: return kernel_ptr<5>(kid);
        case 6: return kernel_ptr<6>(kid);
        case 7: return kernel_ptr<7>(kid);
    }
    return nullptr;
}

cudaError_t kernel_prepare(int LS, int kid, int* ctas_per_sm) {
    const void* fn = kernel_for(LS, kid);
    if (!fn) return cudaErrorInvalidValue;
    const size_t smem = cta_smem_bytes(LS);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, fn, cta_threads(LS), smem);
}

cudaError_t kernel_launch(int LS, int kid, const PtyArgs& a, int grid, cudaStream_t stream) {
    const void* fn = kernel_for(LS, kid);
    if (!fn || grid <= 0) return cudaErrorInvalidValue;
    PtyArgs copy = a;
    void* args[] = {&copy};
    return cudaLaunchKernel(fn, dim3(grid), dim3(cta_threads(LS)), args, cta_smem_bytes(LS), stream);
}

}  // namespace ptylm
