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
#include "ptycho_device.cuh"
#include "reduce.cuh"
#include "team_fft.cuh"

namespace ptylm {

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
                    const PixelTerms t = pixel_terms<true>(a.loss, h, __ldg(yk + e * G::T));
                    sl += t.l;
                    sd += t.dl * t.dl;
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
