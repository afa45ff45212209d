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
#include <type_traits>

#include "kernels.h"
#include "ptycho_device.cuh"
#include "reduce.cuh"
#include "team_fft.cuh"

namespace ptylm {

// Per-kernel argument structs, built from PtyArgs by kernel_launch.  They stay small (the
// matvec's 88 bytes): larger by-value argument blocks cost the register-bound matvec spills.
struct FwdArgs {
    const float2* O;
    const float2* P;
    const int2* pos;
    const float* y;
    float2* a_cache;
    float2* out;
    float* out_real;
    double* partials;
    unsigned* counter;
    double* scal;
    const float2* tw;
    float* trp;
    float2* outP_part;
    int K, nx;
    float b;
    int loss;
};
struct MatvecArgs {
    const float2* O;      // the direction vO
    const float2* P;
    const int2* pos;
    const float2* a_cache;
    float2* out;
    const float2* tw;
    const float2* VP;     // joint: probe part of the direction
    const float2* Olin;   // joint: object at the linearisation point
    float2* outP_part;    // joint: per-team probe accumulators
    int K, nx;
    const double* skip;   // return at once when *skip != 0 (NULL: never)
};
struct AdjArgs {          // J^T w and J v
    const float2* O;      // linearisation point
    const float2* V;      // jvp direction vO
    const float2* VP;     // jvp joint: probe direction
    const float2* P;
    const int2* pos;
    const float* w;
    float2* out;
    float* out_real;
    float2* scratch;
    const float2* tw;
    float2* outP_part;
    int K, nx;
    float b;
};

// ---------------------------------------------------------------------------------------
// Forward model + error metric (+ cache and gradient when CACHE; intensities only when
// INTENSITY).
// ---------------------------------------------------------------------------------------
// Whether k_forward stages the measurements in shared memory (it then needs 4 M more bytes).
template <int LS, bool CACHE, bool INTENSITY, bool JOINT, bool MAG>
__host__ __device__ constexpr bool forward_stages_y() { return LS == 7 && !INTENSITY && !JOINT && !MAG; }

template <int LS, int LE, bool CACHE, bool INTENSITY = false, bool JOINT = false, bool MAG = false>
__global__ void __launch_bounds__(Geo<LS, LE>::THREADS, 512 / Geo<LS, LE>::THREADS)
k_forward(FwdArgs a) {
    using G = Geo<LS, LE>;
    TeamCtx<G> c = team_setup<G>(a.tw);
    const float invS = 1.0f / G::S;
    double acc_l = 0.0, acc_d = 0.0;
    const int ky = freq_ky<G>(c.tid);
    const int stride = gridDim.x * G::TEAMS;
    // 128^2 object-only linearisations fuse each position's gradient scatter with the next
    // position's gather (one probe load serves both), as the GGN product does.
    constexpr bool FUSED = CACHE && LS == 7 && !JOINT && !INTENSITY && !MAG;
    // 128^2 object-only error-metric evaluations (with or without the cache) stage each
    // position's measurements (64 KB) in shared memory with asynchronous copies issued
    // before the FFT, instead of waiting on 32 dependent loads per thread after it.
    constexpr bool STAGE_Y = forward_stages_y<LS, CACHE, INTENSITY, JOINT, MAG>();
    static_assert((G::TW_WORDS + G::EXW) % 2 == 0, "staged measurements must start 16-byte aligned");
    float* sy = reinterpret_cast<float*>(c.sm + G::EXW);
    const ScheduledProbe<G> probe(a.P, c.tid);
    float2 v[G::E];
    int k = blockIdx.x * G::TEAMS + c.team;
    if constexpr (FUSED) {
        if (k < a.K) {
            const int2 rc = a.pos[k];
            gather_times_probe<G>(v, a.O, probe, a.nx, rc.x, rc.y, c.tid);
        }
    }
    for (; k < a.K; k += stride) {
        const int2 rc = a.pos[k];
        const float* yk = a.y + (size_t)k * G::M + c.tid;  // measurements in team-register order
        // the gather's loads go first: the measurement copies are only waited for after the FFT
        if constexpr (!FUSED) gather_times_probe<G>(v, a.O, probe, a.nx, rc.x, rc.y, c.tid);
        if constexpr (STAGE_Y) cp_async_tile(sy, a.y + (size_t)k * G::M, sizeof(float) * G::M, c.tid, G::T);
        else if constexpr (!INTENSITY && !MAG) prefetch_tile_l2(a.y + (size_t)k * G::M, sizeof(float) * G::M, c.tid);
        float sl = 0.0f, sd = 0.0f;
        LossSums ls;  // this thread's error-metric sums at position k (loss_pixel)
        if constexpr (CACHE) {
            float2* ak = a.a_cache + (size_t)k * G::M;
            // psihat = g / S (Eq. expected_count: h = |psihat|^2 + b); the cache gets
            // psihat sqrt(d2l) / zeta, g becomes psihat dl / zeta with the inverse's 1/S folded in
            auto group = [&](auto loss_c, float2* g, int j) {
                constexpr int LOSS = decltype(loss_c)::value;
                float2 av[G::BY];
#pragma unroll
                for (int k2y = 0; k2y < G::BY; ++k2y) {
                    const int e = j * G::BY + k2y;
                    const float ym = STAGE_Y ? sy[e * G::T + c.tid] : __ldg(yk + e * G::T);
                    float ca, cg;
                    loss_pixel<LOSS, true>(g[k2y], ym, a.b, invS, ls, ca, cg);
                    av[k2y] = g[k2y] * ca;
                    g[k2y] = g[k2y] * cg;
                }
                store_cache_group<G>(ak, av, j);
            };
            team_fft_roundtrip<G>(
                v, c.sm, c.tw, c.tid,
                [&](float2* g, int j) {
                    if (a.loss == 0) group(std::integral_constant<int, 0>{}, g, j);
                    else group(std::integral_constant<int, 1>{}, g, j);
                },
                [&] {
                    if constexpr (STAGE_Y) cp_async_wait_all();   // the pass-3 barrier follows
                });
            float s2;  // sum of d2l over this thread's pixels (closed-form diagonal)
            if (a.loss == 0) ls.finish<0>(G::E, sl, sd, s2);
            else ls.finish<1>(G::E, sl, sd, s2);
            if (a.trp) a.trp[(size_t)k * G::T + c.tid] = s2;
            if constexpr (FUSED) {
                const int kn = k + stride;
                if (kn < a.K) {
                    const int2 rn = a.pos[kn];
                    scatter_then_gather<G>(v, a.out, a.O, probe, a.nx, rc.x, rc.y, rn.x, rn.y, c.tid);
                } else {
                    scatter_times_conj_probe<G>(v, a.out, probe, a.nx, rc.x, rc.y, c.tid);
                }
            } else {
                scatter_times_conj_probe<G>(v, a.out, probe, a.nx, rc.x, rc.y, c.tid);
            }
            if constexpr (JOINT)
                accumulate_probe_adjoint<G>(v, a.outP_part + (size_t)(blockIdx.x * G::TEAMS + c.team) * G::M,
                                            a.O, a.nx, rc.x, rc.y, c.tid);
        } else {
            team_fft_fwd<G>(v, c.sm, c.tw, c.tid);
            if constexpr (STAGE_Y) {
                cp_async_wait_all();
                __syncthreads();
            }
            if constexpr (MAG || INTENSITY) {
                float hv[G::E];
#pragma unroll
                for (int e = 0; e < G::E; ++e) {
                    const float2 ps = v[e] * invS;
                    const float h = ps.x * ps.x + ps.y * ps.y + a.b;
                    if constexpr (MAG) {
                        // zeta in natural order; the unit phasor u = psihat / zeta in team order
                        const float r = rsqrtf(h);
                        hv[e] = h * r;
                        if (a.a_cache) a.a_cache[(size_t)k * G::M + e * G::T + c.tid] = ps * r;
                    } else {
                        hv[e] = h;
                    }
                }
                store_natural<G>(hv, reinterpret_cast<float*>(c.sm), a.out_real + (size_t)k * G::M, c.tid);
            } else {
                auto pixels = [&](auto loss_c) {
                    constexpr int LOSS = decltype(loss_c)::value;
#pragma unroll
                    for (int e = 0; e < G::E; ++e) {
                        float ca, cg;
                        loss_pixel<LOSS, false>(v[e], STAGE_Y ? sy[e * G::T + c.tid] : __ldg(yk + e * G::T), a.b,
                                                invS, ls, ca, cg);
                    }
                    float s2;
                    ls.finish<LOSS>(G::E, sl, sd, s2);
                };
                if (a.loss == 0) pixels(std::integral_constant<int, 0>{});
                else pixels(std::integral_constant<int, 1>{});
            }
        }
        acc_l += (double)sl;
        acc_d += (double)sd;
        team_sync<G>();
    }
    double sums[2] = {acc_l, acc_d};
    if constexpr (!INTENSITY && !MAG) grid_reduce<2>(sums, a.partials, a.counter, a.scal, S_F, OP_STORE, 1.0);
}

// ---------------------------------------------------------------------------------------
// GGN-vector product: out += J^T (Hess l . J v), with t = Re(conj(a) F(P S_k v)),
// chihat = a t (App. A steps 2-4; the closed-form diagonal Hessian of step 3(ii) is folded
// into a).  out must hold lambda D v (or zero) on entry.
// ---------------------------------------------------------------------------------------
template <int LS, int LE, bool JOINT = false>
__global__ void __launch_bounds__(Geo<LS, LE>::THREADS, 512 / Geo<LS, LE>::THREADS)
k_ggn_matvec(MatvecArgs a) {
    using G = Geo<LS, LE>;
    if (a.skip && __ldcg(a.skip) != 0.0) return;  // every CTA reads the same value
    TeamCtx<G> c = team_setup<G>(a.tw);
    const float invM = 1.0f / G::M;
    const int stride = gridDim.x * G::TEAMS;
    // 128^2 object-only products fuse each position's scatter with the next one's gather
    // (one probe load serves both); elsewhere the registers this keeps live across the
    // loop would spill.
    constexpr bool FUSED = LS == 7 && !JOINT;
    float2 v[G::E];
    int k = blockIdx.x * G::TEAMS + c.team;
    if constexpr (FUSED) {
        if (k < a.K) {
            const int2 rc = a.pos[k];
            gather_times_probe<G>(v, a.O, a.P, a.nx, rc.x, rc.y, c.tid);
        }
    }
    for (; k < a.K; k += stride) {
        const int2 rc = a.pos[k];
        const float2* ak = a.a_cache + (size_t)k * G::M;
        prefetch_tile_l2(ak, sizeof(float2) * G::M, c.tid);
        if constexpr (!FUSED) {
            if constexpr (JOINT) gather_joint<G>(v, a.O, a.P, a.VP, a.Olin, a.nx, rc.x, rc.y, c.tid);
            else gather_times_probe<G>(v, a.O, a.P, a.nx, rc.x, rc.y, c.tid);
        }
        team_fft_roundtrip<G>(v, c.sm, c.tw, c.tid, [&](float2* g, int j) {
            float2 av[G::BY];
            load_cache_group<G>(ak, av, j, c.tid);
#pragma unroll
            for (int k2y = 0; k2y < G::BY; ++k2y) {
                const float t = (av[k2y].x * g[k2y].x + av[k2y].y * g[k2y].y) * invM;
                g[k2y] = av[k2y] * t;
            }
        });
        if constexpr (FUSED) {
            const int kn = k + stride;
            if (kn < a.K) {
                const int2 rn = a.pos[kn];
                scatter_then_gather<G>(v, a.out, a.O, a.P, a.nx, rc.x, rc.y, rn.x, rn.y, c.tid);
            } else {
                scatter_times_conj_probe<G>(v, a.out, a.P, a.nx, rc.x, rc.y, c.tid);
            }
        } else {
            scatter_times_conj_probe<G>(v, a.out, a.P, a.nx, rc.x, rc.y, c.tid);
            if constexpr (JOINT)
                accumulate_probe_adjoint<G>(v, a.outP_part + (size_t)(blockIdx.x * G::TEAMS + c.team) * G::M, a.Olin,
                                            a.nx, rc.x, rc.y, c.tid);
        }
        // No barrier before the next position: its first shared-memory writes go to the
        // slots this same thread read last (team_fft_roundtrip).
    }
}

// ---------------------------------------------------------------------------------------
// J^T w: chihat = psihat w / zeta, recomputing psihat from (O, P).  out += result.
// ---------------------------------------------------------------------------------------
template <int LS, int LE, bool JOINT = false>
__global__ void __launch_bounds__(Geo<LS, LE>::THREADS, 512 / Geo<LS, LE>::THREADS)
k_jtvp(AdjArgs a) {
    using G = Geo<LS, LE>;
    TeamCtx<G> c = team_setup<G>(a.tw);
    const float invS = 1.0f / G::S;
    const int ky = freq_ky<G>(c.tid);
    float2 v[G::E];
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
        if constexpr (JOINT)
            accumulate_probe_adjoint<G>(v, a.outP_part + (size_t)(blockIdx.x * G::TEAMS + c.team) * G::M, a.O,
                                        a.nx, rc.x, rc.y, c.tid);
        // No barrier before the next position: its first shared-memory writes go to the
        // slots this same thread read last (team_fft_roundtrip).
    }
}

// ---------------------------------------------------------------------------------------
// J v = Re(conj(psihat) F(P S_k v)) / zeta, written in natural [K][S][S] order.  psihat is
// recomputed and parked in a per-team global scratch slot while the direction is transformed.
// ---------------------------------------------------------------------------------------
template <int LS, int LE, bool JOINT = false>
__global__ void __launch_bounds__(Geo<LS, LE>::THREADS, 512 / Geo<LS, LE>::THREADS)
k_jvp(AdjArgs a) {
    using G = Geo<LS, LE>;
    TeamCtx<G> c = team_setup<G>(a.tw);
    const float invS = 1.0f / G::S;
    float2* slot = a.scratch + (size_t)(blockIdx.x * G::TEAMS + c.team) * G::M + c.tid;
    float2 v[G::E];
    for (int k = blockIdx.x * G::TEAMS + c.team; k < a.K; k += gridDim.x * G::TEAMS) {
        const int2 rc = a.pos[k];
        gather_times_probe<G>(v, a.O, a.P, a.nx, rc.x, rc.y, c.tid);
        team_fft_fwd<G>(v, c.sm, c.tw, c.tid);
#pragma unroll
        for (int e = 0; e < G::E; ++e) slot[e * G::T] = v[e];
        team_sync<G>();
        if constexpr (JOINT) gather_joint<G>(v, a.V, a.P, a.VP, a.O, a.nx, rc.x, rc.y, c.tid);
        else gather_times_probe<G>(v, a.V, a.P, a.nx, rc.x, rc.y, c.tid);
        team_fft_fwd<G>(v, c.sm, c.tw, c.tid);
        float jv[G::E];
#pragma unroll
        for (int e = 0; e < G::E; ++e) {
            const float2 ps = slot[e * G::T] * invS;
            const float2 dps = v[e] * invS;
            const float inv_zeta = rsqrtf(ps.x * ps.x + ps.y * ps.y + a.b);
            jv[e] = (ps.x * dps.x + ps.y * dps.y) * inv_zeta;
        }
        store_natural<G>(jv, reinterpret_cast<float*>(c.sm), a.out_real + (size_t)k * G::M, c.tid);
        team_sync<G>();
    }
}

// ---------------------------------------------------------------------------------------
// Measurements from natural [K][S][S] order to the kernels' team-register order
// y_perm[k][e*T + t] = y[k][ky(t)][kx(t, e)] (its square root for the Gaussian metric,
// whose terms only use sqrt(y)).
// ---------------------------------------------------------------------------------------
template <int LS, int LE>
__global__ void k_permute_measurements(const float* __restrict__ y, float* __restrict__ y_perm, long total,
                                       int take_sqrt, unsigned* bad) {
    using G = Geo<LS, LE>;
    bool ok = true;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        const long k = i / G::M;
        const int r = (int)(i - k * G::M);
        const int e = r / G::T, t = r % G::T;
        const float v = y[k * G::M + freq_ky<G>(t) * G::S + freq_kx<G>(t, e)];
        ok = ok && (v >= 0.0f) && (v <= 3.402823466e38f);   // counts are finite and >= 0 (NaN fails both)
        if (y_perm) y_perm[i] = take_sqrt ? sqrtf(v) : v;
    }
    if (bad && !ok) atomicOr(bad, 1u);
}

// the FFT tiles a single-problem context may use: (side, log2 values per thread)
#define PTYLM_TILE_CASES(X) X(5, 5) X(5, 4) X(6, 5) X(6, 4) X(7, 5)

cudaError_t permute_measurements(int LS, int LE, const float* y, float* y_perm, int K, int take_sqrt, int blocks,
                                 cudaStream_t stream, unsigned* bad) {
    const long total = (long)K << (2 * LS);
    if (total == 0) return cudaSuccess;
    switch (LS * 8 + LE) {
#define PTYLM_PERMUTE(ls, le) \
    case ls * 8 + le: k_permute_measurements<ls, le><<<blocks, 256, 0, stream>>>(y, y_perm, total, take_sqrt, bad); break;
        PTYLM_TILE_CASES(PTYLM_PERMUTE)
#undef PTYLM_PERMUTE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// J v and J^T w from a stored unit phasor u = psihat / zeta (team order, a_cache slot):
//   J v = Re(conj(u) F(P S_k vO + vP S_k O)),   J^T w = S_k^T conj(P) F^H(u w)  (+ probe part)
// one 2D FFT per position instead of two (psihat is not recomputed).
// ---------------------------------------------------------------------------------------
template <int LS, int LE, bool JOINT = false>
__global__ void __launch_bounds__(Geo<LS, LE>::THREADS, 512 / Geo<LS, LE>::THREADS)
k_jvp_phasor(AdjArgs a, const float2* __restrict__ u) {
    using G = Geo<LS, LE>;
    TeamCtx<G> c = team_setup<G>(a.tw);
    const float invS = 1.0f / G::S;
    float2 v[G::E];
    for (int k = blockIdx.x * G::TEAMS + c.team; k < a.K; k += gridDim.x * G::TEAMS) {
        const int2 rc = a.pos[k];
        if constexpr (JOINT) gather_joint<G>(v, a.V, a.P, a.VP, a.O, a.nx, rc.x, rc.y, c.tid);
        else gather_times_probe<G>(v, a.V, a.P, a.nx, rc.x, rc.y, c.tid);
        team_fft_fwd<G>(v, c.sm, c.tw, c.tid);
        const float2* uk = u + (size_t)k * G::M + c.tid;
        float jv[G::E];
#pragma unroll
        for (int e = 0; e < G::E; ++e) {
            const float2 ue = __ldg(uk + e * G::T);
            jv[e] = (ue.x * v[e].x + ue.y * v[e].y) * invS;
        }
        store_natural<G>(jv, reinterpret_cast<float*>(c.sm), a.out_real + (size_t)k * G::M, c.tid);
        team_sync<G>();
    }
}

template <int LS, int LE, bool JOINT = false>
__global__ void __launch_bounds__(Geo<LS, LE>::THREADS, 512 / Geo<LS, LE>::THREADS)
k_jtvp_phasor(AdjArgs a, const float2* __restrict__ u) {
    using G = Geo<LS, LE>;
    TeamCtx<G> c = team_setup<G>(a.tw);
    const float invS = 1.0f / G::S;
    float2 v[G::E];
    for (int k = blockIdx.x * G::TEAMS + c.team; k < a.K; k += gridDim.x * G::TEAMS) {
        const int2 rc = a.pos[k];
        const float2* uk = u + (size_t)k * G::M + c.tid;
        float wv[G::E];
        load_natural<G>(a.w + (size_t)k * G::M, reinterpret_cast<float*>(c.sm), wv, c.tid);
#pragma unroll
        for (int e = 0; e < G::E; ++e) v[e] = __ldg(uk + e * G::T) * (wv[e] * invS);
        team_sync<G>();  // every thread's reads of the staged w are done
        team_fft_inv<G>(v, c.sm, c.tw, c.tid);
        scatter_times_conj_probe<G>(v, a.out, a.P, a.nx, rc.x, rc.y, c.tid);
        if constexpr (JOINT)
            accumulate_probe_adjoint<G>(v, a.outP_part + (size_t)(blockIdx.x * G::TEAMS + c.team) * G::M, a.O,
                                        a.nx, rc.x, rc.y, c.tid);
    }
}

// ---------------------------------------------------------------------------------------
// Closed-form GGN diagonal, App. B (Eqs. ggn_diag_elem_final, ggn_diag_mat, ggn_joint_diag),
// in real coordinates: D_O[n] = sum_{k: n in patch k} |P[n - r_k]|^2 tr_k / (2M) and
// D_P[m] = sum_k |O[r_k + m]|^2 tr_k / (2M), tr_k = sum_m d2l_km.
// ---------------------------------------------------------------------------------------
template <int LS, int LE>
__global__ void __launch_bounds__(Geo<LS, LE>::T)
k_diag_object(const float* __restrict__ trp, const int2* __restrict__ pos, const float2* __restrict__ P, int nx,
              float* D_O, float* tr) {
    using G = Geo<LS, LE>;
    const int k = blockIdx.x, tid = threadIdx.x;
    double s[1] = {(double)trp[(size_t)k * G::T + tid]};
    block_sum<1>(s);
    __shared__ float trk;
    if (tid == 0) {
        trk = (float)s[0];
        tr[k] = trk;
    }
    __syncthreads();
    const float scale = trk / (2.0f * G::M);
    const int2 rc = pos[k];
    const int x = tid & (G::S - 1), b = tid >> G::LOG_S;
#pragma unroll 8
    for (int a = 0; a < G::E; ++a) {
        const int y = G::BX * a + b;
        const float2 p = P[y * G::S + x];
        atomicAdd(D_O + (size_t)(rc.x + y) * nx + rc.y + x, (p.x * p.x + p.y * p.y) * scale);
    }
}

template <int LS, int LE>
__global__ void k_diag_probe(const float* __restrict__ tr, const int2* __restrict__ pos, int K,
                             const float2* __restrict__ O, int nx, float* D_P) {
    using G = Geo<LS, LE>;
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < G::M; m += gridDim.x * blockDim.x) {
        const int y = m >> G::LOG_S, x = m & (G::S - 1);
        float acc = 0.0f;
        for (int k = 0; k < K; ++k) {
            const int2 rc = pos[k];
            const float2 o = O[(size_t)(rc.x + y) * nx + rc.y + x];
            acc += (o.x * o.x + o.y * o.y) * tr[k];
        }
        D_P[m] = acc / (2.0f * G::M);
    }
}

cudaError_t launch_ggn_diag(int LS, int LE, const float* trp, const int2* pos, int K, const float2* O, const float2* P,
                            int nx, float* D_O, float* D_P, float* tr, cudaStream_t stream) {
    if (K == 0) return cudaSuccess;
    switch (LS * 8 + LE) {
#define PTYLM_DIAG(ls, le)                                                                                  \
    case ls * 8 + le:                                                                                         \
        k_diag_object<ls, le><<<K, Geo<ls, le>::T, 0, stream>>>(trp, pos, P, nx, D_O, tr);                   \
        if (D_P) k_diag_probe<ls, le><<<(Geo<ls, le>::M + 255) / 256, 256, 0, stream>>>(tr, pos, K, O, nx, D_P); \
        break;
        PTYLM_TILE_CASES(PTYLM_DIAG)
#undef PTYLM_DIAG
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Host-side dispatch.
// ---------------------------------------------------------------------------------------
int cta_threads(int LS, int LE) {
    switch (LS * 8 + LE) {
#define PTYLM_THREADS(ls, le) case ls * 8 + le: return Geo<ls, le>::THREADS;
        PTYLM_TILE_CASES(PTYLM_THREADS)
#undef PTYLM_THREADS
    }
    return 0;
}

int cta_teams(int LS, int LE) {
    switch (LS * 8 + LE) {
#define PTYLM_TEAMS(ls, le) case ls * 8 + le: return Geo<ls, le>::TEAMS;
        PTYLM_TILE_CASES(PTYLM_TEAMS)
#undef PTYLM_TEAMS
    }
    return 0;
}

size_t cta_smem_bytes(int LS, int LE) {
    switch (LS * 8 + LE) {
#define PTYLM_SMEM(ls, le) case ls * 8 + le: return sizeof(float2) * (Geo<ls, le>::TW_WORDS + Geo<ls, le>::TEAMS * Geo<ls, le>::EXW);
        PTYLM_TILE_CASES(PTYLM_SMEM)
#undef PTYLM_SMEM
    }
    return 0;
}

template <int LS, int LE>
static const void* kernel_ptr(int kid) {
    switch (kid) {
        case KID_FWD_LOSS: return (const void*)k_forward<LS, LE, false>;
        case KID_FWD_CACHE: return (const void*)k_forward<LS, LE, true>;
        case KID_MATVEC: return (const void*)k_ggn_matvec<LS, LE>;
        case KID_JTVP: return (const void*)k_jtvp<LS, LE>;
        case KID_JVP: return (const void*)k_jvp<LS, LE>;
        case KID_FWD_INTENSITY: return (const void*)k_forward<LS, LE, false, true>;
        case KID_FWD_CACHE_J: return (const void*)k_forward<LS, LE, true, false, true>;
        case KID_MATVEC_J: return (const void*)k_ggn_matvec<LS, LE, true>;
        case KID_JTVP_J: return (const void*)k_jtvp<LS, LE, true>;
        case KID_JVP_J: return (const void*)k_jvp<LS, LE, true>;
        case KID_FWD_MAG: return (const void*)k_forward<LS, LE, false, false, false, true>;
        case KID_JVP_U: return (const void*)k_jvp_phasor<LS, LE, false>;
        case KID_JVP_U_J: return (const void*)k_jvp_phasor<LS, LE, true>;
        case KID_JTVP_U: return (const void*)k_jtvp_phasor<LS, LE, false>;
        case KID_JTVP_U_J: return (const void*)k_jtvp_phasor<LS, LE, true>;
    }
    return nullptr;
}

static const void* kernel_for(int LS, int LE, int kid) {
    switch (LS * 8 + LE) {
#define PTYLM_KERNEL(ls, le) case ls * 8 + le: return kernel_ptr<ls, le>(kid);
        PTYLM_TILE_CASES(PTYLM_KERNEL)
#undef PTYLM_KERNEL
    }
    return nullptr;
}

// Dynamic shared memory of kernel `kid`: the team buffers, plus the staged measurements of
// the 128^2 error-metric kernel.
static size_t kernel_smem_bytes(int LS, int LE, int kid) {
    const bool stage = LS == 7 && ((kid == KID_FWD_LOSS && forward_stages_y<7, false, false, false, false>()) ||
                                   (kid == KID_FWD_CACHE && forward_stages_y<7, true, false, false, false>()));
    return cta_smem_bytes(LS, LE) + (stage ? sizeof(float) * Geo<7>::M : 0);
}

cudaError_t kernel_prepare(int LS, int LE, int kid, int* ctas_per_sm) {
    const void* fn = kernel_for(LS, LE, kid);
    if (!fn) return cudaErrorInvalidValue;
    const size_t smem = kernel_smem_bytes(LS, LE, kid);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, fn, cta_threads(LS, LE), smem);
}

cudaError_t kernel_launch(int LS, int LE, int kid, const PtyArgs& a, int grid, cudaStream_t stream) {
    const void* fn = kernel_for(LS, LE, kid);
    if (!fn || grid <= 0) return cudaErrorInvalidValue;
    FwdArgs fa{a.O, a.P, a.pos, a.y, a.a_cache, a.out, a.out_real, a.partials, a.counter, a.scal, a.tw,
               a.trp, a.outP_part, a.K, a.nx, a.b, a.loss};
    MatvecArgs ma{a.O, a.P, a.pos, a.a_cache, a.out, a.tw, a.VP, a.Olin, a.outP_part, a.K, a.nx, a.skip};
    AdjArgs ja{a.O, a.V, a.VP, a.P, a.pos, a.w, a.out, a.out_real, a.scratch, a.tw, a.outP_part, a.K, a.nx, a.b};
    const float2* u = a.a_cache;
    void* arg = nullptr;
    switch (kid) {
        case KID_FWD_LOSS: case KID_FWD_CACHE: case KID_FWD_INTENSITY: case KID_FWD_CACHE_J: case KID_FWD_MAG:
            arg = &fa;
            break;
        case KID_MATVEC: case KID_MATVEC_J: arg = &ma; break;
        default: arg = &ja; break;
    }
    void* args[] = {arg, &u};
    return cudaLaunchKernel(fn, dim3(grid), dim3(cta_threads(LS, LE)), args, kernel_smem_bytes(LS, LE, kid), stream);
}

}  // namespace ptylm
