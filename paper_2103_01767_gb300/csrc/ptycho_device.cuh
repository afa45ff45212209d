// ptycho_device.cuh -- device helpers shared by the per-position kernels: vector L2
// reductions and prefetches, the per-pixel error-metric terms, the team prologue and the
// patch gather / scatter of pass 1.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "team_fft.cuh"

namespace ptylm {

__device__ __forceinline__ void red_add_c64(float2* addr, float2 v) {
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(addr), "f"(v.x), "f"(v.y) : "memory");
}

// Read-only load that does not allocate in L1: for the object patch values, which each
// position reads once, so that they do not push the kernel's spilled registers (and other
// reused lines) out of L1.
__device__ __forceinline__ float2 ldg_stream(const float2* p) {
    float2 v;
    asm volatile("ld.global.nc.L1::no_allocate.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
    return v;
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

// Cache a, team-register order.  For BY >= 2 the two elements (e, e+1) of a thread that
// share a pass-3 group are adjacent, so one 16-byte access moves both: element e of thread
// t lives at float2 index (e/2)*2T + 2t + (e%2) of the position's M-element tile.  For
// BY == 1 (one element per group) the layout is e*T + t.
template <class G>
__device__ __forceinline__ void store_cache_group(float2* ak, const float2* av, int j) {
    const int tid = threadIdx.x % G::T;
    if constexpr (G::BY >= 2) {
        float4* a4 = reinterpret_cast<float4*>(ak) + tid;
#pragma unroll
        for (int i = 0; i < G::BY / 2; ++i)
            a4[(j * (G::BY / 2) + i) * G::T] = make_float4(av[2 * i].x, av[2 * i].y, av[2 * i + 1].x, av[2 * i + 1].y);
    } else {
        ak[j * G::T + tid] = av[0];
    }
}
template <class G>
__device__ __forceinline__ void load_cache_group(const float2* ak, float2* av, int j, int tid) {
    if constexpr (G::BY >= 2) {
        const float4* a4 = reinterpret_cast<const float4*>(ak) + tid;
#pragma unroll
        for (int i = 0; i < G::BY / 2; ++i) {
            const float4 q = __ldcs(a4 + (j * (G::BY / 2) + i) * G::T);
            av[2 * i] = make_float2(q.x, q.y);
            av[2 * i + 1] = make_float2(q.z, q.w);
        }
    } else {
        av[0] = __ldcs(ak + j * G::T + tid);
    }
}

// Asynchronous copy of `bytes` (a multiple of 16, both ends 16-byte aligned) from global to
// shared memory by the team's threads in 16-byte pieces; the caller waits with
// cp_async_wait_all() and a team barrier before any thread reads the copy.
__device__ __forceinline__ void cp_async_tile(void* dst_smem, const void* src, unsigned bytes, int tid, int nthreads) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst_smem));
    const char* s = reinterpret_cast<const char*>(src);
    for (unsigned off = 16u * tid; off < bytes; off += 16u * nthreads)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d + off), "l"(s + off) : "memory");
    asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Per-pixel error-metric terms of Sec. 4.1 Eq. ell_magnitude, from h = |psihat|^2 + b and
// the stored measurement term ym (sqrt(y) for the Gaussian metric, y for Poisson):
//   Gaussian  l = (zeta - sqrt y)^2 / 2,   dl = zeta - sqrt y,     d2l = 1
//   Poisson   l = zeta^2 - y log zeta^2,   dl = 2 zeta - 2 y/zeta, d2l = 2 + 2 y/zeta^2
// returned as the combinations the kernels use: l, dl, dl/zeta and sqrt(d2l)/zeta.  With
// r = h^(-1/2) (so zeta = h r, 1/zeta = r) the Poisson ratios are dl/zeta = 2 (h - y) r^2
// and sqrt(d2l)/zeta = sqrt(2 (h + y)) r^2: no division or IEEE square root per pixel.
struct PixelTerms {
    float l, dl, dl_over_zeta, sqrt_d2l_over_zeta, d2l;
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
        t.d2l = 1.0f;
    } else {
        // the hardware logarithm: its ~2^-21 relative error is far below the FP32 rounding
        // already in h, and l only enters f (FP64 sums) and the gain ratio
        t.l = WANT_L ? h - (ym > 0.0f ? ym * __logf(h) : 0.0f) : 0.0f;
        const float hy = h - ym;
        t.dl = 2.0f * hy * r;
        t.dl_over_zeta = 2.0f * hy * r * r;
        const float s = 2.0f * (h + ym);
        t.sqrt_d2l_over_zeta = s * rsqrtf(s) * r * r;
        t.d2l = s * r * r;
    }
    return t;
}

// The same terms for the single-problem error-metric kernels, taken straight from the
// unnormalised FFT output q (psihat = q / S, h = |q|^2 / M + b) with every constant factor
// of the per-thread sums applied once per position (LossSums::finish) instead of per pixel:
//   Gaussian  s0 = sum d^2, d = zeta - sqrt y       (l = s0 / 2, dl^2 = s0, d2l = 1 each)
//   Poisson   s0 = sum h,  s1 = sum y log2 h        (l = s0 - s1 ln 2)
//             s2 = sum ((h - y) r)^2                (dl^2 = 4 s2)
//             s3 = sum (h + y) r^2                  (d2l = 2 s3)
// With CACHE the cache factor a = psihat sqrt(d2l) / zeta = q ca and the gradient's
// frequency term (psihat / zeta) dl / S = q cg are returned as the real scales ca, cg.
// y log2 h needs no guard for y = 0: h >= b > 0.
struct LossSums {
    float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
    // this thread's sums of l, dl^2 and d2l over its `pixels` pixels
    template <int LOSS>
    __device__ __forceinline__ void finish(int pixels, float& l, float& dl2, float& d2l) const {
        if constexpr (LOSS == 0) {
            l = 0.5f * s0;
            dl2 = s0;
            d2l = (float)pixels;
        } else {
            l = fmaf(-0.69314718055994531f, s1, s0);
            dl2 = 4.0f * s2;
            d2l = 2.0f * s3;
        }
    }
};

template <int LOSS, bool CACHE>
__device__ __forceinline__ void loss_pixel(float2 q, float ym, float b, float invS, LossSums& acc, float& ca,
                                           float& cg) {
    const float invM = invS * invS;
    const float h = fmaf(invM, fmaf(q.x, q.x, q.y * q.y), b);
    const float r = rsqrtf(h);
    if constexpr (LOSS == 0) {
        const float d = fmaf(h, r, -ym);  // zeta - sqrt y
        acc.s0 = fmaf(d, d, acc.s0);
        if constexpr (CACHE) {
            ca = invS * r;         // sqrt(d2l) / zeta / S
            cg = (d * r) * invM;   // dl / zeta / S^2
        }
    } else {
        const float hy = h - ym;
        acc.s0 += h;
        acc.s1 = fmaf(ym, __log2f(h), acc.s1);
        const float u = hy * r;
        acc.s2 = fmaf(u, u, acc.s2);
        if constexpr (CACHE) {
            const float hp = h + ym;
            const float r2 = r * r;
            acc.s3 = fmaf(hp, r2, acc.s3);
            ca = (invS * 1.41421356237309505f) * (hp * rsqrtf(hp)) * r2;  // sqrt(2 (h + y)) / h / S
            cg = (hy * r2) * (2.0f * invM);                                 // 2 (h - y) / h / S^2
        }
    }
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
    fill_twiddles<G>(c.tw, tw_g, threadIdx.x, blockDim.x);
    c.team = threadIdx.x / G::T;
    c.tid = threadIdx.x % G::T;
    c.sm = dyn + G::TW_WORDS + c.team * G::EXW;
    __syncthreads();
    return c;
}

// Where a thread's E probe values P[BX*a + b][x] (a = 0..E-1, pass-1 layout, thread
// t = x + S*b) come from, 8 at a time (a = a0 .. a0 + 7): plain loads from the probe array
// (L1 / L2).
template <class G>
struct GlobalProbe {
    const float2* pr;
    __device__ __forceinline__ GlobalProbe(const float2* P, int tid)
        : pr(P + (tid >> G::LOG_S) * G::S + (tid & (G::S - 1))) {}
    template <class Dep>
    __device__ __forceinline__ void load8(float2* pv, int a0, const Dep*) const {
#pragma unroll
        for (int i = 0; i < 8; ++i) pv[i] = pr[G::BX * G::S * (a0 + i)];  // plain load: an __ldg is hoisted out of the position loop
    }
};

// The same probe values through read-only loads written as non-volatile inline PTX whose
// extra operand is an address of the current position (`dep`): they cannot be hoisted out
// of the position loop, but the compiler schedules them freely.  In the error-metric kernels
// this ordering is faster than GlobalProbe's (trial loss 252 -> 226 us, linearisation
// 442 -> 432 us at 1024^2 / 128^2 / 3600); in the GGN product it is slower (325 -> 340 us),
// so the product keeps GlobalProbe.
template <class G>
struct ScheduledProbe {
    const float2* pr;
    __device__ __forceinline__ ScheduledProbe(const float2* P, int tid)
        : pr(P + (tid >> G::LOG_S) * G::S + (tid & (G::S - 1))) {}
    template <class Dep>
    __device__ __forceinline__ void load8(float2* pv, int a0, const Dep* dep) const {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float2* q = pr + G::BX * G::S * (a0 + i);
            asm("ld.global.nc.v2.f32 {%0, %1}, [%2];" : "=f"(pv[i].x), "=f"(pv[i].y) : "l"(q), "l"(dep));
        }
    }
};

// Pass-1 gather: thread t = x + S*b holds rows y = BX*a + b of column x:
//   v[a] = P[y][x] * A[r0 + y][c0 + x].
// Lanes are consecutive columns: each warp load reads 256 contiguous bytes of one row.
template <class G, class PS>
__device__ __forceinline__ void gather_times_probe(float2* v, const float2* __restrict__ A, const PS& ps, int nx,
                                                   int r0, int c0, int tid) {
    const int x = tid & (G::S - 1), b = tid >> G::LOG_S;
    const float2* src = A + (size_t)(r0 + b) * nx + c0 + x;
    const size_t row_step = (size_t)G::BX * nx;
#pragma unroll
    for (int a0 = 0; a0 < G::E; a0 += 8) {
        float2 pv[8], av[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) av[i] = ldg_stream(src + row_step * (a0 + i));
        ps.load8(pv, a0, src);
#pragma unroll
        for (int i = 0; i < 8; ++i) v[a0 + i] = cmul(pv[i], av[i]);
        sched_fence();
    }
}
template <class G>
__device__ __forceinline__ void gather_times_probe(float2* v, const float2* __restrict__ A,
                                                   const float2* __restrict__ P, int nx, int r0,
                                                   int c0, int tid) {
    gather_times_probe<G>(v, A, GlobalProbe<G>(P, tid), nx, r0, c0, tid);
}

// Pass-1 scatter: out[r0 + y][c0 + x] += conj(P[y][x]) * v[a], same thread layout.
template <class G, class PS>
__device__ __forceinline__ void scatter_times_conj_probe(const float2* v, float2* out, const PS& ps, int nx, int r0,
                                                         int c0, int tid) {
    const int x = tid & (G::S - 1), b = tid >> G::LOG_S;
    float2* dst = out + (size_t)(r0 + b) * nx + c0 + x;
    const size_t row_step = (size_t)G::BX * nx;
#pragma unroll
    for (int a0 = 0; a0 < G::E; a0 += 8) {
        float2 pv[8];
        ps.load8(pv, a0, dst);
#pragma unroll
        for (int i = 0; i < 8; ++i) red_add_c64(dst + row_step * (a0 + i), cmulc(v[a0 + i], pv[i]));
        sched_fence();
    }
}
template <class G>
__device__ __forceinline__ void scatter_times_conj_probe(const float2* v, float2* out,
                                                         const float2* __restrict__ P, int nx,
                                                         int r0, int c0, int tid) {
    scatter_times_conj_probe<G>(v, out, GlobalProbe<G>(P, tid), nx, r0, c0, tid);
}

// Scatter of one position fused with the gather of the next, which share the probe values
// (the same thread layout): per chunk of 8 rows one probe load serves
//   out[r0 + y][c0 + x] += conj(P[y][x]) v[a]        (this position, Eq. jac_ampl adjoint)
//   v[a] = P[y][x] A[r1 + y][c1 + x]                  (next position, Eq. exit_wave)
// and the next position's object loads are in flight while the reductions issue, so the
// two memory phases cost one round trip per chunk instead of two.
template <class G, class PS>
__device__ __forceinline__ void scatter_then_gather(float2* v, float2* out, const float2* __restrict__ A, const PS& ps,
                                                    int nx, int r0, int c0, int r1, int c1, int tid) {
    const int x = tid & (G::S - 1), b = tid >> G::LOG_S;
    float2* dst = out + (size_t)(r0 + b) * nx + c0 + x;
    const float2* src = A + (size_t)(r1 + b) * nx + c1 + x;
    const size_t row_step = (size_t)G::BX * nx;
#pragma unroll
    for (int a0 = 0; a0 < G::E; a0 += 8) {
        float2 pv[8], av[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) av[i] = ldg_stream(src + row_step * (a0 + i));
        ps.load8(pv, a0, src);
#pragma unroll
        for (int i = 0; i < 8; ++i) red_add_c64(dst + row_step * (a0 + i), cmulc(v[a0 + i], pv[i]));
#pragma unroll
        for (int i = 0; i < 8; ++i) v[a0 + i] = cmul(pv[i], av[i]);
        sched_fence();
    }
}
template <class G>
__device__ __forceinline__ void scatter_then_gather(float2* v, float2* out, const float2* __restrict__ A,
                                                    const float2* __restrict__ P, int nx, int r0, int c0,
                                                    int r1, int c1, int tid) {
    scatter_then_gather<G>(v, out, A, GlobalProbe<G>(P, tid), nx, r0, c0, r1, c1, tid);
}

// Per-detector-pixel values between a thread's pass-3 layout (element e of thread t is the
// frequency (freq_ky(t), freq_kx(t, e))) and natural [S][S] order in global memory, through the
// team's exchange buffer viewed as S rows of S + 1 floats: a warp's lanes hold consecutive
// rows, so the padding keeps the scattered shared-memory accesses conflict-free, and the
// global side moves whole rows (coalesced) instead of one float per row and lane.
// Both start with a team barrier (the buffer must be free) and end with one; the caller
// synchronises the team again before the buffer's next use.
template <class G>
__device__ __forceinline__ void store_natural(const float* val, float* smf, float* out_k, int tid) {
    team_sync<G>();
    const int ky = freq_ky<G>(tid);
#pragma unroll
    for (int e = 0; e < G::E; ++e) smf[ky * (G::S + 1) + freq_kx<G>(tid, e)] = val[e];
    team_sync<G>();
#pragma unroll 8
    for (int i = 0; i < G::E; ++i) {
        const int idx = i * G::T + tid;
        out_k[idx] = smf[(idx >> G::LOG_S) * (G::S + 1) + (idx & (G::S - 1))];
    }
}
template <class G>
__device__ __forceinline__ void load_natural(const float* __restrict__ in_k, float* smf, float* val, int tid) {
    team_sync<G>();
#pragma unroll 8
    for (int i = 0; i < G::E; ++i) {
        const int idx = i * G::T + tid;
        smf[(idx >> G::LOG_S) * (G::S + 1) + (idx & (G::S - 1))] = __ldg(in_k + idx);
    }
    team_sync<G>();
    const int ky = freq_ky<G>(tid);
#pragma unroll
    for (int e = 0; e < G::E; ++e) val[e] = smf[ky * (G::S + 1) + freq_kx<G>(tid, e)];
}

// Joint gather (Eq. jac_ampl with both blocks): v[a] = P[y][x] A[r0+y][c0+x] + B[y][x] C[r0+y][c0+x],
// i.e. P . S_k dO + dP . S_k O for the direction (A, B) = (dO, dP) at the object C.
template <class G>
__device__ __forceinline__ void gather_joint(float2* v, const float2* __restrict__ A, const float2* __restrict__ P,
                                             const float2* __restrict__ B, const float2* __restrict__ C, int nx,
                                             int r0, int c0, int tid) {
    const int x = tid & (G::S - 1), b = tid >> G::LOG_S;
    const size_t off = (size_t)(r0 + b) * nx + c0 + x;
    const int poff = b * G::S + x;
    const size_t row_step = (size_t)G::BX * nx;
#pragma unroll
    for (int a0 = 0; a0 < G::E; a0 += 8) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int a = a0 + i;
            const float2 p = P[poff + G::BX * G::S * a];
            const float2 dp = B[poff + G::BX * G::S * a];
            const float2 da = __ldg(A + off + row_step * a);
            const float2 o = __ldg(C + off + row_step * a);
            const float2 t0 = cmul(p, da), t1 = cmul(dp, o);
            v[a] = make_float2(t0.x + t1.x, t0.y + t1.y);
        }
        sched_fence();
    }
}

// Probe block of the adjoint: part[y][x] += conj(C[r0+y][c0+x]) * v[a] in the team's own
// accumulator row (each element has one owner thread within the team: no atomics).
template <class G>
__device__ __forceinline__ void accumulate_probe_adjoint(const float2* v, float2* part, const float2* __restrict__ C,
                                                         int nx, int r0, int c0, int tid) {
    const int x = tid & (G::S - 1), b = tid >> G::LOG_S;
    const size_t off = (size_t)(r0 + b) * nx + c0 + x;
    const int poff = b * G::S + x;
    const size_t row_step = (size_t)G::BX * nx;
#pragma unroll
    for (int a0 = 0; a0 < G::E; a0 += 8) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int a = a0 + i;
            const float2 o = __ldg(C + off + row_step * a);
            float2* dst = part + poff + G::BX * G::S * a;
            const float2 t = cconjmul(o, v[a]);
            const float2 cur = *dst;
            *dst = make_float2(cur.x + t.x, cur.y + t.y);
        }
        sched_fence();
    }
}

}  // namespace ptylm
