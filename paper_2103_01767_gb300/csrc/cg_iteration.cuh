// cg_iteration.cuh -- one iteration of the truncated (P)CG of Algorithm 1 (arXiv 2103.01767,
// Sec. 4.2; Jacobi preconditioner of Sec. 3.3) after its GGN product, as a single
// cooperative launch:
//
//   alpha = r.z / p.q;  x += alpha p;  r -= alpha q;  z = r / ((1 + lambda) D);
//   beta = r.z(new) / r.z;  p = z + beta p;  q = lambda D p
//
// (q = (G + lambda D) p on entry; D == NULL means D = I and z = r).  The three phases run
// over the same grid-stride elements per thread, in the three-launch form's order and
// arithmetic; the vectors (8 bytes per element each) stay in L2 between the phases, so the
// re-reads of p, q, r and D cost little HBM traffic, and the iteration pays one launch
// instead of three.  The FP64 reductions are those of
// grid_reduce: per-CTA partials summed in block order by the CTA whose arrival completes
// the round, which then updates the scalar slots exactly as OP_ALPHA / OP_BETA do and
// releases the round.
//
// With tol >= 0 the CTA that finishes the second reduction also counts the iteration
// (S_CG_ITERS) and sets S_CG_DONE once ||r|| <= tol; a launch that finds S_CG_DONE set
// returns at once, as does the GGN product given the same flag, so the host can queue
// several iterations between two reads of the scalars.
//
// Waits: the launch is cooperative (every CTA resident), and each wait is additionally
// bounded; a wait that gives up sets S_CG_TIMEOUT and carries on, so no launch can hang.
// The last CTA to leave resets the counters (arrivals cnt[0], exits cnt[1], released round
// cnt[kCoopRelease]) for the next launch.
#pragma once
#include <cuda_runtime.h>

#include "reduce.cuh"

namespace ptylm {

__device__ __forceinline__ float rdotf(float2 a, float2 b) { return a.x * b.x + a.y * b.y; }

// Jacobi preconditioner z = r / Dg(G + lambda D) = r / ((1 + lambda) D), D = Dg(G)
// (Sec. 3.3); the identity when D is NULL.
__device__ __forceinline__ float2 precondition(float2 r, const float* D, float lambda, long i) {
    if (!D) return r;
    const float inv = 1.0f / ((1.0f + lambda) * D[i]);
    return make_float2(r.x * inv, r.y * inv);
}

constexpr unsigned kCoopSpinLimit = 1u << 24;   // x >= 32 ns sleep: about a second (the default limit)

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_gpu(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned atom_add_acq_rel_gpu(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// FP64 sum of W per-thread values over the grid into the slots (`op`), then a grid-wide
// barrier: on return every CTA may read the updated slots.  Round j of a launch (1, 2)
// completes when cnt[0] reaches j * gridDim.x; cnt[kCoopRelease] (its own 128-byte line,
// so the pollers do not contend with the arrivals) holds the last released round.  The
// arrival is an acquire-release add (it publishes the CTA's partial and, for the last CTA,
// makes every partial visible); the release is a release store read by acquire loads.
template <int W>
__device__ void coop_reduce_round(double (&s)[W], double* part, unsigned* cnt, double* sc, int op, unsigned round,
                                  unsigned spin_limit, double tol = -1.0) {
    __shared__ bool is_last;
    block_sum<W>(s);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int c = 0; c < W; ++c) part[blockIdx.x * W + c] = s[c];
        const unsigned prev = atom_add_acq_rel_gpu(cnt, 1u);
        is_last = (prev == round * gridDim.x - 1);
    }
    __syncthreads();
    if (is_last) {
        double t[W];
#pragma unroll
        for (int c = 0; c < W; ++c) t[c] = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
#pragma unroll
            for (int c = 0; c < W; ++c) t[c] += __ldcg(part + b * W + c);
        block_sum<W>(t);
        if (threadIdx.x == 0) {
            apply_final_op(t, W, sc, 0, op);
            if (tol >= 0.0) {  // the CG stopping test ||r|| <= tol, taken on the device
                sc[S_CG_ITERS] += 1.0;
                sc[S_CG_DONE] = sqrt(sc[S_RR]) <= tol ? 1.0 : 0.0;
            }
            st_release_gpu(cnt + kCoopRelease, round);
        }
    } else if (threadIdx.x == 0) {
        unsigned spins = 0;
        while (ld_acquire_gpu(cnt + kCoopRelease) < round) {
            if (++spins > spin_limit) {
                *(volatile double*)(sc + S_CG_TIMEOUT) = 1.0;
                break;
            }
            __nanosleep(32);
        }
    }
    __syncthreads();
}

// Elements a thread loads before it uses any of them (HBM needs several MB in flight).
constexpr int kCgUnroll = 2;

__global__ void __launch_bounds__(256) k_cg_iteration(float2* __restrict__ x, float2* __restrict__ r,
                                                      float2* __restrict__ p, float2* __restrict__ q,
                                                      const float* __restrict__ D, float lambda, long n,
                                                      double* part, unsigned* cnt, double* sc, double tol,
                                                      unsigned spin_limit) {
    constexpr int U = kCgUnroll;
    if (tol >= 0.0 && __ldcg(sc + S_CG_DONE) != 0.0) return;  // converged earlier: every CTA sees the same flag
    const long stride = (long)gridDim.x * blockDim.x;
    const long i0 = blockIdx.x * (long)blockDim.x + threadIdx.x;

    // p.q -> alpha
    float f = 0.0f;
    for (long base = i0; base < n; base += U * stride) {
        float2 pv[U], qv[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const long i = base + k * stride;
            pv[k] = qv[k] = make_float2(0.0f, 0.0f);
            if (i < n) {
                pv[k] = p[i];
                qv[k] = q[i];
            }
        }
#pragma unroll
        for (int k = 0; k < U; ++k)
            if (base + k * stride < n) f += rdotf(pv[k], qv[k]);
    }
    double s1[1] = {f};
    coop_reduce_round<1>(s1, part, cnt, sc, OP_ALPHA, 1u, spin_limit);
    const float alpha = (float)__ldcg(sc + S_ALPHA);

    // x += alpha p, r -= alpha q; r.z and r.r -> beta
    float f0 = 0.0f, f1 = 0.0f;
    for (long base = i0; base < n; base += U * stride) {
        float2 pv[U], qv[U], xv[U], rv[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const long i = base + k * stride;
            pv[k] = qv[k] = xv[k] = rv[k] = make_float2(0.0f, 0.0f);
            if (i < n) {
                pv[k] = p[i];
                qv[k] = q[i];
                xv[k] = x[i];
                rv[k] = r[i];
            }
        }
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const long i = base + k * stride;
            if (i < n) {
                float2 xi = xv[k], ri = rv[k];
                xi.x += alpha * pv[k].x;
                xi.y += alpha * pv[k].y;
                ri.x -= alpha * qv[k].x;
                ri.y -= alpha * qv[k].y;
                x[i] = xi;
                r[i] = ri;
                f0 += rdotf(ri, precondition(ri, D, lambda, i));
                f1 += rdotf(ri, ri);
            }
        }
    }
    double s2[2] = {f0, f1};
    coop_reduce_round<2>(s2, part + gridDim.x, cnt, sc, OP_BETA, 2u, spin_limit, tol);
    const float beta = (float)__ldcg(sc + S_BETA);

    // p = z + beta p, q = lambda D p
    for (long base = i0; base < n; base += U * stride) {
        float2 rv[U], pv[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const long i = base + k * stride;
            rv[k] = pv[k] = make_float2(0.0f, 0.0f);
            if (i < n) {
                rv[k] = r[i];
                pv[k] = p[i];
            }
        }
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const long i = base + k * stride;
            if (i < n) {
                const float2 zi = precondition(rv[k], D, lambda, i);
                const float2 pn = make_float2(zi.x + beta * pv[k].x, zi.y + beta * pv[k].y);
                p[i] = pn;
                const float d = lambda * (D ? D[i] : 1.0f);
                q[i] = make_float2(d * pn.x, d * pn.y);
            }
        }
    }
    if (threadIdx.x == 0 && atomicAdd(cnt + 1, 1u) == gridDim.x - 1) {
        // every CTA has passed both rounds: nobody reads the counters any more
        cnt[0] = 0u;
        cnt[kCoopRelease] = 0u;
        cnt[1] = 0u;
        __threadfence();
    }
}

}  // namespace ptylm
