// reduce.cuh -- FP64 grid reductions finished by the last CTA, and the device scalar slots
// of the truncated CG / LM driver (Algorithm 1 of arXiv 2103.01767).
//
// Every CTA block-sums its per-thread values in FP64 and stores one partial per column;
// after a __threadfence it bumps a counter, and the CTA that sees the count reach gridDim.x
// sums all partials in block order (deterministic), applies a scalar update to the FP64
// slots and resets the counter.  Nothing waits on another CTA, so no launch can hang.
#pragma once
#include <cuda_runtime.h>

namespace ptylm {

// FP64 scalar slots on the device.
enum Slot {
    S_F = 0, S_DL2 = 1,                 // forward: f, ||grad_zeta l||^2
    S_RR = 2, S_PAP = 3, S_ALPHA = 4, S_RRNEW = 5, S_BETA = 6,
    S_GG = 7,                           // ||grad f||^2
    S_DD = 8, S_DG = 9, S_DR = 10,      // step dots for the predicted reduction
    S_ER = 11, S_EI = 12, S_NO = 13, S_NR = 14,  // object-error sums
    S_RZ = 15,                          // r.z of the preconditioned CG (= r.r without preconditioner)
    S_GS = 16, S_SS = 17,               // Algorithm 2: g.s and ||s||^2
    S_FMIN = 18,                        // Poisson: sum y - y log y
    S_CG_TIMEOUT = 19,                  // set when a wait of the single-launch CG iteration gave up
    S_CG_DONE = 20, S_CG_ITERS = 21,    // device-side CG stopping: converged flag, iterations run
    S_COUNT = 24
};

// What the last CTA does with the column sums c[] (scaled by `scale`).
enum FinalOp {
    OP_STORE = 0,   // sc[dst + i] = c[i]
    OP_ALPHA = 1,   // p.Ap = c[0];  alpha = r.z / p.Ap
    OP_BETA = 2,    // beta = c[0] / r.z;  r.z = c[0];  r.r = c[1]
    OP_START = 3    // r.z = c[0];  r.r = c[1]   (CG start)
};

// Counters, one per reduction site (kernels on one stream never overlap).
// From CNT_COOP: arrivals and exits of the single-launch CG iteration, and 32 words (one
// 128-byte line) further its released round (cg_iteration.cuh).
// CNT_YBAD: flag set by the measurement copy when an entry of y is negative or not finite.
enum Counter { CNT_FWD = 0, CNT_VEC = 1, CNT_YBAD = 2, CNT_COOP = 32, CNT_COUNT = 96 };
constexpr int kCoopRelease = 32;

constexpr int kMaxReduceWidth = 4;

template <int W>
__device__ __forceinline__ void warp_sum(double (&s)[W]) {
#pragma unroll
    for (int c = 0; c < W; ++c)
        for (int off = 16; off > 0; off >>= 1) s[c] += __shfl_down_sync(0xffffffffu, s[c], off);
}

// Sum of W per-thread FP64 values over the CTA (blockDim a multiple of 32, <= 1024);
// thread 0 receives the result.
template <int W>
__device__ __forceinline__ void block_sum(double (&s)[W]) {
    __shared__ double red[W][32];
    warp_sum<W>(s);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < W; ++c) red[c][warp] = s[c];
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int c = 0; c < W; ++c) s[c] = lane < nw ? red[c][lane] : 0.0;
        warp_sum<W>(s);
    }
    __syncthreads();
}

__device__ __forceinline__ void apply_final_op(const double* c, int W, double* sc, int dst, int op) {
    switch (op) {
        case OP_STORE:
            for (int i = 0; i < W; ++i) sc[dst + i] = c[i];
            break;
        case OP_ALPHA:
            sc[S_PAP] = c[0];
            sc[S_ALPHA] = sc[S_RZ] / c[0];
            break;
        case OP_BETA:
            sc[S_RRNEW] = c[1];
            sc[S_BETA] = c[0] / sc[S_RZ];
            sc[S_RZ] = c[0];
            sc[S_RR] = c[1];
            break;
        case OP_START:
            sc[S_RZ] = c[0];
            sc[S_RR] = c[1];
            break;
    }
}

// Grid-wide FP64 reduction of W per-thread values finished by the last CTA (see header).
// part: [gridDim.x][W] scratch; counter: zero on entry, zero again on exit; sc: slots.
// Every thread of every CTA must call it exactly once.
template <int W>
__device__ void grid_reduce(double (&s)[W], double* part, unsigned* counter, double* sc, int dst, int op,
                            double scale) {
    __shared__ bool is_last;
    block_sum<W>(s);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int c = 0; c < W; ++c) part[blockIdx.x * W + c] = s[c];
        __threadfence();
        const unsigned prev = atomicAdd(counter, 1u);
        is_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double t[W];
#pragma unroll
    for (int c = 0; c < W; ++c) t[c] = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
#pragma unroll
        for (int c = 0; c < W; ++c) t[c] += __ldcg(part + b * W + c);
    block_sum<W>(t);
    if (threadIdx.x == 0) {
        double cs[W];
#pragma unroll
        for (int c = 0; c < W; ++c) cs[c] = t[c] * scale;
        apply_final_op(cs, W, sc, dst, op);
        *counter = 0u;
        __threadfence();
    }
}

}  // namespace ptylm
