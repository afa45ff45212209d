// ptylm_abi.cu -- C-ABI entry points (include/ptylm.h), context management, the CG and
// LM vector kernels with FP64 reductions, and the truncated LM driver (Algorithm 1 of
// arXiv 2103.01767, Sec. 4.2).
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <chrono>
#include <optional>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ptylm.h"
#include "kernels.h"
#include "cg_iteration.cuh"
#include "reduce.cuh"

using namespace ptylm;

// ---------------------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------------------
static thread_local std::string g_last_error;

static ptylm_status fail(ptylm_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

void ptylm::set_last_error(const char* msg) { g_last_error = msg; }

#define CUDA_TRY(expr)                                                                     \
    do {                                                                                   \
        cudaError_t e_ = (expr);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(PTYLM_ERR_CUDA, "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                               \
    } while (0)

#define STATUS_TRY(expr)                      \
    do {                                      \
        ptylm_status s_ = (expr);             \
        if (s_ != PTYLM_OK) return s_;        \
    } while (0)

// ---------------------------------------------------------------------------------------
// Vector kernels of the truncated (P)CG and of Algorithms 1 and 2.  Vectors run over the
// state z (the object, then the probe for joint contexts).  Products are formed in FP32
// and summed per thread over its few grid-stride elements, then reduced in FP64 by
// grid_reduce (reduce.cuh), whose last CTA also updates the FP64 scalars (alpha, beta, r.z,
// r.r): a CG iteration is the matvec plus three launches, with no host round trip (or the
// matvec plus one cooperative launch, k_cg_iteration in cg_iteration.cuh).
// Jacobi preconditioner (Sec. 3.3): z = r / Dg(G + lambda D) = r / ((1 + lambda) D) when
// D = Dg(G); no preconditioner (z = r) when D is NULL (rdotf and precondition live in
// cg_iteration.cuh, shared with the single-launch iteration).
// ---------------------------------------------------------------------------------------
static constexpr int VEC_THREADS = 256;

#define GRID_STRIDE(i, n) \
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < (n); i += (long)gridDim.x * blockDim.x)

// out = lambda * D * v   (D == NULL: identity).  Initialises the matvec accumulator.
__global__ void k_damping_init(const float2* __restrict__ v, const float* __restrict__ D, float lambda,
                               float2* __restrict__ out, long n) {
    GRID_STRIDE(i, n) {
        const float d = lambda * (D ? D[i] : 1.0f);
        const float2 x = v[i];
        out[i] = make_float2(d * x.x, d * x.y);
    }
}

// Up to three real-coordinate dot products a_i . b_i (the first optionally weighted by
// w0, i.e. a0^T diag(w0) b0) into slots [dst, dst + W), then `op`.
template <int W>
__global__ void k_dots(const float2* __restrict__ a0, const float2* __restrict__ b0, const float* __restrict__ w0,
                       const float2* __restrict__ a1, const float2* __restrict__ b1,
                       const float2* __restrict__ a2, const float2* __restrict__ b2, long n,
                       double* part, unsigned* counter, double* sc, int dst, int op) {
    float f[W];
#pragma unroll
    for (int c = 0; c < W; ++c) f[c] = 0.0f;
    GRID_STRIDE(i, n) {
        f[0] += (w0 ? w0[i] : 1.0f) * rdotf(a0[i], b0[i]);
        if constexpr (W > 1) f[1] += rdotf(a1[i], b1[i]);
        if constexpr (W > 2) f[2] += rdotf(a2[i], b2[i]);
    }
    double s[W];
#pragma unroll
    for (int c = 0; c < W; ++c) s[c] = f[c];
    grid_reduce<W>(s, part, counter, sc, dst, op, 1.0);
}

// CG start: r = -g - q, z = precond(r), p = z, q = lambda D p; r.z and r.r into the slots.
__global__ void k_cg_start(const float2* __restrict__ g, float2* __restrict__ q, float2* __restrict__ r,
                           float2* __restrict__ p, const float* __restrict__ D, float lambda, long n, double* part,
                           unsigned* counter, double* sc) {
    float f0 = 0.0f, f1 = 0.0f;
    GRID_STRIDE(i, n) {
        const float2 gi = g[i], qi = q[i];
        const float2 ri = make_float2(-gi.x - qi.x, -gi.y - qi.y);
        const float2 zi = precondition(ri, D, lambda, i);
        r[i] = ri;
        p[i] = zi;
        const float d = lambda * (D ? D[i] : 1.0f);
        q[i] = make_float2(d * zi.x, d * zi.y);
        f0 += rdotf(ri, zi);
        f1 += rdotf(ri, ri);
    }
    double s[2] = {f0, f1};
    grid_reduce<2>(s, part, counter, sc, 0, OP_START, 1.0);
}

// The stopping test before the first CG iteration, taken on the device: S_CG_DONE =
// (||r0|| <= tol), S_CG_ITERS = 0 (one thread).
__global__ void k_cg_check(double* sc, double tol) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        sc[S_CG_DONE] = sqrt(sc[S_RR]) <= tol ? 1.0 : 0.0;
        sc[S_CG_ITERS] = 0.0;
    }
}

// x += alpha p, r -= alpha q; new r.z and r.r -> beta (alpha read from the slots).
__global__ void k_cg_update(float2* __restrict__ x, float2* __restrict__ r, const float2* __restrict__ p,
                            const float2* __restrict__ q, const float* __restrict__ D, float lambda, long n,
                            double* part, unsigned* counter, double* sc) {
    const float alpha = (float)sc[S_ALPHA];
    float f0 = 0.0f, f1 = 0.0f;
    GRID_STRIDE(i, n) {
        const float2 pi = p[i], qi = q[i];
        float2 xi = x[i], ri = r[i];
        xi.x += alpha * pi.x;
        xi.y += alpha * pi.y;
        ri.x -= alpha * qi.x;
        ri.y -= alpha * qi.y;
        x[i] = xi;
        r[i] = ri;
        f0 += rdotf(ri, precondition(ri, D, lambda, i));
        f1 += rdotf(ri, ri);
    }
    double s[2] = {f0, f1};
    grid_reduce<2>(s, part, counter, sc, 0, OP_BETA, 1.0);
}

// p = precond(r) + beta p;  q = lambda D p (starts the next matvec's accumulator).
__global__ void k_cg_direction(const float2* __restrict__ r, float2* __restrict__ p, float2* __restrict__ q,
                               const float* __restrict__ D, float lambda, long n, const double* __restrict__ sc) {
    const float beta = (float)sc[S_BETA];
    GRID_STRIDE(i, n) {
        const float2 zi = precondition(r[i], D, lambda, i), pi = p[i];
        const float2 pn = make_float2(zi.x + beta * pi.x, zi.y + beta * pi.y);
        p[i] = pn;
        const float d = lambda * (D ? D[i] : 1.0f);
        q[i] = make_float2(d * pn.x, d * pn.y);
    }
}

// z = x + alpha d
__global__ void k_axpy(const float2* __restrict__ x, const float2* __restrict__ d, float alpha,
                       float2* __restrict__ z, long n) {
    GRID_STRIDE(i, n) {
        const float2 a = x[i], b = d[i];
        z[i] = make_float2(a.x + alpha * b.x, a.y + alpha * b.y);
    }
}

// Radial projection onto |z_i| <= radius (Eq. constraints): object part [0, N), probe part
// [N, n) with its own radius (Sec. 4.3: the constraint sets are separable).
__global__ void k_project(float2* __restrict__ z, long N, long n, float rO, float rP) {
    GRID_STRIDE(i, n) {
        const float r = i < N ? rO : rP;
        const float2 v = z[i];
        const float a2 = v.x * v.x + v.y * v.y;
        if (a2 > r * r) {
            const float s = r * rsqrtf(a2);
            z[i] = make_float2(v.x * s, v.y * s);
        }
    }
}

// Poisson: sum over measurements of y - y log y (the metric's value where h = y).
__global__ void k_poisson_fmin(const float* __restrict__ y, long n, double* part, unsigned* counter, double* sc) {
    float f = 0.0f;
    GRID_STRIDE(i, n) {
        const float v = y[i];
        f += v - (v > 0.0f ? v * logf(v) : 0.0f);
    }
    double s[1] = {f};
    grid_reduce<1>(s, part, counter, sc, S_FMIN, OP_STORE, 1.0);
}

// Probe block of an adjoint: out[m] (+)= sum over team slots of part[slot][m], slots in order.
__global__ void k_probe_reduce(const float2* __restrict__ part, int slots, int M, float2* __restrict__ out,
                               int accumulate) {
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x) {
        float2 acc = accumulate ? out[m] : make_float2(0.0f, 0.0f);
        for (int s = 0; s < slots; ++s) {
            const float2 v = part[(size_t)s * M + m];
            acc.x += v.x;
            acc.y += v.y;
        }
        out[m] = acc;
    }
}

// Per-block maxima of a non-negative array (first pass of the diagonal floor).
__global__ void k_block_max(const float* __restrict__ D, long n, double* part) {
    __shared__ float red[VEC_THREADS];
    float m = 0.0f;
    GRID_STRIDE(i, n) m = fmaxf(m, D[i]);
    red[threadIdx.x] = m;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + h]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// D = max(D, floor_rel * max D) (the maximum re-derived by every block from the partials).
__global__ void k_apply_floor(float* __restrict__ D, long n, const double* __restrict__ part, int nparts,
                              float floor_rel) {
    __shared__ float fl;
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int b = 0; b < nparts; ++b) m = fmax(m, part[b]);
        fl = (float)(floor_rel * m);
    }
    __syncthreads();
    GRID_STRIDE(i, n) D[i] = fmaxf(D[i], fl);
}

// Object-error sums over a mask: <O, O_ref> (re, im), ||O||^2, ||O_ref||^2.
__global__ void k_err_sums(const float2* __restrict__ O, const float2* __restrict__ R,
                           const uint8_t* __restrict__ mask, long n, double* part, unsigned* counter,
                           double* sc) {
    float f[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    GRID_STRIDE(i, n) {
        if (mask && !mask[i]) continue;
        const float2 o = O[i], r = R[i];
        f[0] += o.x * r.x + o.y * r.y;   // Re conj(O) R
        f[1] += o.x * r.y - o.y * r.x;   // Im conj(O) R
        f[2] += o.x * o.x + o.y * o.y;
        f[3] += r.x * r.x + r.y * r.y;
    }
    double s[4] = {f[0], f[1], f[2], f[3]};
    grid_reduce<4>(s, part, counter, sc, S_ER, OP_STORE, 1.0);
}

// ---------------------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------------------
// Timed sections: the per-position kernels (KernelId), then the CG iteration's vector work.
static constexpr int PROF_CG = KID_COUNT, PROF_COUNT = KID_COUNT + 1;
static_assert(PROF_CG == PTYLM_KERNEL_CG_ITERATION, "profile ids follow the kernel ids");

struct ptylm_ctx {
    ptylm_desc d;
    unsigned cg_spin_limit = kCoopSpinLimit;  // polls per bounded wait of the CG iteration
    int LS = 0, LE = 5, S = 0, M = 0;   // FFT tile: side 2^LS, 2^LE values per thread
    long N = 0;
    long L = 0;                    // length of the state z: N, or N + M for joint contexts
    cudaStream_t stream = nullptr;
    int device = 0, num_sms = 0;
    int grid[KID_COUNT] = {0};
    int vec_grid = 0;
    int coop_grid = 0;             // grid of the single-launch CG iteration (0: three launches)
    int cg_chunk = 1;              // CG iterations the last solve took (the next solve queues as many at once)
    size_t allocated = 0;
    std::vector<void*> allocations;

    int2* pos = nullptr;
    float* y_perm = nullptr;       // measurements in the kernels' team-register order
    float2* tw = nullptr;
    float2* a_cache = nullptr;
    float2* grad = nullptr;
    float2* O_lin = nullptr;
    float2* P_lin = nullptr;
    double* partials = nullptr;
    int partials_cap = 0;
    unsigned* counters = nullptr;  // grid_reduce counters [CNT_COUNT]
    double* scal = nullptr;        // device FP64 scalars [S_COUNT]
    double* scal_host = nullptr;   // pinned mirror
    float2* jvp_scratch = nullptr;
    float2* probe_part = nullptr;  // joint: per-team probe accumulators [probe_slots][M]
    int probe_slots = 0;
    float* trp = nullptr;          // per-thread d2l sums of the last linearisation [K][T]
    // Look-ahead linearisation (object-only lm_solve): the trial point's forward pass also
    // fills this second set; when the step is accepted the sets swap, so the next outer
    // iteration starts without a forward pass of its own.
    float2 *a_cache_b = nullptr, *grad_b = nullptr, *O_lin_b = nullptr;
    float* trp_b = nullptr;
    bool lookahead_failed = false; // the second set did not fit the workspace budget
    float* tr = nullptr;           // per-position d2l sums [K]
    float2* u_cache = nullptr;     // unit phasor psihat / zeta at the point [K][M] (team order)
    bool u_valid = false;          // u_cache holds the phasor of the current point
    bool has_point = false;        // O_lin / P_lin hold a point (jvp, jtvp)
    bool has_lin = false;          // ... and the loss cache, gradient and d2l sums match it
    double f_lin = 0.0, dl2_lin = 0.0;
    float b_eff = 0.0f;            // background the kernels use: b, plus s_t inside lm_solve

    // CG / LM vectors over z (allocated on first use)
    float2 *cg_x = nullptr, *cg_r = nullptr, *cg_p = nullptr, *cg_q = nullptr, *trial = nullptr;
    float2* ls_dir = nullptr;      // Algorithm 2 search direction
    float* Dg = nullptr;           // scaling D = Dg(G) over z
    // staging for host pointers
    float2 *stage_a = nullptr, *stage_b = nullptr, *stage_P = nullptr;

    // instrumentation
    long long launches = 0;
    unsigned prof_mask = 0;        // bit k: time the launches of section k (kernel id, or PROF_CG)
    struct Rec { int kid; cudaEvent_t a, b; };
    std::vector<cudaEvent_t> ev_free;
    std::vector<Rec> recs;
    double prof_ms[PROF_COUNT] = {0};
    long long prof_n[PROF_COUNT] = {0};
};

// Accumulate the elapsed time of every recorded launch (synchronises the stream).
static ptylm_status prof_flush(ptylm_ctx* c) {
    if (c->recs.empty()) return PTYLM_OK;
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    for (auto& r : c->recs) {
        float ms = 0.0f;
        CUDA_TRY(cudaEventElapsedTime(&ms, r.a, r.b));
        c->prof_ms[r.kid] += ms;
        c->prof_n[r.kid] += 1;
        c->ev_free.push_back(r.a);
        c->ev_free.push_back(r.b);
    }
    c->recs.clear();
    return PTYLM_OK;
}

static ptylm_status take_event(ptylm_ctx* c, cudaEvent_t* e) {
    if (c->ev_free.empty()) {
        CUDA_TRY(cudaEventCreate(e));
        return PTYLM_OK;
    }
    *e = c->ev_free.back();
    c->ev_free.pop_back();
    return PTYLM_OK;
}

bool ptylm::ctx_view(const ptylm_ctx* c, CtxView* v) {
    if (!c || !v) return false;
    v->y_team = c->y_perm;
    v->pos = c->pos;
    v->tw = c->tw;
    v->K = c->d.K;
    v->ny = c->d.ny;
    v->nx = c->d.nx;
    v->m = c->S;
    v->loss = c->d.loss;
    v->num_sms = c->num_sms;
    v->stream = c->stream;
    return true;
}

// Events around a timed section when profiling covers it (no-ops otherwise).
static bool prof_wants(const ptylm_ctx* c, int id) { return (c->prof_mask >> id) & 1u; }

static ptylm_status prof_begin(ptylm_ctx* c, int id, cudaEvent_t* e0, cudaEvent_t* e1) {
    if (!prof_wants(c, id)) return PTYLM_OK;
    if (c->recs.size() >= 2048) STATUS_TRY(prof_flush(c));
    STATUS_TRY(take_event(c, e0));
    STATUS_TRY(take_event(c, e1));
    CUDA_TRY(cudaEventRecord(*e0, c->stream));
    return PTYLM_OK;
}

static ptylm_status prof_end(ptylm_ctx* c, int id, cudaEvent_t e0, cudaEvent_t e1) {
    if (!prof_wants(c, id)) return PTYLM_OK;
    CUDA_TRY(cudaEventRecord(e1, c->stream));
    c->recs.push_back({id, e0, e1});
    return PTYLM_OK;
}

// Launch a per-position kernel, timing it with events when profiling is on.
static ptylm_status launch(ptylm_ctx* c, int kid, const PtyArgs& a) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    STATUS_TRY(prof_begin(c, kid, &e0, &e1));
    CUDA_TRY(kernel_launch(c->LS, c->LE, kid, a, c->grid[kid], c->stream));
    ++c->launches;
    return prof_end(c, kid, e0, e1);
}

// Count a vector-kernel launch and check it was accepted.
static ptylm_status vec_launched(ptylm_ctx* c) {
    ++c->launches;
    CUDA_TRY(cudaGetLastError());
    return PTYLM_OK;
}

static ptylm_status ctx_alloc(ptylm_ctx* c, void** p, size_t bytes, const char* what) {
    if (c->d.workspace_budget && c->allocated + bytes > c->d.workspace_budget)
        return fail(PTYLM_ERR_NOMEM, "workspace budget %zu bytes exceeded allocating %s (%zu bytes, %zu in use)",
                    c->d.workspace_budget, what, bytes, c->allocated);
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(PTYLM_ERR_NOMEM, "cudaMalloc(%zu) for %s failed: %s", bytes, what, cudaGetErrorString(e));
    }
    c->allocated += bytes;
    c->allocations.push_back(*p);
    return PTYLM_OK;
}

template <class T>
static ptylm_status ctx_alloc_t(ptylm_ctx* c, T** p, size_t count, const char* what) {
    void* q = nullptr;
    ptylm_status s = ctx_alloc(c, &q, count * sizeof(T), what);
    *p = static_cast<T*>(q);
    return s;
}

static void ctx_free_all(ptylm_ctx* c) {
    for (auto& r : c->recs) {
        c->ev_free.push_back(r.a);
        c->ev_free.push_back(r.b);
    }
    c->recs.clear();
    for (cudaEvent_t e : c->ev_free) cudaEventDestroy(e);
    c->ev_free.clear();
    for (void* p : c->allocations) cudaFree(p);
    c->allocations.clear();
    if (c->scal_host) cudaFreeHost(c->scal_host);
    c->scal_host = nullptr;
}

static bool is_host_pointer(const void* p) {
    if (!p) return false;
    cudaPointerAttributes attr;
    cudaError_t e = cudaPointerGetAttributes(&attr, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return attr.type == cudaMemoryTypeHost || attr.type == cudaMemoryTypeUnregistered;
}

static int vec_blocks(const ptylm_ctx* c) { return c->vec_grid; }

static ptylm_status read_scalars(ptylm_ctx* c, int first, int count) {
    CUDA_TRY(cudaMemcpyAsync(c->scal_host + first, c->scal + first, sizeof(double) * count,
                             cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return PTYLM_OK;
}

// Dot products over n elements (the first optionally weighted) into slots [dst, dst + W).
static ptylm_status dots(ptylm_ctx* c, int W, long n, const float2* a0, const float2* b0, const float* w0,
                         const float2* a1, const float2* b1, const float2* a2, const float2* b2, int dst,
                         int op = OP_STORE) {
    const int nb = vec_blocks(c);
    unsigned* cnt = c->counters + CNT_VEC;
    double* part = c->partials;
    if (W == 1) k_dots<1><<<nb, VEC_THREADS, 0, c->stream>>>(a0, b0, w0, a1, b1, a2, b2, n, part, cnt, c->scal, dst, op);
    else if (W == 2) k_dots<2><<<nb, VEC_THREADS, 0, c->stream>>>(a0, b0, w0, a1, b1, a2, b2, n, part, cnt, c->scal, dst, op);
    else k_dots<3><<<nb, VEC_THREADS, 0, c->stream>>>(a0, b0, w0, a1, b1, a2, b2, n, part, cnt, c->scal, dst, op);
    return vec_launched(c);
}

static PtyArgs base_args(const ptylm_ctx* c) {
    PtyArgs a;
    memset(&a, 0, sizeof a);
    a.pos = c->pos;
    a.y = c->y_perm;
    a.tw = c->tw;
    a.K = c->d.K;
    a.nx = c->d.nx;
    a.b = c->b_eff;
    a.loss = c->d.loss;
    a.partials = c->partials;
    a.scal = c->scal;
    a.outP_part = c->probe_part;
    return a;
}

static bool joint(const ptylm_ctx* c) { return c->d.joint != 0; }

// Sum the probe accumulators of `kid`'s teams into out [M] (overwrite or add).
static ptylm_status probe_reduce(ptylm_ctx* c, int kid, float2* out, bool accumulate) {
    const int slots = c->grid[kid] * cta_teams(c->LS, c->LE);
    k_probe_reduce<<<(c->M + VEC_THREADS - 1) / VEC_THREADS, VEC_THREADS, 0, c->stream>>>(c->probe_part, slots, c->M,
                                                                                        out, accumulate ? 1 : 0);
    return vec_launched(c);
}

static ptylm_status clear_probe_part(ptylm_ctx* c, int kid) {
    const size_t slots = (size_t)c->grid[kid] * cta_teams(c->LS, c->LE);
    CUDA_TRY(cudaMemsetAsync(c->probe_part, 0, sizeof(float2) * slots * c->M, c->stream));
    return PTYLM_OK;
}

// ---------------------------------------------------------------------------------------
// Internal operations on device pointers
// ---------------------------------------------------------------------------------------

// Forward model + loss; cache=1 also stores a, the linearisation point, the per-thread d2l
// sums and grad f over z (object part by scatter, probe part by team accumulators).
static ptylm_status op_forward(ptylm_ctx* c, const float2* O, const float2* P, int cache) {
    const int kid = cache ? (joint(c) ? KID_FWD_CACHE_J : KID_FWD_CACHE) : KID_FWD_LOSS;
    if (cache) {
        if (O != c->O_lin) CUDA_TRY(cudaMemcpyAsync(c->O_lin, O, sizeof(float2) * c->N, cudaMemcpyDeviceToDevice, c->stream));
        if (P != c->P_lin) CUDA_TRY(cudaMemcpyAsync(c->P_lin, P, sizeof(float2) * c->M, cudaMemcpyDeviceToDevice, c->stream));
        CUDA_TRY(cudaMemsetAsync(c->grad, 0, sizeof(float2) * c->L, c->stream));
        if (joint(c)) STATUS_TRY(clear_probe_part(c, kid));
        c->has_lin = false;
        c->u_valid = false;
    }
    if (c->d.K == 0) {
        CUDA_TRY(cudaMemsetAsync(c->scal + S_F, 0, 2 * sizeof(double), c->stream));
    } else {
        PtyArgs a = base_args(c);
        a.O = cache ? c->O_lin : O;
        a.P = cache ? c->P_lin : P;
        a.a_cache = c->a_cache;
        a.out = c->grad;
        a.counter = c->counters + CNT_FWD;
        a.trp = cache ? c->trp : nullptr;
        STATUS_TRY(launch(c, kid, a));
        if (cache && joint(c)) STATUS_TRY(probe_reduce(c, kid, c->grad + c->N, false));
    }
    if (cache) c->has_lin = c->has_point = true;
    return PTYLM_OK;
}

// One CG iteration after q = (G + lambda D) p: alpha, x, r, beta, p and q = lambda D p
// (the next product's damping term), as one cooperative launch or as three launches.  With
// tol >= 0 (cooperative form only) the device applies the stopping test ||r|| <= tol itself
// (S_CG_DONE, S_CG_ITERS) and the iteration is a no-op once it has passed.
static ptylm_status cg_iteration(ptylm_ctx* c, float2* x, float2* r, float2* p, float2* q, const float* D,
                                 float lambda, bool separate, double tol = -1.0) {
    long n = c->L;
    double* part = c->partials;
    double* sc = c->scal;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    STATUS_TRY(prof_begin(c, PROF_CG, &e0, &e1));
    if (!separate && c->coop_grid > 0) {
        unsigned* cnt = c->counters + CNT_COOP;
        unsigned spin = c->cg_spin_limit;
        void* args[] = {&x, &r, &p, &q, &D, &lambda, &n, &part, &cnt, &sc, &tol, &spin};
        CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_cg_iteration, dim3(c->coop_grid), dim3(VEC_THREADS), args, 0,
                                             c->stream));
        ++c->launches;
    } else {
        STATUS_TRY(dots(c, 1, n, p, q, nullptr, nullptr, nullptr, nullptr, nullptr, S_PAP, OP_ALPHA));
        const int nb = vec_blocks(c);
        k_cg_update<<<nb, VEC_THREADS, 0, c->stream>>>(x, r, p, q, D, lambda, n, part, c->counters + CNT_VEC, sc);
        STATUS_TRY(vec_launched(c));                                      // x, r; beta
        k_cg_direction<<<nb, VEC_THREADS, 0, c->stream>>>(r, p, q, D, lambda, n, sc);
        STATUS_TRY(vec_launched(c));                                      // p, q = lambda D p
    }
    return prof_end(c, PROF_CG, e0, e1);
}

// Forward pass with cache and gradient at `O` (object-only contexts; the probe is the one of
// the current linearisation) into the look-ahead set; the error metric and ||grad l||^2
// land in the scalar slots as for any forward pass.
static ptylm_status op_forward_lookahead(ptylm_ctx* c, const float2* O) {
    CUDA_TRY(cudaMemcpyAsync(c->O_lin_b, O, sizeof(float2) * c->N, cudaMemcpyDeviceToDevice, c->stream));
    CUDA_TRY(cudaMemsetAsync(c->grad_b, 0, sizeof(float2) * c->L, c->stream));
    PtyArgs a = base_args(c);
    a.O = c->O_lin_b;
    a.P = c->P_lin;
    a.a_cache = c->a_cache_b;
    a.out = c->grad_b;
    a.counter = c->counters + CNT_FWD;
    a.trp = c->trp_b;
    return launch(c, KID_FWD_CACHE, a);
}

// Allocate the look-ahead set once, after everything lm_solve needs; false (and no error)
// when the workspace budget has no room for the whole set (then nothing of it is taken) or
// the device runs out midway, in which case the context never asks again.
static bool lookahead_set(ptylm_ctx* c) {
    if (c->trp_b) return true;
    if (c->lookahead_failed) return false;
    const size_t need = sizeof(float2) * ((size_t)c->d.K * c->M + c->L + c->N) +
                        sizeof(float) * (size_t)c->d.K * (c->M >> c->LE);
    // room is kept for the buffers a later PLM or projected solve would still take
    const size_t reserve = (c->Dg ? 0 : sizeof(float) * c->L) + (c->ls_dir ? 0 : sizeof(float2) * c->L);
    if (c->d.workspace_budget && c->allocated + need + reserve > c->d.workspace_budget) {
        c->lookahead_failed = true;
        return false;
    }
    if (ctx_alloc_t(c, &c->a_cache_b, (size_t)c->d.K * c->M, "look-ahead cache") != PTYLM_OK ||
        ctx_alloc_t(c, &c->grad_b, c->L, "look-ahead gradient") != PTYLM_OK ||
        ctx_alloc_t(c, &c->O_lin_b, c->N, "look-ahead point") != PTYLM_OK ||
        ctx_alloc_t(c, &c->trp_b, (size_t)c->d.K * (c->M >> c->LE), "look-ahead d2l sums") != PTYLM_OK) {
        c->lookahead_failed = true;   // a partial set stays allocated until the context is freed
        g_last_error.clear();
        return false;
    }
    return true;
}

// Make the look-ahead set the linearisation.
static void swap_lookahead(ptylm_ctx* c) {
    std::swap(c->a_cache, c->a_cache_b);
    std::swap(c->grad, c->grad_b);
    std::swap(c->O_lin, c->O_lin_b);
    std::swap(c->trp, c->trp_b);
    c->has_lin = c->has_point = true;
    c->u_valid = false;
}

// out += G v over z at the linearisation point (out already holds the damping term).
// With `skip`, the product is not formed (and out keeps its value) once *skip != 0.
static ptylm_status op_matvec_accumulate(ptylm_ctx* c, const float2* v, float2* out, const double* skip = nullptr) {
    if (c->d.K == 0) return PTYLM_OK;
    const int kid = joint(c) ? KID_MATVEC_J : KID_MATVEC;
    if (joint(c)) STATUS_TRY(clear_probe_part(c, kid));
    PtyArgs a = base_args(c);
    a.skip = skip;
    a.O = v;
    a.P = c->P_lin;
    a.a_cache = c->a_cache;
    a.out = out;
    if (joint(c)) {
        a.VP = v + c->N;
        a.Olin = c->O_lin;
    }
    STATUS_TRY(launch(c, kid, a));
    if (joint(c)) STATUS_TRY(probe_reduce(c, kid, out + c->N, true));
    return PTYLM_OK;
}

// out = (G + lambda D) v over z at the linearisation point (device pointers).
static ptylm_status op_matvec(ptylm_ctx* c, const float2* v, double lambda, const float* D, float2* out) {
    const int nb = vec_blocks(c);
    k_damping_init<<<nb, VEC_THREADS, 0, c->stream>>>(v, D, (float)lambda, out, c->L);
    STATUS_TRY(vec_launched(c));
    return op_matvec_accumulate(c, v, out);
}

// Closed-form Dg(G) over z at the linearisation point, floored at floor_rel * max.
static ptylm_status op_ggn_diag(ptylm_ctx* c, float* D, double floor_rel) {
    CUDA_TRY(cudaMemsetAsync(D, 0, sizeof(float) * c->L, c->stream));
    CUDA_TRY(launch_ggn_diag(c->LS, c->LE, c->trp, c->pos, c->d.K, c->O_lin, c->P_lin, c->d.nx, D,
                             joint(c) ? D + c->N : nullptr, c->tr, c->stream));
    c->launches += joint(c) ? 2 : 1;
    if (floor_rel > 0.0) {
        // each block (object, probe) is floored by its own maximum: their scales differ
        const int nb = vec_blocks(c);
        for (int blk = 0; blk < (joint(c) ? 2 : 1); ++blk) {
            float* Db = blk == 0 ? D : D + c->N;
            const long nblk = blk == 0 ? c->N : c->M;
            k_block_max<<<nb, VEC_THREADS, 0, c->stream>>>(Db, nblk, c->partials);
            STATUS_TRY(vec_launched(c));
            k_apply_floor<<<nb, VEC_THREADS, 0, c->stream>>>(Db, nblk, c->partials, nb, (float)floor_rel);
            STATUS_TRY(vec_launched(c));
        }
    }
    return PTYLM_OK;
}

// ---------------------------------------------------------------------------------------
// C-ABI
// ---------------------------------------------------------------------------------------
extern "C" {

const char* ptylm_strerror(ptylm_status s) {
    switch (s) {
        case PTYLM_OK: return "success";
        case PTYLM_ERR_ARG: return "invalid argument";
        case PTYLM_ERR_NOMEM: return "out of device memory or workspace budget";
        case PTYLM_ERR_CUDA: return "CUDA runtime error";
        case PTYLM_ERR_NAN: return "non-finite value in a reduction";
        case PTYLM_ERR_TIMEOUT: return "bounded device wait timed out";
        case PTYLM_ERR_STALLED: return "LM damping overflowed without an accepted step";
        case PTYLM_ERR_STATE: return "no linearisation point (call forward_loss with cache=1)";
        case PTYLM_WARN_CG_MAXIT: return "CG reached its iteration limit";
    }
    return "unknown status";
}

const char* ptylm_last_error(void) { return g_last_error.c_str(); }

void ptylm_default_lm_params(ptylm_lm_params* p, int loss) {
    if (!p) return;
    memset(p, 0, sizeof *p);
    p->mu0 = 1e-5;
    p->mu_min = 1e-8;
    p->kappa = 4.0;
    p->nu = 1.0;
    p->rho_min = 1e-4;
    p->beta = loss == PTYLM_LOSS_POISSON ? 0.9 : 0.1;
    p->mu_max = 1e16;
    p->max_outer = 50;
    p->max_cg = 100;
    p->fixed_cg = 0;
    p->target_err = 0.0;
    p->scaled = 0;
    p->projected = 0;
    p->radius_O = 1.0;
    p->radius_P = 1e8;
    p->gamma = 1e-6;
    p->tau_s = 1e-8;
    p->p_s = 2.1;
    p->sigma = 1e-4;
    p->max_ls = 30;
    p->diag_floor = 1e-6;
    p->surrogate0 = 1.0;
    p->surrogate_end = 1e-4;
    p->surrogate_T = 0;
    p->separate_cg_kernels = 0;
    p->wait_polls = 0;
}

// s_t of the App. E schedule: surrogate0 (surrogate_end / surrogate0)^(t / (T - 1)) for
// t < T, else 0.
static double surrogate_at(const ptylm_lm_params* p, int t) {
    if (p->surrogate_T <= 0 || t >= p->surrogate_T) return 0.0;
    if (p->surrogate_T == 1) return p->surrogate0;
    return p->surrogate0 * std::pow(p->surrogate_end / p->surrogate0, (double)t / (double)(p->surrogate_T - 1));
}

ptylm_status lm_init(ptylm_ctx** out, const ptylm_desc* desc, const int32_t* positions_dev,
                     const float* y_dev, void* stream) {
    g_last_error.clear();
    if (!out || !desc) return fail(PTYLM_ERR_ARG, "ctx and desc must be non-NULL");
    *out = nullptr;
    const ptylm_desc& d = *desc;
    if (d.my != d.mx) return fail(PTYLM_ERR_ARG, "probe must be square (my=%d, mx=%d)", d.my, d.mx);
    int LS = 0;
    if (d.my == 32) LS = 5;
    else if (d.my == 64) LS = 6;
    else if (d.my == 128) LS = 7;
    else return fail(PTYLM_ERR_ARG, "probe side %d unsupported (32, 64 or 128)", d.my);
    if (d.ny < d.my || d.nx < d.mx) return fail(PTYLM_ERR_ARG, "object %dx%d smaller than probe %dx%d", d.ny, d.nx, d.my, d.mx);
    if (d.K < 0) return fail(PTYLM_ERR_ARG, "K must be >= 0");
    if (d.loss != PTYLM_LOSS_GAUSSIAN && d.loss != PTYLM_LOSS_POISSON) return fail(PTYLM_ERR_ARG, "unknown loss %d", d.loss);
    if (!(d.background > 0.0f) || !std::isfinite(d.background)) return fail(PTYLM_ERR_ARG, "background must be finite and > 0");
    if (d.joint != 0 && d.joint != 1) return fail(PTYLM_ERR_ARG, "joint must be 0 or 1");
    if (d.K > 0 && (!positions_dev || !y_dev)) return fail(PTYLM_ERR_ARG, "positions and y must be non-NULL when K > 0");
    if ((long)d.ny * d.nx > (1L << 31)) return fail(PTYLM_ERR_ARG, "object too large");
    if (d.values_per_thread != 0 && d.values_per_thread != 32 && !(d.values_per_thread == 16 && LS <= 6))
        return fail(PTYLM_ERR_ARG, "values_per_thread must be 0, 32, or 16 for probe sides 32 and 64");

    // Validate positions on the host before anything is allocated or launched.
    std::vector<int32_t> hpos((size_t)d.K * 2);
    if (d.K > 0) {
        cudaError_t e = cudaMemcpy(hpos.data(), positions_dev, sizeof(int32_t) * 2 * d.K, cudaMemcpyDefault);
        if (e != cudaSuccess) return fail(PTYLM_ERR_CUDA, "reading positions: %s", cudaGetErrorString(e));
        for (int k = 0; k < d.K; ++k) {
            const int r = hpos[2 * k], cc = hpos[2 * k + 1];
            if (r < 0 || cc < 0 || r > d.ny - d.my || cc > d.nx - d.mx)
                return fail(PTYLM_ERR_ARG, "position %d = (%d, %d) outside [0, %d] x [0, %d]", k, r, cc,
                            d.ny - d.my, d.nx - d.mx);
        }
    }

    ptylm_ctx* c = new ptylm_ctx();
    c->d = d;
    c->b_eff = d.background;
    c->LS = LS;
    c->S = 1 << LS;
    c->M = c->S * c->S;
    c->N = (long)d.ny * d.nx;
    c->L = c->N + (d.joint ? c->M : 0);
    c->stream = static_cast<cudaStream_t>(stream);
    auto bail = [&](ptylm_status s) {
        ctx_free_all(c);
        delete c;
        return s;
    };
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(PTYLM_ERR_CUDA, "no usable CUDA device"));
    }
    // FFT tile: 32 values per thread, or 16 for sides 32 and 64 when teams of S^2/32 threads
    // would fill less than half of the GPU's thread slots (few positions): twice the threads
    // per patch halve each position's dependent chain of FFT passes
    if (d.values_per_thread == 16) c->LE = 4;
    else if (d.values_per_thread == 32) c->LE = 5;
    else c->LE = (LS <= 6 && (long)d.K * (c->M / 32) < (long)c->num_sms * 1024) ? 4 : 5;
    const int teams = cta_teams(LS, c->LE);
    for (int kid = 0; kid < KID_COUNT; ++kid) {
        int per_sm = 0;
        cudaError_t e = kernel_prepare(LS, c->LE, kid, &per_sm);
        if (e != cudaSuccess || per_sm <= 0)
            return bail(fail(PTYLM_ERR_CUDA, "kernel %d for side %d cannot launch: %s", kid, c->S,
                             e != cudaSuccess ? cudaGetErrorString(e) : "zero occupancy"));
        const int need = std::max(1, (d.K + teams - 1) / teams);
        c->grid[kid] = std::min(per_sm * c->num_sms, need);
    }
    // 4 CTAs per SM: enough loads in flight for the vector streams, and few enough partial
    // sums that the last CTA of each FP64 reduction finishes quickly
    c->vec_grid = std::min<long>(c->num_sms * 4L, std::max<long>(1, (c->L + VEC_THREADS - 1) / VEC_THREADS));
    c->probe_slots = d.joint ? std::max({c->grid[KID_FWD_CACHE_J], c->grid[KID_MATVEC_J], c->grid[KID_JTVP_J]}) * teams : 0;
    c->partials_cap = std::max(c->vec_grid, *std::max_element(c->grid, c->grid + KID_COUNT));
    // Single-launch CG iteration: the vector grid (all of it co-resident at 48 registers a
    // thread, so both forms give each thread the same elements and sum them in the same
    // order), capped at what is co-resident; 0 (three launches per iteration) when the
    // device cannot launch it cooperatively.
    {
        int coop = 0, per_sm = 0;
        if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->device) == cudaSuccess && coop &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)k_cg_iteration, VEC_THREADS, 0) ==
                cudaSuccess)
            c->coop_grid = (int)std::min<long>(c->vec_grid, (long)per_sm * c->num_sms);
        cudaGetLastError();
        c->partials_cap = std::max(c->partials_cap, c->coop_grid);   // rounds 1 and 2 use 3 x grid doubles
    }

    ptylm_status s;
    if ((s = ctx_alloc_t(c, &c->pos, std::max(1, d.K), "positions")) != PTYLM_OK) return bail(s);
    if ((s = ctx_alloc_t(c, &c->tw, c->S, "twiddles")) != PTYLM_OK) return bail(s);
    if ((s = ctx_alloc_t(c, &c->a_cache, (size_t)d.K * c->M, "frequency cache")) != PTYLM_OK) return bail(s);
    if ((s = ctx_alloc_t(c, &c->y_perm, (size_t)d.K * c->M, "measurements")) != PTYLM_OK) return bail(s);
    if ((s = ctx_alloc_t(c, &c->grad, c->L, "gradient")) != PTYLM_OK) return bail(s);
    if ((s = ctx_alloc_t(c, &c->trp, (size_t)std::max(1, d.K) * (c->M >> c->LE), "d2l sums")) != PTYLM_OK) return bail(s);
    if ((s = ctx_alloc_t(c, &c->tr, std::max(1, d.K), "per-position d2l sums")) != PTYLM_OK) return bail(s);
    if (d.joint && (s = ctx_alloc_t(c, &c->probe_part, (size_t)c->probe_slots * c->M, "probe accumulators")) != PTYLM_OK)
        return bail(s);
    if ((s = ctx_alloc_t(c, &c->O_lin, c->N, "object linearisation point")) != PTYLM_OK) return bail(s);
    if ((s = ctx_alloc_t(c, &c->P_lin, c->M, "probe linearisation point")) != PTYLM_OK) return bail(s);
    if ((s = ctx_alloc_t(c, &c->partials, (size_t)c->partials_cap * kMaxReduceWidth, "partials")) != PTYLM_OK) return bail(s);
    if ((s = ctx_alloc_t(c, &c->counters, CNT_COUNT, "reduction counters")) != PTYLM_OK) return bail(s);
    if ((s = ctx_alloc_t(c, &c->scal, S_COUNT, "scalars")) != PTYLM_OK) return bail(s);
    if (cudaMallocHost((void**)&c->scal_host, sizeof(double) * S_COUNT) != cudaSuccess) {
        cudaGetLastError();
        c->scal_host = nullptr;
        return bail(fail(PTYLM_ERR_NOMEM, "pinned scalar buffer"));
    }

    // Twiddles W_S^j = exp(-2 pi i j / S) in FP64, rounded once to FP32.
    std::vector<float2> htw(c->S);
    for (int j = 0; j < c->S; ++j) {
        const double ang = 2.0 * M_PI * (double)j / (double)c->S;
        htw[j] = make_float2((float)std::cos(ang), (float)-std::sin(ang));
    }
    std::vector<int2> hp((size_t)std::max(1, d.K));
    for (int k = 0; k < d.K; ++k) hp[k] = make_int2(hpos[2 * k], hpos[2 * k + 1]);
    if (cudaMemcpyAsync(c->tw, htw.data(), sizeof(float2) * c->S, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaMemcpyAsync(c->pos, hp.data(), sizeof(int2) * std::max(1, d.K), cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->scal, 0, sizeof(double) * S_COUNT, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->counters, 0, sizeof(unsigned) * CNT_COUNT, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
        cudaError_t e = cudaGetLastError();
        return bail(fail(PTYLM_ERR_CUDA, "uploading context tables: %s", cudaGetErrorString(e)));
    }
    if (d.K > 0) {
        cudaError_t e = permute_measurements(LS, c->LE, y_dev, c->y_perm, d.K, d.loss == PTYLM_LOSS_GAUSSIAN, c->vec_grid,
                                             c->stream, c->counters + CNT_YBAD);
        unsigned bad = 0;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&c->scal_host[0], c->counters + CNT_YBAD, sizeof(unsigned), cudaMemcpyDeviceToHost,
                                c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return bail(fail(PTYLM_ERR_CUDA, "copying measurements: %s", cudaGetErrorString(e)));
        memcpy(&bad, &c->scal_host[0], sizeof bad);
        if (bad) return bail(fail(PTYLM_ERR_ARG, "measurements y must be finite and >= 0"));
        if (cudaMemsetAsync(c->counters + CNT_YBAD, 0, sizeof(unsigned), c->stream) != cudaSuccess)
            return bail(fail(PTYLM_ERR_CUDA, "clearing the measurement flag"));
    }
    *out = c;
    return PTYLM_OK;
}

// Whether y (natural order, K M entries) is finite and >= 0: one read-only pass on the
// context stream, then a wait for the flag.
static ptylm_status check_measurements(ptylm_ctx* c, const float* y_dev) {
    CUDA_TRY(cudaMemsetAsync(c->counters + CNT_YBAD, 0, sizeof(unsigned), c->stream));
    CUDA_TRY(permute_measurements(c->LS, c->LE, y_dev, nullptr, c->d.K, 0, c->vec_grid, c->stream, c->counters + CNT_YBAD));
    ++c->launches;
    unsigned bad = 0;
    CUDA_TRY(cudaMemcpyAsync(&c->scal_host[0], c->counters + CNT_YBAD, sizeof(unsigned), cudaMemcpyDeviceToHost,
                             c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    memcpy(&bad, &c->scal_host[0], sizeof bad);
    CUDA_TRY(cudaMemsetAsync(c->counters + CNT_YBAD, 0, sizeof(unsigned), c->stream));
    if (bad) return fail(PTYLM_ERR_ARG, "measurements y must be finite and >= 0");
    return PTYLM_OK;
}

ptylm_status ptylm_set_measurements(ptylm_ctx* c, const float* y_dev) {
    g_last_error.clear();
    if (!c) return fail(PTYLM_ERR_ARG, "ctx must be non-NULL");
    if (c->d.K > 0 && !y_dev) return fail(PTYLM_ERR_ARG, "y must be non-NULL when K > 0");
    if (c->d.K == 0) {
        c->has_lin = false;
        return PTYLM_OK;
    }
    STATUS_TRY(check_measurements(c, y_dev));  // rejected data leave the context as it was
    c->has_lin = false;  // the loss cache depends on y; the point and the phasor do not
    CUDA_TRY(permute_measurements(c->LS, c->LE, y_dev, c->y_perm, c->d.K, c->d.loss == PTYLM_LOSS_GAUSSIAN, c->vec_grid,
                                  c->stream, nullptr));
    ++c->launches;
    return PTYLM_OK;
}

ptylm_status forward_intensity(ptylm_ctx* c, const ptylm_c64* O, const ptylm_c64* P, float* h_out) {
    g_last_error.clear();
    if (!c || !O || !P || !h_out) return fail(PTYLM_ERR_ARG, "ctx, O, P and h_out must be non-NULL");
    if (c->d.K == 0) return PTYLM_OK;
    PtyArgs a = base_args(c);
    a.O = reinterpret_cast<const float2*>(O);
    a.P = reinterpret_cast<const float2*>(P);
    a.out_real = h_out;
    STATUS_TRY(launch(c, KID_FWD_INTENSITY, a));
    return PTYLM_OK;
}

ptylm_status forward_magnitude(ptylm_ctx* c, const ptylm_c64* O, const ptylm_c64* P, float* zeta_out,
                               int store_phasor) {
    g_last_error.clear();
    if (!c || !O || !P || !zeta_out) return fail(PTYLM_ERR_ARG, "ctx, O, P and zeta_out must be non-NULL");
    CUDA_TRY(cudaMemcpyAsync(c->O_lin, O, sizeof(float2) * c->N, cudaMemcpyDeviceToDevice, c->stream));
    CUDA_TRY(cudaMemcpyAsync(c->P_lin, P, sizeof(float2) * c->M, cudaMemcpyDeviceToDevice, c->stream));
    c->has_lin = false;
    c->u_valid = false;
    c->has_point = true;
    if (store_phasor && !c->u_cache)
        STATUS_TRY(ctx_alloc_t(c, &c->u_cache, (size_t)std::max(1, c->d.K) * c->M, "phasor cache"));
    if (c->d.K == 0) return PTYLM_OK;
    PtyArgs a = base_args(c);
    a.O = c->O_lin;
    a.P = c->P_lin;
    a.out_real = zeta_out;
    a.a_cache = store_phasor ? c->u_cache : nullptr;
    STATUS_TRY(launch(c, KID_FWD_MAG, a));
    c->u_valid = store_phasor != 0;
    return PTYLM_OK;
}

ptylm_status ptylm_profile_select(ptylm_ctx* c, unsigned mask) {
    if (!c) return fail(PTYLM_ERR_ARG, "ctx must be non-NULL");
    if (mask) {
        STATUS_TRY(prof_flush(c));
        for (int k = 0; k < PROF_COUNT; ++k) {
            c->prof_ms[k] = 0.0;
            c->prof_n[k] = 0;
        }
        c->launches = 0;
    }
    c->prof_mask = mask & ((1u << PROF_COUNT) - 1u);
    return PTYLM_OK;
}

ptylm_status ptylm_profile(ptylm_ctx* c, int enable) { return ptylm_profile_select(c, enable ? ~0u : 0u); }

ptylm_status ptylm_profile_read(ptylm_ctx* c, int kernel, double* total_ms, long long* launches) {
    if (!c) return fail(PTYLM_ERR_ARG, "ctx must be non-NULL");
    if (kernel < -1 || kernel >= PROF_COUNT) return fail(PTYLM_ERR_ARG, "unknown kernel id %d", kernel);
    STATUS_TRY(prof_flush(c));
    if (kernel == -1) {
        if (total_ms) *total_ms = 0.0;
        if (launches) *launches = c->launches;
    } else {
        if (total_ms) *total_ms = c->prof_ms[kernel];
        if (launches) *launches = c->prof_n[kernel];
    }
    return PTYLM_OK;
}

ptylm_status lm_destroy(ptylm_ctx* c) {
    if (!c) return PTYLM_OK;
    cudaStreamSynchronize(c->stream);
    ctx_free_all(c);
    delete c;
    return PTYLM_OK;
}

ptylm_status forward_loss(ptylm_ctx* c, const ptylm_c64* O, const ptylm_c64* P, double* f_host,
                          double* dl_norm2_host, int cache) {
    g_last_error.clear();
    if (!c || !O || !P) return fail(PTYLM_ERR_ARG, "ctx, O and P must be non-NULL");
    STATUS_TRY(op_forward(c, reinterpret_cast<const float2*>(O), reinterpret_cast<const float2*>(P), cache));
    STATUS_TRY(read_scalars(c, S_F, 2));
    const double f = c->scal_host[S_F], dl2 = c->scal_host[S_DL2];
    if (cache) {
        c->f_lin = f;
        c->dl2_lin = dl2;
    }
    if (f_host) *f_host = f;
    if (dl_norm2_host) *dl_norm2_host = dl2;
    if (!std::isfinite(f) || !std::isfinite(dl2)) return fail(PTYLM_ERR_NAN, "loss is not finite (f=%g)", f);
    return PTYLM_OK;
}

ptylm_status gradient(ptylm_ctx* c, ptylm_c64* gO, ptylm_c64* gP) {
    g_last_error.clear();
    if (!c || !gO) return fail(PTYLM_ERR_ARG, "ctx and gO must be non-NULL");
    if (gP && !joint(c)) return fail(PTYLM_ERR_ARG, "probe gradient needs a joint context");
    if (!c->has_lin) return fail(PTYLM_ERR_STATE, "no linearisation point");
    CUDA_TRY(cudaMemcpyAsync(gO, c->grad, sizeof(float2) * c->N, cudaMemcpyDeviceToDevice, c->stream));
    if (gP) CUDA_TRY(cudaMemcpyAsync(gP, c->grad + c->N, sizeof(float2) * c->M, cudaMemcpyDeviceToDevice, c->stream));
    return PTYLM_OK;
}

ptylm_status jvp(ptylm_ctx* c, const ptylm_c64* vO, const ptylm_c64* vP, float* out) {
    g_last_error.clear();
    if (!c || !vO || !out) return fail(PTYLM_ERR_ARG, "ctx, vO and out must be non-NULL");
    if (vP && !joint(c)) return fail(PTYLM_ERR_ARG, "probe direction needs a joint context");
    if (!c->has_point) return fail(PTYLM_ERR_STATE, "no linearisation point");
    if (c->d.K == 0) return PTYLM_OK;
    const int kid = c->u_valid ? (vP ? KID_JVP_U_J : KID_JVP_U) : (vP ? KID_JVP_J : KID_JVP);
    if (!c->u_valid && !c->jvp_scratch) {
        const size_t slots = (size_t)std::max(c->grid[KID_JVP], c->grid[KID_JVP_J]) * cta_teams(c->LS, c->LE);
        STATUS_TRY(ctx_alloc_t(c, &c->jvp_scratch, slots * c->M, "jvp scratch"));
    }
    PtyArgs a = base_args(c);
    a.O = c->O_lin;
    a.V = reinterpret_cast<const float2*>(vO);
    a.VP = reinterpret_cast<const float2*>(vP);
    a.P = c->P_lin;
    a.out_real = out;
    a.scratch = c->jvp_scratch;
    a.a_cache = c->u_valid ? c->u_cache : nullptr;
    STATUS_TRY(launch(c, kid, a));
    return PTYLM_OK;
}

ptylm_status jtvp(ptylm_ctx* c, const float* w, ptylm_c64* outO, ptylm_c64* outP) {
    g_last_error.clear();
    if (!c || !w || !outO) return fail(PTYLM_ERR_ARG, "ctx, w and outO must be non-NULL");
    if (outP && !joint(c)) return fail(PTYLM_ERR_ARG, "probe part needs a joint context");
    if (!c->has_point) return fail(PTYLM_ERR_STATE, "no linearisation point");
    CUDA_TRY(cudaMemsetAsync(outO, 0, sizeof(float2) * c->N, c->stream));
    if (outP) CUDA_TRY(cudaMemsetAsync(outP, 0, sizeof(float2) * c->M, c->stream));
    if (c->d.K == 0) return PTYLM_OK;
    const int kid = c->u_valid ? (outP ? KID_JTVP_U_J : KID_JTVP_U) : (outP ? KID_JTVP_J : KID_JTVP);
    if (outP) STATUS_TRY(clear_probe_part(c, kid));
    PtyArgs a = base_args(c);
    a.O = c->O_lin;
    a.P = c->P_lin;
    a.w = w;
    a.out = reinterpret_cast<float2*>(outO);
    a.a_cache = c->u_valid ? c->u_cache : nullptr;
    STATUS_TRY(launch(c, kid, a));
    if (outP) STATUS_TRY(probe_reduce(c, kid, reinterpret_cast<float2*>(outP), false));
    return PTYLM_OK;
}

ptylm_status ggn_matvec(ptylm_ctx* c, const ptylm_c64* vO, const ptylm_c64* vP, double lambda,
                        const float* D, ptylm_c64* outO, ptylm_c64* outP) {
    g_last_error.clear();
    if (!c || !vO || !outO) return fail(PTYLM_ERR_ARG, "ctx, vO and outO must be non-NULL");
    if (joint(c) != (vP != nullptr) || joint(c) != (outP != nullptr))
        return fail(PTYLM_ERR_ARG, "vP and outP are required in joint contexts and must be NULL otherwise");
    if (!c->has_lin) return fail(PTYLM_ERR_STATE, "no linearisation point");
    if (!std::isfinite(lambda)) return fail(PTYLM_ERR_ARG, "lambda must be finite");
    const bool host_in = is_host_pointer(vO) || (vP && is_host_pointer(vP));
    const bool host_out = is_host_pointer(outO) || (outP && is_host_pointer(outP));
    if (!c->stage_a) STATUS_TRY(ctx_alloc_t(c, &c->stage_a, c->L, "staging (vector)"));
    if (!c->stage_b) STATUS_TRY(ctx_alloc_t(c, &c->stage_b, c->L, "staging (result)"));
    // gather z-vectors contiguously (object part, then probe part)
    const float2* v = reinterpret_cast<const float2*>(vO);
    if (host_in || joint(c)) {
        const cudaMemcpyKind k = host_in ? cudaMemcpyDefault : cudaMemcpyDeviceToDevice;
        CUDA_TRY(cudaMemcpyAsync(c->stage_a, vO, sizeof(float2) * c->N, k, c->stream));
        if (vP) CUDA_TRY(cudaMemcpyAsync(c->stage_a + c->N, vP, sizeof(float2) * c->M, k, c->stream));
        v = c->stage_a;
    }
    float2* o = (host_out || joint(c)) ? c->stage_b : reinterpret_cast<float2*>(outO);
    STATUS_TRY(op_matvec(c, v, lambda, D, o));
    if (host_out || joint(c)) {
        const cudaMemcpyKind k = host_out ? cudaMemcpyDefault : cudaMemcpyDeviceToDevice;
        CUDA_TRY(cudaMemcpyAsync(outO, o, sizeof(float2) * c->N, k, c->stream));
        if (outP) CUDA_TRY(cudaMemcpyAsync(outP, o + c->N, sizeof(float2) * c->M, k, c->stream));
        if (host_out) CUDA_TRY(cudaStreamSynchronize(c->stream));
    }
    return PTYLM_OK;
}

ptylm_status ggn_diag(ptylm_ctx* c, float* D_out, double floor_rel) {
    g_last_error.clear();
    if (!c || !D_out) return fail(PTYLM_ERR_ARG, "ctx and D_out must be non-NULL");
    if (!c->has_lin) return fail(PTYLM_ERR_STATE, "no linearisation point");
    if (!(floor_rel >= 0.0) || !(floor_rel < 1.0)) return fail(PTYLM_ERR_ARG, "floor_rel must be in [0, 1)");
    return op_ggn_diag(c, D_out, floor_rel);
}

static ptylm_status lm_solve_impl(ptylm_ctx* c, ptylm_c64* O_inout, ptylm_c64* P_inout, const ptylm_lm_params* prm,
                                  ptylm_lm_state* state, ptylm_lm_stats* stats) {
    g_last_error.clear();
    if (!c || !O_inout || !P_inout || !prm) return fail(PTYLM_ERR_ARG, "ctx, O, P and params must be non-NULL");
    if (prm->max_outer < 0 || prm->max_cg < 0 || !(prm->kappa > 1.0) || !(prm->mu0 > 0.0) || prm->wait_polls < 0)
        return fail(PTYLM_ERR_ARG, "invalid LM parameters");
    c->cg_spin_limit = prm->wait_polls > 0 ? (unsigned)prm->wait_polls : kCoopSpinLimit;
    if (prm->projected && (!(prm->radius_O > 0.0) || !(prm->radius_P > 0.0) || prm->max_ls < 0))
        return fail(PTYLM_ERR_ARG, "invalid projection parameters");
    if (c->d.K == 0) return fail(PTYLM_ERR_ARG, "lm_solve needs at least one scan position");
    if (prm->surrogate_T < 0 ||
        (prm->surrogate_T > 0 && (!(prm->surrogate0 > 0.0) || !(prm->surrogate_end > 0.0) ||
                                  !std::isfinite(prm->surrogate0) || !std::isfinite(prm->surrogate_end))))
        return fail(PTYLM_ERR_ARG, "invalid surrogate schedule");
    // Every exit restores the true background; a linearisation taken under s_t > 0 is not
    // the true metric's, so it is dropped.
    struct SurrogateGuard {
        ptylm_ctx* c;
        bool used = false;
        ~SurrogateGuard() {
            c->b_eff = c->d.background;
            if (used) c->has_lin = c->u_valid = false;
        }
    } surrogate_guard{c};
    const long N = c->N, L = c->L;
    const size_t zbytes = sizeof(float2) * L;
    if (!c->cg_x) {
        STATUS_TRY(ctx_alloc_t(c, &c->cg_x, L, "CG x"));
        STATUS_TRY(ctx_alloc_t(c, &c->cg_r, L, "CG r"));
        STATUS_TRY(ctx_alloc_t(c, &c->cg_p, L, "CG p"));
        STATUS_TRY(ctx_alloc_t(c, &c->cg_q, L, "CG q"));
        STATUS_TRY(ctx_alloc_t(c, &c->trial, L, "trial point"));
    }
    if (prm->projected && !c->ls_dir) STATUS_TRY(ctx_alloc_t(c, &c->ls_dir, L, "line-search direction"));
    if (prm->scaled && !c->Dg) STATUS_TRY(ctx_alloc_t(c, &c->Dg, L, "scaling"));
    if (!c->stage_a) STATUS_TRY(ctx_alloc_t(c, &c->stage_a, L, "iterate"));
    if (!c->stage_P) STATUS_TRY(ctx_alloc_t(c, &c->stage_P, c->M, "probe"));
    // The look-ahead set (a second cache, gradient, point and d2l sums) is optional: when the
    // workspace budget has no room for it every outer iteration runs its own forward pass.
    const bool lookahead = !joint(c) && c->d.K > 0 && !prm->projected && lookahead_set(c);
    const bool host_O = is_host_pointer(O_inout), host_P = is_host_pointer(P_inout);
    const cudaMemcpyKind kin_O = host_O ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const cudaMemcpyKind kin_P = host_P ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    // The state z = [O; P] lives in stage_a throughout (the caller's buffers are read once,
    // written once); object-only contexts keep the fixed probe in stage_P.
    float2* z = c->stage_a;
    CUDA_TRY(cudaMemsetAsync(c->scal + S_CG_TIMEOUT, 0, sizeof(double), c->stream));
    CUDA_TRY(cudaMemcpyAsync(z, O_inout, sizeof(float2) * N, kin_O, c->stream));
    if (joint(c)) CUDA_TRY(cudaMemcpyAsync(z + N, P_inout, sizeof(float2) * c->M, kin_P, c->stream));
    else CUDA_TRY(cudaMemcpyAsync(c->stage_P, P_inout, sizeof(float2) * c->M, kin_P, c->stream));
    auto probe_of = [&](float2* state) -> const float2* { return joint(c) ? state + N : c->stage_P; };
    float2 *x = c->cg_x, *r = c->cg_r, *p = c->cg_p, *q = c->cg_q, *trial = c->trial;
    const float* D = prm->scaled ? c->Dg : nullptr;
    const int nb = vec_blocks(c);
    unsigned* cnt = c->counters + CNT_VEC;
    CUDA_TRY(cudaMemsetAsync(x, 0, zbytes, c->stream));
    // a resumed run starts from the saved warm start, damping and outer-iteration count
    const int t0 = state ? state->t : 0;
    if (state && state->delta)
        CUDA_TRY(cudaMemcpyAsync(x, state->delta, zbytes,
                                 is_host_pointer(state->delta) ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                                 c->stream));

    double f_min = 0.0;  // Algorithm 2 compares f - f_min (the Poisson metric can be negative)
    if (prm->projected && c->d.loss == PTYLM_LOSS_POISSON) {
        k_poisson_fmin<<<nb, VEC_THREADS, 0, c->stream>>>(c->y_perm, (long)c->d.K * c->M, c->partials, cnt, c->scal);
        STATUS_TRY(vec_launched(c));
        STATUS_TRY(read_scalars(c, S_FMIN, 1));
        f_min = c->scal_host[S_FMIN];
    }
    auto loss_at = [&](float2* state, double* f_out) -> ptylm_status {
        STATUS_TRY(op_forward(c, state, probe_of(state), 0));
        STATUS_TRY(read_scalars(c, S_F, 1));
        *f_out = c->scal_host[S_F];
        return PTYLM_OK;
    };
    auto project = [&](float2* state) -> ptylm_status {
        k_project<<<nb, VEC_THREADS, 0, c->stream>>>(state, N, L, (float)prm->radius_O, (float)prm->radius_P);
        return vec_launched(c);
    };

    double mu = state ? state->mu : prm->mu0;
    int cg_total = 0, matvecs = 0, t = 0;
    bool hit_maxit = false;
    ptylm_status status = PTYLM_OK;
    double f_cur = NAN, err = NAN;
    auto object_error = [&](double* e_out) -> ptylm_status {
        k_err_sums<<<nb, VEC_THREADS, 0, c->stream>>>(z, reinterpret_cast<const float2*>(prm->O_ref), prm->mask, N,
                                                      c->partials, cnt, c->scal);
        STATUS_TRY(vec_launched(c));
        STATUS_TRY(read_scalars(c, S_ER, 4));
        const double ac = std::hypot(c->scal_host[S_ER], c->scal_host[S_EI]);
        const double e2 = std::max(0.0, c->scal_host[S_NO] + c->scal_host[S_NR] - 2.0 * ac);
        *e_out = std::sqrt(e2 / c->scal_host[S_NR]);
        return PTYLM_OK;
    };

    bool ahead = false;   // the linearisation at z came with the accepted trial point
    const auto t_start = std::chrono::steady_clock::now();
    struct NvtxOuter {
        bool open = false;
        void begin(int t) {
            end();
            char name[48];
            snprintf(name, sizeof name, "lm: outer iteration %d", t);
            nvtxRangePushA(name);
            open = true;
        }
        void end() {
            if (open) nvtxRangePop();
            open = false;
        }
        ~NvtxOuter() { end(); }
    } nvtx_outer;
    for (t = t0; t < t0 + prm->max_outer; ++t) {
        const int h = t - t0;   // history entry of this outer iteration
        nvtx_outer.begin(t);
        const double s_t = surrogate_at(prm, t);
        c->b_eff = (float)(c->d.background + s_t);
        surrogate_guard.used = s_t > 0.0;
        // Linearise: f, ||grad_zeta l||^2, cache a, grad f, Dg(G) (Algorithm 1, first step).
        if (!ahead) STATUS_TRY(op_forward(c, z, probe_of(z), 1));
        ahead = false;
        STATUS_TRY(dots(c, 1, L, c->grad, c->grad, nullptr, nullptr, nullptr, nullptr, nullptr, S_GG));
        if (D) STATUS_TRY(op_ggn_diag(c, c->Dg, prm->diag_floor));
        STATUS_TRY(read_scalars(c, S_F, S_GG - S_F + 1));
        const double f = c->scal_host[S_F], dl2 = c->scal_host[S_DL2], gg = c->scal_host[S_GG];
        if (!std::isfinite(f) || !std::isfinite(gg)) {
            status = fail(PTYLM_ERR_NAN, "non-finite loss or gradient at outer iteration %d", t);
            break;
        }
        f_cur = f;
        const double gnorm = std::sqrt(gg);
        const double eta = std::min(prm->beta, std::sqrt(gnorm));  // Eq. lma_termination_eta
        const double tol = eta * gnorm;                              // Eq. lma_termination_magnitude
        if (stats && stats->hist_len > h) {
            if (stats->hist_f) stats->hist_f[h] = f;
            if (stats->hist_gnorm) stats->hist_gnorm[h] = gnorm;
        }
        double rho = 0.0, lambda_last = NAN;
        int cg_this = 0;
        bool stalled = false, timed_out = false;
        struct NvtxSolve {   // closed on every exit from this outer iteration
            NvtxSolve() { nvtxRangePushA("lm: CG solves and trial points"); }
            ~NvtxSolve() { nvtxRangePop(); }
        };
        std::optional<NvtxSolve> nvtx_solve;
        nvtx_solve.emplace();
        while (!(rho > prm->rho_min)) {
            // lambda = mu ||grad_zeta l||^nu (D = I) or mu (D = Dg(G)), Algorithm 1
            const double lambda = D ? mu : mu * std::pow(std::sqrt(dl2), prm->nu);
            lambda_last = lambda;
            const float lam32 = (float)lambda;
            // ---- truncated (P)CG on (G + lambda D) x = -g, warm-started from x ----
            STATUS_TRY(op_matvec(c, x, lambda, D, q));                            // q = (G + lambda D) x
            ++matvecs;
            k_cg_start<<<nb, VEC_THREADS, 0, c->stream>>>(c->grad, q, r, p, D, lam32, L, c->partials, cnt, c->scal);
            STATUS_TRY(vec_launched(c));                                          // r, p = P^-1 r, q = lambda D p
            int it = 0;
            bool converged = false;
            const bool separate = prm->separate_cg_kernels != 0;
            if (prm->fixed_cg <= 0 && !separate && c->coop_grid > 0) {
                // The stopping test (Eq. lma_termination_magnitude) runs on the device before and
                // after each iteration; the host queues as many iterations as the last solve took
                // (then a quarter of that at a time) and reads the count and the flag once per batch.
                if (prm->max_cg == 0) {
                    STATUS_TRY(read_scalars(c, S_RR, 1));
                    converged = std::sqrt(c->scal_host[S_RR]) <= tol;
                } else {
                    k_cg_check<<<1, 32, 0, c->stream>>>(c->scal, tol);
                    STATUS_TRY(vec_launched(c));
                    const int first = std::max(1, c->cg_chunk);
                    int queued = 0, batch = first;
                    for (;;) {
                        const int nq = std::min(batch, prm->max_cg - queued);
                        for (int i = 0; i < nq; ++i) {
                            STATUS_TRY(op_matvec_accumulate(c, p, q, c->scal + S_CG_DONE));   // q += G p
                            STATUS_TRY(cg_iteration(c, x, r, p, q, D, lam32, false, tol));
                        }
                        queued += nq;
                        STATUS_TRY(read_scalars(c, S_CG_DONE, 2));
                        it = (int)c->scal_host[S_CG_ITERS];
                        converged = c->scal_host[S_CG_DONE] != 0.0;
                        if (converged || queued >= prm->max_cg) break;
                        batch = std::max(1, first / 4);
                    }
                    c->cg_chunk = it;
                }
                matvecs += it;
            } else {
                for (;;) {
                    if (prm->fixed_cg > 0) {
                        if (it >= prm->fixed_cg) break;
                    } else {
                        STATUS_TRY(read_scalars(c, S_RR, 1));
                        if (std::sqrt(c->scal_host[S_RR]) <= tol) { converged = true; break; }
                        if (it >= prm->max_cg) break;
                    }
                    STATUS_TRY(op_matvec_accumulate(c, p, q));                        // q += G p
                    ++matvecs;
                    STATUS_TRY(cg_iteration(c, x, r, p, q, D, lam32, separate));
                    ++it;
                }
            }
            cg_this += it;
            if (!converged && prm->fixed_cg <= 0 && it >= prm->max_cg) hit_maxit = true;
            // ---- trial point and gain ratio (Algorithm 1) ----
            k_axpy<<<nb, VEC_THREADS, 0, c->stream>>>(z, x, 1.0f, trial, L);
            STATUS_TRY(vec_launched(c));
            // the trial's forward pass doubles as the next linearisation when the next outer
            // iteration exists and uses the same background
            const bool ahead_here = lookahead && t + 1 < t0 + prm->max_outer &&
                                    surrogate_at(prm, t + 1) == s_t;
            if (ahead_here) STATUS_TRY(op_forward_lookahead(c, trial));
            else STATUS_TRY(op_forward(c, trial, probe_of(trial), 0));
            STATUS_TRY(dots(c, 3, L, x, x, D, x, c->grad, x, r, S_DD));
            STATUS_TRY(read_scalars(c, S_F, S_CG_TIMEOUT - S_F + 1));
            if (c->scal_host[S_CG_TIMEOUT] != 0.0) {
                timed_out = true;
                break;
            }
            const double f_trial = c->scal_host[S_F];
            const double dd = c->scal_host[S_DD], dg = c->scal_host[S_DG], dr = c->scal_host[S_DR];
            const double dfa = f - f_trial;
            const double dfp = 0.5 * (lambda * dd - dg) + 0.5 * dr;  // -(g.d + d.G.d/2)
            rho = (dfp > 0.0 && std::isfinite(f_trial)) ? dfa / dfp : -1.0;
            if (rho > 0.75) mu = std::max(mu / prm->kappa, prm->mu_min);
            else if (rho > 0.25) { /* keep mu */ }
            else mu = prm->kappa * mu;
            if (rho > prm->rho_min) {
                if (!prm->projected) {
                    CUDA_TRY(cudaMemcpyAsync(z, trial, zbytes, cudaMemcpyDeviceToDevice, c->stream));
                    f_cur = f_trial;
                    if (ahead_here) {
                        swap_lookahead(c);
                        ahead = true;
                    }
                } else {
                    // ---- Algorithm 2: projected step, descent test, Armijo backtracking ----
                    STATUS_TRY(project(trial));
                    double fp = 0.0;
                    STATUS_TRY(loss_at(trial, &fp));
                    if (fp - f_min < prm->gamma * (f - f_min)) {
                        CUDA_TRY(cudaMemcpyAsync(z, trial, zbytes, cudaMemcpyDeviceToDevice, c->stream));
                        f_cur = fp;
                    } else {
                        float2* sdir = c->ls_dir;
                        k_axpy<<<nb, VEC_THREADS, 0, c->stream>>>(trial, z, -1.0f, sdir, L);   // s = Pi(z + dz) - z
                        STATUS_TRY(vec_launched(c));
                        STATUS_TRY(dots(c, 2, L, c->grad, sdir, nullptr, sdir, sdir, nullptr, nullptr, S_GS));
                        STATUS_TRY(read_scalars(c, S_GS, 2));
                        const double gs = c->scal_host[S_GS], ss = c->scal_host[S_SS];
                        double sn2 = ss;
                        if (!(gs <= -prm->tau_s * std::pow(std::sqrt(ss), prm->p_s))) {
                            // not a descent direction: projected gradient step, s = -g
                            k_axpy<<<nb, VEC_THREADS, 0, c->stream>>>(c->grad, c->grad, -2.0f, sdir, L);
                            STATUS_TRY(vec_launched(c));
                            sn2 = gg;
                        }
                        double alpha = 1.0;
                        for (int ls = 0; ls < prm->max_ls; ++ls, alpha *= 0.5) {
                            k_axpy<<<nb, VEC_THREADS, 0, c->stream>>>(z, sdir, (float)alpha, trial, L);
                            STATUS_TRY(vec_launched(c));
                            STATUS_TRY(project(trial));
                            double fl = 0.0;
                            STATUS_TRY(loss_at(trial, &fl));
                            if (fl <= f - prm->sigma * alpha * sn2) {             // Eq. armijo_criterion
                                CUDA_TRY(cudaMemcpyAsync(z, trial, zbytes, cudaMemcpyDeviceToDevice, c->stream));
                                f_cur = fl;
                                break;
                            }
                        }
                    }
                }
            } else if (mu > prm->mu_max) {
                stalled = true;
                break;
            }
        }
        nvtx_solve.reset();
        cg_total += cg_this;
        if (stats && stats->hist_len > h) {
            if (stats->hist_mu) stats->hist_mu[h] = mu;
            if (stats->hist_cg) stats->hist_cg[h] = cg_this;
            if (stats->hist_rho) stats->hist_rho[h] = rho;
            if (stats->hist_lambda) stats->hist_lambda[h] = lambda_last;
            if (stats->hist_time)
                stats->hist_time[h] = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
        }
        if (timed_out) {
            status = fail(PTYLM_ERR_TIMEOUT, "a grid-wide wait of the CG iteration gave up at outer iteration %d", t);
            break;
        }
        if (stalled) {
            status = fail(PTYLM_ERR_STALLED, "mu exceeded %g at outer iteration %d", prm->mu_max, t);
            ++t;
            break;
        }
        if (prm->O_ref) {
            STATUS_TRY(object_error(&err));
            if (stats && stats->hist_len > h && stats->hist_err) stats->hist_err[h] = err;
            if (prm->target_err > 0.0 && err <= prm->target_err) {
                ++t;
                break;
            }
        } else if (stats && stats->hist_len > h && stats->hist_err) {
            stats->hist_err[h] = NAN;
        }
    }
    CUDA_TRY(cudaMemcpyAsync(O_inout, z, sizeof(float2) * N, host_O ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                             c->stream));
    if (joint(c))
        CUDA_TRY(cudaMemcpyAsync(P_inout, z + N, sizeof(float2) * c->M,
                                 host_P ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (state) {
        state->t = t;
        state->mu = mu;
        if (state->delta)
            CUDA_TRY(cudaMemcpy(state->delta, x, zbytes,
                                is_host_pointer(state->delta) ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice));
    }
    if (stats) {
        stats->n_outer = t - t0;
        stats->cg_total = cg_total;
        stats->matvecs_total = matvecs;
        stats->f_final = f_cur;
        stats->err_final = err;
    }
    if (status != PTYLM_OK) return status;
    return hit_maxit ? PTYLM_WARN_CG_MAXIT : PTYLM_OK;
}

ptylm_status lm_solve(ptylm_ctx* c, ptylm_c64* O_inout, ptylm_c64* P_inout, const ptylm_lm_params* prm,
                      ptylm_lm_stats* stats) {
    return lm_solve_impl(c, O_inout, P_inout, prm, nullptr, stats);
}

ptylm_status lm_solve_resume(ptylm_ctx* c, ptylm_c64* O_inout, ptylm_c64* P_inout, const ptylm_lm_params* prm,
                             ptylm_lm_state* state, ptylm_lm_stats* stats) {
    g_last_error.clear();
    if (!state) return fail(PTYLM_ERR_ARG, "state must be non-NULL (lm_solve starts afresh)");
    if (state->t < 0 || !(state->mu > 0.0) || !std::isfinite(state->mu))
        return fail(PTYLM_ERR_ARG, "invalid LM state (t = %d, mu = %g)", state->t, state->mu);
    return lm_solve_impl(c, O_inout, P_inout, prm, state, stats);
}

}  // extern "C"
