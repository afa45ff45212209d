// ptylm_batch.cu -- C-ABI of batches of independent reconstructions (include/ptylm.h):
// context, chunked vector kernels with per-problem FP64 scalars, the batched truncated CG
// captured as a CUDA graph, the batched Algorithm 1 driver and the schedule autotuner.
//
// Batch vectors are the concatenation of the problems' objects.  Vector kernels run one
// 256-thread block per chunk of at most 4096 elements of one problem; a dot product's last
// block sums each problem's chunk partials in chunk order (FP64) and applies the CG scalar
// update of that problem, so a CG iteration of all problems is four launches (the batched
// GGN product, p.q -> alpha, x/r update -> beta and convergence, new direction) with no
// host round trip.  Problems whose CG has converged (or whose LM has finished) are masked
// out of every launch, including the per-position work items of the GGN product.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ptylm.h"
#include "batch.h"
#include "kernels.h"
#include "reduce.cuh"

using namespace ptylm;

namespace {

ptylm_status bfail(ptylm_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    set_last_error(buf);
    return s;
}

#define BCUDA_TRY(expr)                                                                          \
    do {                                                                                         \
        cudaError_t e_ = (expr);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return bfail(PTYLM_ERR_CUDA, "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), \
                         __FILE__, __LINE__);                                                    \
    } while (0)

#define BSTATUS_TRY(expr)               \
    do {                                \
        ptylm_status s_ = (expr);       \
        if (s_ != PTYLM_OK) return s_;  \
    } while (0)

constexpr int BVEC_THREADS = 256;
constexpr int CHUNK = 4096;

struct Chunk {
    long begin;
    int len, prob;
};

__device__ __forceinline__ float brdot(float2 a, float2 b) { return a.x * b.x + a.y * b.y; }

#define CHUNK_LOOP(c, g) for (long g = (c).begin + threadIdx.x; g < (c).begin + (c).len; g += blockDim.x)

// Scaling of a batch vector: problems with scaled[b] use the diagonal D (PLM, D = Dg(G)),
// the others the identity (LM).
struct Scale {
    const float* D;      // [total] or NULL
    const int* scaled;   // [B] or NULL
    __device__ __forceinline__ bool on(int b) const { return D && scaled && scaled[b]; }
};

// out = lambda_b D_b v over the chunks of problems with mask[b] (the damping term of the GGN
// product, written before the per-position kernel accumulates into out).
__global__ void kb_damp(const Chunk* ch, const int* mask, const float* lam, const float2* __restrict__ v,
                        float2* __restrict__ out, Scale sc) {
    const Chunk c = ch[blockIdx.x];
    if (mask && !mask[c.prob]) return;
    const float l = lam ? lam[c.prob] : 0.0f;
    const bool dsc = sc.on(c.prob);
    CHUNK_LOOP(c, g) {
        const float2 x = v[g];
        const float w = dsc ? l * sc.D[g] : l;
        out[g] = make_float2(w * x.x, w * x.y);
    }
}

// D over the chunks of problems with mask[b]: zero; per-problem maximum (non-negative floats
// compare as their bit patterns); floor at floor_rel * that maximum (reading C10).
__global__ void kb_dzero(const Chunk* ch, const int* mask, float* D) {
    const Chunk c = ch[blockIdx.x];
    if (mask && !mask[c.prob]) return;
    CHUNK_LOOP(c, g) D[g] = 0.0f;
}
__global__ void kb_dmax(const Chunk* ch, const int* mask, const float* __restrict__ D, unsigned* dmax) {
    const Chunk c = ch[blockIdx.x];
    if (mask && !mask[c.prob]) return;
    float m = 0.0f;
    CHUNK_LOOP(c, g) m = fmaxf(m, D[g]);
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(dmax + c.prob, __float_as_uint(m));
}
__global__ void kb_dfloor(const Chunk* ch, const int* mask, const unsigned* __restrict__ dmax,
                          const float* __restrict__ floor_rel, float* D) {
    const Chunk c = ch[blockIdx.x];
    if (mask && !mask[c.prob]) return;
    const float fl = floor_rel[c.prob] * __uint_as_float(dmax[c.prob]);
    CHUNK_LOOP(c, g) D[g] = fmaxf(D[g], fl);
}

// z = x + d (mask), z = x (copy mask), z = 0 (mask)
__global__ void kb_axpy(const Chunk* ch, const int* mask, const float2* __restrict__ x, const float2* __restrict__ d,
                        float2* __restrict__ z) {
    const Chunk c = ch[blockIdx.x];
    if (mask && !mask[c.prob]) return;
    CHUNK_LOOP(c, g) {
        const float2 a = x[g];
        const float2 b = d ? d[g] : make_float2(0.0f, 0.0f);
        z[g] = make_float2(a.x + b.x, a.y + b.y);
    }
}
__global__ void kb_zero(const Chunk* ch, const int* mask, float2* __restrict__ z) {
    const Chunk c = ch[blockIdx.x];
    if (mask && !mask[c.prob]) return;
    CHUNK_LOOP(c, g) z[g] = make_float2(0.0f, 0.0f);
}

// What the last block does per problem after the FP64 sums c[] are formed.
enum BatchPost { POST_NONE = 0, POST_START = 1, POST_UPDATE = 2 };

struct DotArgs {
    const Chunk* ch;
    const int* chunk_first;   // [B + 1]
    int B;
    int* mask;                // problems taking part (NULL: all)
    double* part;             // [n_chunks][4]
    unsigned* counter;
    double* sc;               // [B][S_COUNT]
    int dst, op, post;
    int* cg_it;               // POST_START / POST_UPDATE
    const int* lm_active;     // POST_START: problems whose CG starts
    const double* tol2;       // [B] stop when r.r <= tol2
    const int* max_cg;        // [B]
    int* any_active;          // number of problems still iterating
    Scale w0;                 // kb_dots: weight D on the first product of scaled problems
};

// Per chunk partial sums -> per problem FP64 sums (chunk order) -> op and CG bookkeeping.
template <int W>
__device__ void batch_finish(const DotArgs& d, double (&s)[W]) {
    __shared__ bool is_last;
    __shared__ int s_any;
    block_sum<W>(s);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int w = 0; w < W; ++w) d.part[blockIdx.x * 4 + w] = s[w];
        __threadfence();
        is_last = atomicAdd(d.counter, 1u) == gridDim.x - 1;
        s_any = 0;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    for (int b = threadIdx.x; b < d.B; b += blockDim.x) {
        const bool in = d.post == POST_START ? (d.lm_active == nullptr || d.lm_active[b] != 0)
                                             : (d.mask == nullptr || d.mask[b] != 0);
        if (!in) {
            if (d.post == POST_START) d.mask[b] = 0;   // problems not solving take no CG iteration
            continue;
        }
        double t[W];
#pragma unroll
        for (int w = 0; w < W; ++w) t[w] = 0.0;
        for (int q = d.chunk_first[b]; q < d.chunk_first[b + 1]; ++q)
#pragma unroll
            for (int w = 0; w < W; ++w) t[w] += __ldcg(d.part + q * 4 + w);
        double* sc = d.sc + (size_t)b * S_COUNT;
        apply_final_op(t, W, sc, d.dst, d.op);
        if (d.post == POST_START) {
            d.cg_it[b] = 0;
            const int a = (sc[S_RR] > d.tol2[b] && d.max_cg[b] > 0) ? 1 : 0;
            d.mask[b] = a;
            atomicAdd(&s_any, a);
        } else if (d.post == POST_UPDATE) {
            const int it = ++d.cg_it[b];
            const int a = (sc[S_RR] > d.tol2[b] && it < d.max_cg[b]) ? 1 : 0;
            d.mask[b] = a;
            atomicAdd(&s_any, a);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (d.post != POST_NONE) *d.any_active = s_any;
        *d.counter = 0u;
        __threadfence();
    }
}

// Up to three dot products a_i . b_i per problem into slots [dst, dst + W), then op.
template <int W>
__global__ void kb_dots(DotArgs d, const float2* __restrict__ a0, const float2* __restrict__ b0,
                        const float2* __restrict__ a1, const float2* __restrict__ b1,
                        const float2* __restrict__ a2, const float2* __restrict__ b2) {
    const Chunk c = d.ch[blockIdx.x];
    float f[W];
#pragma unroll
    for (int w = 0; w < W; ++w) f[w] = 0.0f;
    if (!d.mask || d.mask[c.prob]) {
        const bool dsc = d.w0.on(c.prob);
        CHUNK_LOOP(c, g) {
            f[0] += dsc ? d.w0.D[g] * brdot(a0[g], b0[g]) : brdot(a0[g], b0[g]);
            if constexpr (W > 1) f[1] += brdot(a1[g], b1[g]);
            if constexpr (W > 2) f[2] += brdot(a2[g], b2[g]);
        }
    }
    double s[W];
#pragma unroll
    for (int w = 0; w < W; ++w) s[w] = f[w];
    batch_finish<W>(d, s);
}

// (P)CG start: r = -g - q, p = z = M^-1 r with the Jacobi preconditioner M = (1 + lambda) D
// of (G + lambda D) for scaled problems (M = I otherwise), q = lambda D p; r.z and r.r ->
// slots, mask = r.r > tol2.
__global__ void kb_cg_start(DotArgs d, const float2* __restrict__ g, float2* __restrict__ q, float2* __restrict__ r,
                            float2* __restrict__ p, const float* __restrict__ lam, Scale sc) {
    const Chunk c = d.ch[blockIdx.x];
    float frz = 0.0f, frr = 0.0f;
    if (!d.lm_active || d.lm_active[c.prob]) {
        const float l = lam[c.prob];
        const bool dsc = sc.on(c.prob);
        CHUNK_LOOP(c, i) {
            const float2 gi = g[i], qi = q[i];
            const float2 ri = make_float2(-gi.x - qi.x, -gi.y - qi.y);
            const float di = dsc ? sc.D[i] : 1.0f;
            const float m = dsc ? 1.0f / ((1.0f + l) * di) : 1.0f;
            const float2 zi = make_float2(m * ri.x, m * ri.y);
            r[i] = ri;
            p[i] = zi;
            q[i] = make_float2(l * di * zi.x, l * di * zi.y);
            frz += brdot(ri, zi);
            frr += brdot(ri, ri);
        }
    }
    double s[2] = {frz, frr};
    batch_finish<2>(d, s);
}

// x += alpha p, r -= alpha q; new r.z (z = M^-1 r) and r.r -> beta, mask = r.r > tol2 and
// iterations < max.
__global__ void kb_cg_update(DotArgs d, float2* __restrict__ x, float2* __restrict__ r, const float2* __restrict__ p,
                             const float2* __restrict__ q, const float* __restrict__ lam, Scale sc) {
    const Chunk c = d.ch[blockIdx.x];
    float frz = 0.0f, frr = 0.0f;
    if (d.mask[c.prob]) {
        const float alpha = (float)d.sc[(size_t)c.prob * S_COUNT + S_ALPHA];
        const float l1 = 1.0f + lam[c.prob];
        const bool dsc = sc.on(c.prob);
        CHUNK_LOOP(c, i) {
            const float2 pi = p[i], qi = q[i];
            float2 xi = x[i], ri = r[i];
            xi.x += alpha * pi.x;
            xi.y += alpha * pi.y;
            ri.x -= alpha * qi.x;
            ri.y -= alpha * qi.y;
            x[i] = xi;
            r[i] = ri;
            const float rr = brdot(ri, ri);
            frr += rr;
            frz += dsc ? rr / (l1 * sc.D[i]) : rr;
        }
    }
    double s[2] = {frz, frr};
    batch_finish<2>(d, s);
}

// p = M^-1 r + beta p, q = lambda D p (the next product's damping term).
__global__ void kb_cg_direction(const Chunk* ch, const int* mask, const double* sc, const float2* __restrict__ r,
                                float2* __restrict__ p, float2* __restrict__ q, const float* __restrict__ lam,
                                Scale dsc_) {
    const Chunk c = ch[blockIdx.x];
    if (!mask[c.prob]) return;
    const float beta = (float)sc[(size_t)c.prob * S_COUNT + S_BETA];
    const float l = lam[c.prob];
    const bool dsc = dsc_.on(c.prob);
    CHUNK_LOOP(c, i) {
        const float2 ri = r[i], pi = p[i];
        const float di = dsc ? dsc_.D[i] : 1.0f;
        const float m = dsc ? 1.0f / ((1.0f + l) * di) : 1.0f;
        const float2 pn = make_float2(m * ri.x + beta * pi.x, m * ri.y + beta * pi.y);
        p[i] = pn;
        q[i] = make_float2(l * di * pn.x, l * di * pn.y);
    }
}

// Object-error sums Re/Im conj(O) R, |O|^2, |R|^2 over masked pixels, per problem.
__global__ void kb_err_sums(DotArgs d, const float2* __restrict__ O, const float2* __restrict__ R,
                            const uint8_t* __restrict__ pix) {
    const Chunk c = d.ch[blockIdx.x];
    float f[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (!d.mask || d.mask[c.prob]) {
        CHUNK_LOOP(c, i) {
            if (pix && !pix[i]) continue;
            const float2 o = O[i], rr = R[i];
            f[0] += o.x * rr.x + o.y * rr.y;
            f[1] += o.x * rr.y - o.y * rr.x;
            f[2] += o.x * o.x + o.y * o.y;
            f[3] += rr.x * rr.x + rr.y * rr.y;
        }
    }
    double s[4] = {f[0], f[1], f[2], f[3]};
    batch_finish<4>(d, s);
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------------------
struct ptylm_batch {
    int B = 0;
    std::vector<ptylm_desc> d;
    std::vector<long> off;               // [B + 1] z offsets
    long total = 0;
    cudaStream_t user_stream = nullptr;  // the caller's stream (ordered with ours at every call)
    cudaStream_t stream = nullptr;       // own non-blocking stream (capturable)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    int device = 0, num_sms = 0, grid = 0;
    std::vector<void*> allocs;

    std::vector<BatchProblem> hprobs;
    BatchProblem* probs = nullptr;
    BatchItem* items = nullptr;
    int n_items = 0, items_cap = 0;
    unsigned* counters = nullptr;        // [0] work, [1] done, [2] dot counter, [3] bad-measurement flag
    float2* tw = nullptr;
    double* f = nullptr;                 // [B][2]
    int* lm_active = nullptr;            // [B] problems still running their LM
    int* relin = nullptr;                // [B] problems whose linearisation is recomputed
    int* accept = nullptr;               // [B] problems whose trial point is accepted
    int* cg_active = nullptr;            // [B]
    int* cg_it = nullptr;                // [B]
    int* any_active = nullptr;           // [1]
    float* lam = nullptr;                // [B]
    double* tol2 = nullptr;              // [B]
    int* max_cg = nullptr;               // [B]
    double* scal = nullptr;              // [B][S_COUNT]
    Chunk* chunks = nullptr;
    int n_chunks = 0;
    int* chunk_first = nullptr;          // [B + 1]
    double* part = nullptr;              // [n_chunks][4]
    float2 *z = nullptr, *grad = nullptr, *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *trial = nullptr;
    float2* ref = nullptr;               // concatenated reference objects (lm_solve)
    uint8_t* pix = nullptr;              // concatenated error masks (lm_solve)
    float* D = nullptr;                  // [total] closed-form GGN diagonals (PLM scaling)
    unsigned* dmax = nullptr;            // [B] their maxima (float bits)
    int* scaled = nullptr;               // [B] problems whose LM runs with D = Dg(G)
    float* dfloor = nullptr;             // [B] floor of each problem's diagonal, relative to its maximum
    int* pos_first = nullptr;            // [B + 1] prefix sums of the position counts
    int total_pos = 0;

    // pinned host mirrors
    double* h_scal = nullptr;            // [B][S_COUNT]
    double* h_f = nullptr;               // [B][2]
    int* h_int = nullptr;                // [2B + 2] staging for masks / counters

    bool has_lin = false;
    int order = 0, per_team = 1;
    int le32 = 5, le64 = 5;              // FFT tile (log2 values per thread) of the 32^2 / 64^2 problems
    bool tuned = false;
    std::vector<float> tune_ms;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    long long launches = 0;
};

namespace {

ptylm_status balloc(ptylm_batch* bt, void** p, size_t bytes, const char* what) {
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bfail(PTYLM_ERR_NOMEM, "cudaMalloc(%zu) for %s failed: %s", bytes, what, cudaGetErrorString(e));
    }
    bt->allocs.push_back(*p);
    return PTYLM_OK;
}

template <class T>
ptylm_status balloc_t(ptylm_batch* bt, T** p, size_t count, const char* what) {
    void* q = nullptr;
    ptylm_status s = balloc(bt, &q, count * sizeof(T), what);
    *p = static_cast<T*>(q);
    return s;
}

void bfree_all(ptylm_batch* bt) {
    if (bt->graph_exec) cudaGraphExecDestroy(bt->graph_exec);
    if (bt->graph) cudaGraphDestroy(bt->graph);
    for (void* p : bt->allocs) cudaFree(p);
    bt->allocs.clear();
    if (bt->h_scal) cudaFreeHost(bt->h_scal);
    if (bt->h_f) cudaFreeHost(bt->h_f);
    if (bt->h_int) cudaFreeHost(bt->h_int);
    if (bt->ev_in) cudaEventDestroy(bt->ev_in);
    if (bt->ev_out) cudaEventDestroy(bt->ev_out);
    if (bt->stream) cudaStreamDestroy(bt->stream);
}

int ls_of(int m) { return m == 32 ? 5 : (m == 64 ? 6 : (m == 128 ? 7 : 0)); }

// Work items of every problem.  order 0: largest patches first (longest-processing-time
// order; every item of a probe side costs the same), problems in index order within a side;
// order 1: round robin over the problems.  per_team: positions each team handles per item.
std::vector<BatchItem> build_items(const ptylm_batch* bt, int order, int per_team) {
    std::vector<std::vector<BatchItem>> per(bt->B);
    for (int b = 0; b < bt->B; ++b) {
        const int S = bt->d[b].my;
        const int teams = BATCH_THREADS / ((S * S) >> bt->hprobs[b].LE);
        const int span = teams * per_team;
        for (int k0 = 0; k0 < bt->d[b].K; k0 += span) per[b].push_back(BatchItem{b, k0, per_team, 0});
    }
    std::vector<BatchItem> out;
    if (order == 0) {
        for (int LS = 7; LS >= 5; --LS)
            for (int b = 0; b < bt->B; ++b)
                if (ls_of(bt->d[b].my) == LS) out.insert(out.end(), per[b].begin(), per[b].end());
    } else {
        size_t longest = 0;
        for (auto& v : per) longest = std::max(longest, v.size());
        for (size_t i = 0; i < longest; ++i)
            for (int b = 0; b < bt->B; ++b)
                if (i < per[b].size()) out.push_back(per[b][i]);
    }
    return out;
}

ptylm_status upload_items(ptylm_batch* bt, int order, int per_team) {
    std::vector<BatchItem> it = build_items(bt, order, per_team);
    if ((int)it.size() > bt->items_cap) return bfail(PTYLM_ERR_ARG, "internal: work list larger than its buffer");
    if (!it.empty())
        BCUDA_TRY(cudaMemcpyAsync(bt->items, it.data(), sizeof(BatchItem) * it.size(), cudaMemcpyHostToDevice, bt->stream));
    bt->n_items = (int)it.size();
    bt->order = order;
    bt->per_team = per_team;
    return PTYLM_OK;
}

ptylm_status upload_probs(ptylm_batch* bt) {
    BCUDA_TRY(cudaMemcpyAsync(bt->probs, bt->hprobs.data(), sizeof(BatchProblem) * bt->B, cudaMemcpyHostToDevice,
                              bt->stream));
    return PTYLM_OK;
}

ptylm_status upload_mask(ptylm_batch* bt, int* dev, const std::vector<int>& h) {
    std::copy(h.begin(), h.end(), bt->h_int);
    BCUDA_TRY(cudaMemcpyAsync(dev, bt->h_int, sizeof(int) * bt->B, cudaMemcpyHostToDevice, bt->stream));
    // the pinned staging buffer is reused by the next upload: wait for this one
    BCUDA_TRY(cudaStreamSynchronize(bt->stream));
    return PTYLM_OK;
}

BatchArgs batch_args(ptylm_batch* bt, const float2* V, float2* out, const int* active) {
    BatchArgs a;
    a.probs = bt->probs;
    a.items = bt->items;
    a.n_items = bt->n_items;
    a.work = bt->counters;
    a.done = bt->counters + 1;
    a.tw = bt->tw;
    a.V = V;
    a.out = out;
    a.f = bt->f;
    a.active = active;
    return a;
}

ptylm_status launch_batch(ptylm_batch* bt, int kernel, const float2* V, float2* out, const int* active) {
    if (bt->n_items == 0) return PTYLM_OK;
    BCUDA_TRY(batch_launch(kernel, batch_args(bt, V, out, active), bt->grid, bt->stream));
    ++bt->launches;
    return PTYLM_OK;
}

DotArgs dot_args(ptylm_batch* bt, int* mask, int dst, int op, int post = POST_NONE) {
    DotArgs d;
    d.ch = bt->chunks;
    d.chunk_first = bt->chunk_first;
    d.B = bt->B;
    d.mask = mask;
    d.part = bt->part;
    d.counter = bt->counters + 2;
    d.sc = bt->scal;
    d.dst = dst;
    d.op = op;
    d.post = post;
    d.cg_it = bt->cg_it;
    d.lm_active = bt->lm_active;
    d.tol2 = bt->tol2;
    d.max_cg = bt->max_cg;
    d.any_active = bt->any_active;
    d.w0 = Scale{nullptr, nullptr};
    return d;
}

Scale scale_of(ptylm_batch* bt) { return Scale{bt->D, bt->scaled}; }

ptylm_status vec_ok(ptylm_batch* bt) {
    ++bt->launches;
    BCUDA_TRY(cudaGetLastError());
    return PTYLM_OK;
}

// Forward (+ cache and gradient) of the problems in `mask` at the batch vector V.
ptylm_status batch_forward(ptylm_batch* bt, const float2* V, int cache, int* mask) {
    BCUDA_TRY(cudaMemsetAsync(bt->f, 0, sizeof(double) * 2 * bt->B, bt->stream));
    if (cache) {
        kb_zero<<<bt->n_chunks, BVEC_THREADS, 0, bt->stream>>>(bt->chunks, mask, bt->grad);
        BSTATUS_TRY(vec_ok(bt));
    }
    return launch_batch(bt, cache ? BK_FWD_CACHE : BK_FWD_LOSS, V, cache ? bt->grad : nullptr, mask);
}

// FFT tiles of the 32^2 and 64^2 problems (log2 of the values per thread, 5 or 4).  A change
// moves those problems' measurements into the new tile's team-register order (through their
// cache buffers, which the new tile rewrites anyway) and, when a linearisation point exists,
// recomputes its cache, gradient and metric at z in the new layout.
ptylm_status set_tiles(ptylm_batch* bt, int le32, int le64) {
    bool changed = false;
    for (int b = 0; b < bt->B; ++b) {
        BatchProblem& p = bt->hprobs[b];
        const int want = p.LS == 5 ? le32 : (p.LS == 6 ? le64 : 5);
        if (p.LE == want) continue;
        if (p.K > 0) {
            const size_t bytes = sizeof(float) * ((size_t)p.K << (2 * p.LS));
            float* tmp = reinterpret_cast<float*>(p.a_cache);
            BCUDA_TRY(cudaMemcpyAsync(tmp, p.y, bytes, cudaMemcpyDeviceToDevice, bt->stream));
            const int blocks = std::min(bt->num_sms * 8, std::max(1, (int)(((long)p.K << (2 * p.LS)) / 256)));
            BCUDA_TRY(batch_relayout_measurements(p.LS, p.LE, want, tmp, const_cast<float*>(p.y), p.K, blocks,
                                                  bt->stream));
        }
        p.LE = want;
        changed = true;
    }
    bt->le32 = le32;
    bt->le64 = le64;
    if (!changed) return PTYLM_OK;
    BSTATUS_TRY(upload_probs(bt));
    BSTATUS_TRY(upload_items(bt, bt->order, bt->per_team));
    if (bt->has_lin) BSTATUS_TRY(batch_forward(bt, bt->z, 1, nullptr));
    return PTYLM_OK;
}

// Closed-form Dg(G) of the problems in `mask` at their linearisation point, each floored at
// floors[b] times its maximum (host array of B values; 0: no floor).
ptylm_status batch_diag(ptylm_batch* bt, const int* mask, const std::vector<float>& floors) {
    kb_dzero<<<bt->n_chunks, BVEC_THREADS, 0, bt->stream>>>(bt->chunks, mask, bt->D);
    BSTATUS_TRY(vec_ok(bt));
    BCUDA_TRY(batch_diag_launch(bt->probs, bt->pos_first, bt->B, bt->total_pos, mask, bt->D, bt->stream));
    ++bt->launches;
    BCUDA_TRY(cudaMemcpyAsync(bt->dfloor, floors.data(), sizeof(float) * bt->B, cudaMemcpyHostToDevice, bt->stream));
    BCUDA_TRY(cudaMemsetAsync(bt->dmax, 0, sizeof(unsigned) * bt->B, bt->stream));
    kb_dmax<<<bt->n_chunks, BVEC_THREADS, 0, bt->stream>>>(bt->chunks, mask, bt->D, bt->dmax);
    BSTATUS_TRY(vec_ok(bt));
    kb_dfloor<<<bt->n_chunks, BVEC_THREADS, 0, bt->stream>>>(bt->chunks, mask, bt->dmax, bt->dfloor, bt->D);
    BSTATUS_TRY(vec_ok(bt));
    BCUDA_TRY(cudaStreamSynchronize(bt->stream));   // floors is a pageable host buffer
    return PTYLM_OK;
}

ptylm_status read_f_and_scalars(ptylm_batch* bt) {
    BCUDA_TRY(cudaMemcpyAsync(bt->h_f, bt->f, sizeof(double) * 2 * bt->B, cudaMemcpyDeviceToHost, bt->stream));
    BCUDA_TRY(cudaMemcpyAsync(bt->h_scal, bt->scal, sizeof(double) * S_COUNT * bt->B, cudaMemcpyDeviceToHost,
                              bt->stream));
    BCUDA_TRY(cudaStreamSynchronize(bt->stream));
    return PTYLM_OK;
}

// One CG iteration of every problem with cg_active set (the captured sequence).
ptylm_status cg_iteration(ptylm_batch* bt) {
    BSTATUS_TRY(launch_batch(bt, BK_MATVEC, bt->p, bt->q, bt->cg_active));            // q += G p
    kb_dots<1><<<bt->n_chunks, BVEC_THREADS, 0, bt->stream>>>(dot_args(bt, bt->cg_active, S_PAP, OP_ALPHA), bt->p,
                                                              bt->q, nullptr, nullptr, nullptr, nullptr);
    BSTATUS_TRY(vec_ok(bt));                                                             // alpha
    kb_cg_update<<<bt->n_chunks, BVEC_THREADS, 0, bt->stream>>>(dot_args(bt, bt->cg_active, 0, OP_BETA, POST_UPDATE),
                                                                bt->x, bt->r, bt->p, bt->q, bt->lam, scale_of(bt));
    BSTATUS_TRY(vec_ok(bt));                                                             // x, r, beta
    kb_cg_direction<<<bt->n_chunks, BVEC_THREADS, 0, bt->stream>>>(bt->chunks, bt->cg_active, bt->scal, bt->r, bt->p,
                                                                   bt->q, bt->lam, scale_of(bt));
    return vec_ok(bt);                                                                   // p, q = lambda p
}

ptylm_status capture_graph(ptylm_batch* bt) {
    if (bt->graph_exec) {
        cudaGraphExecDestroy(bt->graph_exec);
        bt->graph_exec = nullptr;
    }
    if (bt->graph) {
        cudaGraphDestroy(bt->graph);
        bt->graph = nullptr;
    }
    BCUDA_TRY(cudaStreamBeginCapture(bt->stream, cudaStreamCaptureModeThreadLocal));
    const long long before = bt->launches;
    ptylm_status s = cg_iteration(bt);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(bt->stream, &g);
    bt->launches = before;
    if (s != PTYLM_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    BCUDA_TRY(e);
    bt->graph = g;
    BCUDA_TRY(cudaGraphInstantiate(&bt->graph_exec, g, 0));
    return PTYLM_OK;
}

// Order our stream after the caller's, and the caller's after ours on the way out.
ptylm_status enter(ptylm_batch* bt) {
    BCUDA_TRY(cudaEventRecord(bt->ev_in, bt->user_stream));
    BCUDA_TRY(cudaStreamWaitEvent(bt->stream, bt->ev_in, 0));
    return PTYLM_OK;
}
ptylm_status leave(ptylm_batch* bt) {
    BCUDA_TRY(cudaEventRecord(bt->ev_out, bt->stream));
    BCUDA_TRY(cudaStreamWaitEvent(bt->user_stream, bt->ev_out, 0));
    return PTYLM_OK;
}

double surrogate_level(const ptylm_lm_params* p, int t) {
    if (p->surrogate_T <= 0 || t >= p->surrogate_T) return 0.0;
    if (p->surrogate_T == 1) return p->surrogate0;
    return p->surrogate0 * std::pow(p->surrogate_end / p->surrogate0, (double)t / (double)(p->surrogate_T - 1));
}

}  // namespace

extern "C" {

ptylm_status ptylm_batch_init(ptylm_batch** out, int B, const ptylm_desc* descs, const int32_t* const* positions_dev,
                              const float* const* y_dev, const ptylm_c64* const* probes_dev, void* stream) {
    set_last_error("");
    if (!out || B <= 0 || !descs || !positions_dev || !y_dev || !probes_dev)
        return bfail(PTYLM_ERR_ARG, "batch, descs, positions, y and probes must be given for B >= 1 problems");
    *out = nullptr;
    for (int b = 0; b < B; ++b) {
        const ptylm_desc& d = descs[b];
        if (d.my != d.mx || !ls_of(d.my)) return bfail(PTYLM_ERR_ARG, "problem %d: probe must be square 32, 64 or 128", b);
        if (d.ny < d.my || d.nx < d.mx) return bfail(PTYLM_ERR_ARG, "problem %d: object smaller than the probe", b);
        if (d.K < 0) return bfail(PTYLM_ERR_ARG, "problem %d: K must be >= 0", b);
        if (d.loss != PTYLM_LOSS_GAUSSIAN && d.loss != PTYLM_LOSS_POISSON) return bfail(PTYLM_ERR_ARG, "problem %d: unknown loss", b);
        if (!(d.background > 0.0f) || !std::isfinite(d.background)) return bfail(PTYLM_ERR_ARG, "problem %d: background must be > 0", b);
        if (d.joint) return bfail(PTYLM_ERR_ARG, "problem %d: batches hold object-only problems", b);
        if (d.K > 0 && (!positions_dev[b] || !y_dev[b])) return bfail(PTYLM_ERR_ARG, "problem %d: positions and y required", b);
        if (!probes_dev[b]) return bfail(PTYLM_ERR_ARG, "problem %d: probe required", b);
    }
    ptylm_batch* bt = new ptylm_batch();
    auto bail = [&](ptylm_status s) {
        bfree_all(bt);
        delete bt;
        return s;
    };
    bt->B = B;
    bt->d.assign(descs, descs + B);
    bt->user_stream = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(bt->user_stream) != cudaSuccess ||   // the caller's inputs are complete
        cudaGetDevice(&bt->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&bt->num_sms, cudaDevAttrMultiProcessorCount, bt->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&bt->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&bt->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&bt->ev_out, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return bail(bfail(PTYLM_ERR_CUDA, "no usable CUDA device"));
    }
    int per_sm = 0;
    if (batch_prepare(&per_sm) != cudaSuccess || per_sm <= 0) {
        cudaGetLastError();
        return bail(bfail(PTYLM_ERR_CUDA, "batch kernels cannot launch"));
    }
    bt->grid = per_sm * bt->num_sms;
    bt->off.assign(B + 1, 0);
    std::vector<Chunk> hch;
    std::vector<int> hfirst(B + 1, 0);
    int max_items = 0;
    for (int b = 0; b < B; ++b) {
        const long N = (long)descs[b].ny * descs[b].nx;
        bt->off[b + 1] = bt->off[b] + N;
        hfirst[b] = (int)hch.size();
        for (long s = 0; s < N; s += CHUNK) hch.push_back(Chunk{bt->off[b] + s, (int)std::min<long>(CHUNK, N - s), b});
        // the smallest team count of any tile the autotuner may pick for this side (16 values
        // per thread for sides 32 and 64) bounds the number of items
        const int S = descs[b].my, teams = BATCH_THREADS / (S * S / (S <= 64 ? 16 : 32));
        max_items += (descs[b].K + teams - 1) / teams;
    }
    hfirst[B] = (int)hch.size();
    bt->total = bt->off[B];
    bt->n_chunks = (int)hch.size();
    bt->items_cap = std::max(1, max_items);

    ptylm_status s;
#define BA(ptr, n, what) if ((s = balloc_t(bt, &(ptr), (n), what)) != PTYLM_OK) return bail(s)
    BA(bt->probs, B, "problem table");
    BA(bt->items, bt->items_cap, "work items");
    BA(bt->counters, 4, "counters");
    BA(bt->tw, BATCH_TW, "twiddles");
    BA(bt->f, 2 * B, "error metrics");
    BA(bt->lm_active, B, "masks");
    BA(bt->relin, B, "masks");
    BA(bt->accept, B, "masks");
    BA(bt->cg_active, B, "masks");
    BA(bt->cg_it, B, "CG counts");
    BA(bt->any_active, 1, "CG count");
    BA(bt->lam, B, "damping");
    BA(bt->tol2, B, "CG tolerances");
    BA(bt->max_cg, B, "CG limits");
    BA(bt->scal, (size_t)B * S_COUNT, "scalars");
    BA(bt->chunks, bt->n_chunks, "chunks");
    BA(bt->chunk_first, B + 1, "chunk ranges");
    BA(bt->part, (size_t)bt->n_chunks * 4, "partials");
    BA(bt->z, bt->total, "iterate");
    BA(bt->grad, bt->total, "gradient");
    BA(bt->x, bt->total, "CG x");
    BA(bt->r, bt->total, "CG r");
    BA(bt->p, bt->total, "CG p");
    BA(bt->q, bt->total, "CG q");
    BA(bt->trial, bt->total, "trial point");
    BA(bt->D, bt->total, "GGN diagonals");
    BA(bt->dmax, B, "diagonal maxima");
    BA(bt->scaled, B, "scaling flags");
    BA(bt->dfloor, B, "diagonal floors");
    BA(bt->pos_first, B + 1, "position offsets");
#undef BA
    if (cudaMallocHost((void**)&bt->h_scal, sizeof(double) * S_COUNT * B) != cudaSuccess ||
        cudaMallocHost((void**)&bt->h_f, sizeof(double) * 2 * B) != cudaSuccess ||
        cudaMallocHost((void**)&bt->h_int, sizeof(int) * (2 * B + 2)) != cudaSuccess) {
        cudaGetLastError();
        return bail(bfail(PTYLM_ERR_NOMEM, "pinned host buffers"));
    }

    // per-problem data: positions (validated on the host), measurements (validated on the
    // device: counters[3] is set by any negative or non-finite entry), probe, cache
    if (cudaMemsetAsync(bt->counters, 0, sizeof(unsigned) * 4, bt->stream) != cudaSuccess) {
        cudaGetLastError();
        return bail(bfail(PTYLM_ERR_CUDA, "clearing batch counters"));
    }
    bt->hprobs.resize(B);
    for (int b = 0; b < B; ++b) {
        const ptylm_desc& d = descs[b];
        const int LS = ls_of(d.my), M = d.my * d.mx;
        BatchProblem& p = bt->hprobs[b];
        memset(&p, 0, sizeof p);
        p.K = d.K;
        p.nx = d.nx;
        p.LS = LS;
        p.loss = d.loss;
        p.b = d.background;
        p.LE = 5;
        p.z_off = bt->off[b];
        int2* pos = nullptr;
        float* y = nullptr;
        float2 *ac = nullptr, *P = nullptr;
        if ((s = balloc_t(bt, &pos, std::max(1, d.K), "positions")) != PTYLM_OK) return bail(s);
        if ((s = balloc_t(bt, &y, (size_t)std::max(1, d.K) * M, "measurements")) != PTYLM_OK) return bail(s);
        if ((s = balloc_t(bt, &ac, (size_t)std::max(1, d.K) * M, "frequency cache")) != PTYLM_OK) return bail(s);
        // per-thread d2l sums: T = M / E threads per position, E >= 16 for every tile
        float* trp = nullptr;
        if ((s = balloc_t(bt, &trp, (size_t)std::max(1, d.K) * (M / 16), "diagonal partials")) != PTYLM_OK)
            return bail(s);
        p.trp = trp;
        if ((s = balloc_t(bt, &P, M, "probe")) != PTYLM_OK) return bail(s);
        std::vector<int32_t> hp(2 * (size_t)std::max(1, d.K), 0);
        if (d.K > 0 && cudaMemcpy(hp.data(), positions_dev[b], sizeof(int32_t) * 2 * d.K, cudaMemcpyDefault) != cudaSuccess) {
            cudaGetLastError();
            return bail(bfail(PTYLM_ERR_ARG, "problem %d: positions are not readable device memory", b));
        }
        for (int k = 0; k < d.K; ++k)
            if (hp[2 * k] < 0 || hp[2 * k + 1] < 0 || hp[2 * k] + d.my > d.ny || hp[2 * k + 1] + d.mx > d.nx)
                return bail(bfail(PTYLM_ERR_ARG, "problem %d: position %d (%d, %d) outside the object", b, k, hp[2 * k],
                                  hp[2 * k + 1]));
        if (cudaMemcpy(pos, hp.data(), sizeof(int32_t) * hp.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(P, probes_dev[b], sizeof(float2) * M, cudaMemcpyDefault) != cudaSuccess) {
            cudaGetLastError();
            return bail(bfail(PTYLM_ERR_CUDA, "problem %d: copying positions / probe", b));
        }
        if (d.K > 0) {
            cudaError_t e = permute_measurements(LS, 5, y_dev[b], y, d.K, d.loss == PTYLM_LOSS_GAUSSIAN,
                                                 std::min(bt->num_sms * 8, std::max(1, (int)((long)d.K * M / 256))),
                                                 bt->stream, bt->counters + 3);
            if (e != cudaSuccess) return bail(bfail(PTYLM_ERR_CUDA, "problem %d: measurements: %s", b, cudaGetErrorString(e)));
        }
        p.pos = pos;
        p.y = y;
        p.a_cache = ac;
        p.P = P;
    }
    std::vector<int> hpf(B + 1, 0);
    for (int b = 0; b < B; ++b) hpf[b + 1] = hpf[b] + descs[b].K;
    bt->total_pos = hpf[B];
    std::vector<float2> htw(BATCH_TW);
    int o = 0;
    for (int S : {32, 64, 128})
        for (int j = 0; j < S; ++j, ++o) {
            const double ang = 2.0 * M_PI * (double)j / (double)S;   // W_S^j = exp(-2 pi i j / S)
            htw[o] = make_float2((float)std::cos(ang), (float)-std::sin(ang));
        }
    if (cudaMemcpyAsync(bt->tw, htw.data(), sizeof(float2) * BATCH_TW, cudaMemcpyHostToDevice, bt->stream) != cudaSuccess ||
        cudaMemcpyAsync(bt->chunks, hch.data(), sizeof(Chunk) * hch.size(), cudaMemcpyHostToDevice, bt->stream) != cudaSuccess ||
        cudaMemcpyAsync(bt->chunk_first, hfirst.data(), sizeof(int) * (B + 1), cudaMemcpyHostToDevice, bt->stream) != cudaSuccess ||
        cudaMemsetAsync(bt->counters, 0, sizeof(unsigned) * 3, bt->stream) != cudaSuccess ||
        cudaMemsetAsync(bt->scal, 0, sizeof(double) * S_COUNT * B, bt->stream) != cudaSuccess ||
        cudaMemcpyAsync(bt->pos_first, hpf.data(), sizeof(int) * (B + 1), cudaMemcpyHostToDevice, bt->stream) != cudaSuccess ||
        cudaMemsetAsync(bt->scaled, 0, sizeof(int) * B, bt->stream) != cudaSuccess) {
        cudaGetLastError();
        return bail(bfail(PTYLM_ERR_CUDA, "uploading batch tables"));
    }
    if ((s = upload_probs(bt)) != PTYLM_OK || (s = upload_items(bt, 0, 1)) != PTYLM_OK) return bail(s);
    if (cudaMemcpyAsync(bt->h_int, bt->counters + 3, sizeof(unsigned), cudaMemcpyDeviceToHost, bt->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(bt->stream) != cudaSuccess) {
        cudaGetLastError();
        return bail(bfail(PTYLM_ERR_CUDA, "batch initialisation"));
    }
    if (bt->h_int[0] != 0) return bail(bfail(PTYLM_ERR_ARG, "measurements y must be finite and >= 0"));
    *out = bt;
    return PTYLM_OK;
}

long ptylm_batch_offset(const ptylm_batch* bt, int b) {
    if (!bt || b < 0 || b > bt->B) return -1;
    return bt->off[b];
}

ptylm_status ptylm_batch_forward_loss(ptylm_batch* bt, const ptylm_c64* O, double* f_host, double* dl_norm2_host,
                                      int cache) {
    set_last_error("");
    if (!bt || !O) return bfail(PTYLM_ERR_ARG, "batch and O must be non-NULL");
    BSTATUS_TRY(enter(bt));
    const float2* V = reinterpret_cast<const float2*>(O);
    if (cache) {
        BCUDA_TRY(cudaMemcpyAsync(bt->z, V, sizeof(float2) * bt->total, cudaMemcpyDeviceToDevice, bt->stream));
        V = bt->z;
    }
    BSTATUS_TRY(batch_forward(bt, V, cache, nullptr));
    BCUDA_TRY(cudaMemcpyAsync(bt->h_f, bt->f, sizeof(double) * 2 * bt->B, cudaMemcpyDeviceToHost, bt->stream));
    BCUDA_TRY(cudaStreamSynchronize(bt->stream));
    for (int b = 0; b < bt->B; ++b) {
        if (f_host) f_host[b] = bt->h_f[2 * b];
        if (dl_norm2_host) dl_norm2_host[b] = bt->h_f[2 * b + 1];
    }
    if (cache) bt->has_lin = true;
    return leave(bt);
}

ptylm_status ptylm_batch_gradient(ptylm_batch* bt, ptylm_c64* g) {
    set_last_error("");
    if (!bt || !g) return bfail(PTYLM_ERR_ARG, "batch and g must be non-NULL");
    if (!bt->has_lin) return bfail(PTYLM_ERR_STATE, "no linearisation point (ptylm_batch_forward_loss with cache=1)");
    BSTATUS_TRY(enter(bt));
    BCUDA_TRY(cudaMemcpyAsync(g, bt->grad, sizeof(float2) * bt->total, cudaMemcpyDeviceToDevice, bt->stream));
    return leave(bt);
}

ptylm_status ptylm_batch_ggn_matvec(ptylm_batch* bt, const ptylm_c64* v, ptylm_c64* out, const double* lambda) {
    set_last_error("");
    if (!bt || !v || !out) return bfail(PTYLM_ERR_ARG, "batch, v and out must be non-NULL");
    if (!bt->has_lin) return bfail(PTYLM_ERR_STATE, "no linearisation point (ptylm_batch_forward_loss with cache=1)");
    BSTATUS_TRY(enter(bt));
    std::vector<float> hl(bt->B, 0.0f);
    if (lambda)
        for (int b = 0; b < bt->B; ++b) {
            if (!std::isfinite(lambda[b])) return bfail(PTYLM_ERR_ARG, "lambda[%d] must be finite", b);
            hl[b] = (float)lambda[b];
        }
    BCUDA_TRY(cudaMemcpyAsync(bt->lam, hl.data(), sizeof(float) * bt->B, cudaMemcpyHostToDevice, bt->stream));
    const float2* V = reinterpret_cast<const float2*>(v);
    float2* O = reinterpret_cast<float2*>(out);
    kb_damp<<<bt->n_chunks, BVEC_THREADS, 0, bt->stream>>>(bt->chunks, nullptr, bt->lam, V, O, Scale{nullptr, nullptr});
    BSTATUS_TRY(vec_ok(bt));
    BSTATUS_TRY(launch_batch(bt, BK_MATVEC, V, O, nullptr));
    BCUDA_TRY(cudaStreamSynchronize(bt->stream));   // hl is a pageable host buffer
    return leave(bt);
}

ptylm_status ptylm_batch_ggn_diag(ptylm_batch* bt, float* D_out, double floor_rel) {
    set_last_error("");
    if (!bt || !D_out) return bfail(PTYLM_ERR_ARG, "batch and D_out must be non-NULL");
    if (!(floor_rel >= 0.0) || !(floor_rel < 1.0)) return bfail(PTYLM_ERR_ARG, "floor_rel must be in [0, 1)");
    if (!bt->has_lin) return bfail(PTYLM_ERR_STATE, "no linearisation point (ptylm_batch_forward_loss with cache=1)");
    BSTATUS_TRY(enter(bt));
    BSTATUS_TRY(batch_diag(bt, nullptr, std::vector<float>(bt->B, (float)floor_rel)));
    BCUDA_TRY(cudaMemcpyAsync(D_out, bt->D, sizeof(float) * bt->total, cudaMemcpyDefault, bt->stream));
    return leave(bt);
}

// Schedules of the autotuner: index = sched + 6 * (t32 + 2 * t64) with sched = (order,
// positions per team per item) from kSched, t32 / t64 = 1 when the 32^2 / 64^2 problems run
// the 16-values-per-thread FFT tile.
constexpr int kSched[6][2] = {{0, 1}, {0, 2}, {0, 4}, {1, 1}, {1, 2}, {1, 4}};
constexpr int kSchedules = 24;

ptylm_status apply_schedule(ptylm_batch* bt, int c) {
    const int sched = c % 6, t32 = (c / 6) & 1, t64 = c / 12;
    bt->order = kSched[sched][0];
    bt->per_team = kSched[sched][1];
    BSTATUS_TRY(set_tiles(bt, t32 ? 4 : 5, t64 ? 4 : 5));
    return upload_items(bt, kSched[sched][0], kSched[sched][1]);
}

ptylm_status ptylm_batch_tune(ptylm_batch* bt, int* choice, float* ms, int n_ms) {
    set_last_error("");
    if (!bt) return bfail(PTYLM_ERR_ARG, "batch must be non-NULL");
    if (!bt->has_lin) return bfail(PTYLM_ERR_STATE, "no linearisation point (ptylm_batch_forward_loss with cache=1)");
    BSTATUS_TRY(enter(bt));
    bool has32 = false, has64 = false;
    for (int b = 0; b < bt->B; ++b) {
        has32 |= bt->hprobs[b].LS == 5 && bt->hprobs[b].K > 0;
        has64 |= bt->hprobs[b].LS == 6 && bt->hprobs[b].K > 0;
    }
    cudaEvent_t e0, e1;
    BCUDA_TRY(cudaEventCreate(&e0));
    BCUDA_TRY(cudaEventCreate(&e1));
    int best = 0;
    float best_ms = 1e30f;
    bt->tune_ms.assign(kSchedules, -1.0f);
    ptylm_status s = PTYLM_OK;
    // tiles in the outer loop: a tile change relinearises, a schedule change only rebuilds
    // the work list; tiles that no problem of the batch uses are not timed (entry -1)
    for (int tile = 0; tile < 4 && s == PTYLM_OK; ++tile) {
        if (((tile & 1) && !has32) || ((tile & 2) && !has64)) continue;
        for (int sched = 0; sched < 6 && s == PTYLM_OK; ++sched) {
            const int c = sched + 6 * tile;
            if ((s = apply_schedule(bt, c)) != PTYLM_OK) break;
            if ((s = launch_batch(bt, BK_MATVEC, bt->grad, bt->q, nullptr)) != PTYLM_OK) break;   // warm-up
            cudaEventRecord(e0, bt->stream);
            for (int rep = 0; rep < 3 && s == PTYLM_OK; ++rep) s = launch_batch(bt, BK_MATVEC, bt->grad, bt->q, nullptr);
            cudaEventRecord(e1, bt->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) s = bfail(PTYLM_ERR_CUDA, "timing a schedule");
            float t = 0.0f;
            cudaEventElapsedTime(&t, e0, e1);
            bt->tune_ms[c] = t / 3.0f;
            if (bt->tune_ms[c] < best_ms) {
                best_ms = bt->tune_ms[c];
                best = c;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    BSTATUS_TRY(s);
    BSTATUS_TRY(apply_schedule(bt, best));
    bt->tuned = true;
    if (bt->graph_exec) BSTATUS_TRY(capture_graph(bt));
    if (choice) *choice = best;
    for (int c = 0; c < n_ms && c < kSchedules; ++c) ms[c] = bt->tune_ms[c];
    BCUDA_TRY(cudaStreamSynchronize(bt->stream));
    return leave(bt);
}

ptylm_status ptylm_batch_set_schedule(ptylm_batch* bt, int choice) {
    set_last_error("");
    if (!bt || choice < 0 || choice >= kSchedules) return bfail(PTYLM_ERR_ARG, "schedule must be 0..%d", kSchedules - 1);
    BSTATUS_TRY(enter(bt));
    BSTATUS_TRY(apply_schedule(bt, choice));
    bt->tuned = true;
    if (bt->graph_exec) BSTATUS_TRY(capture_graph(bt));
    BCUDA_TRY(cudaStreamSynchronize(bt->stream));
    return leave(bt);
}

ptylm_status ptylm_batch_lm_solve(ptylm_batch* bt, ptylm_c64* O_inout, const ptylm_lm_params* prm,
                                  ptylm_lm_stats* stats) {
    set_last_error("");
    if (!bt || !O_inout || !prm) return bfail(PTYLM_ERR_ARG, "batch, O and params must be non-NULL");
    const int B = bt->B;
    bool want_err = false;
    for (int b = 0; b < B; ++b) {
        const ptylm_lm_params& q = prm[b];
        if (q.max_outer < 0 || q.max_cg < 0 || !(q.kappa > 1.0) || !(q.mu0 > 0.0))
            return bfail(PTYLM_ERR_ARG, "problem %d: invalid LM parameters", b);
        if (q.projected) return bfail(PTYLM_ERR_ARG, "problem %d: batches run Algorithm 1 without Algorithm 2", b);
        if (q.scaled && !(q.diag_floor >= 0.0 && q.diag_floor < 1.0))
            return bfail(PTYLM_ERR_ARG, "problem %d: diag_floor must be in [0, 1)", b);
        if (q.surrogate_T < 0 || (q.surrogate_T > 0 && (!(q.surrogate0 > 0.0) || !(q.surrogate_end > 0.0))))
            return bfail(PTYLM_ERR_ARG, "problem %d: invalid surrogate schedule", b);
        if (q.O_ref) want_err = true;
    }
    BSTATUS_TRY(enter(bt));
    const size_t zbytes = sizeof(float2) * bt->total;
    BCUDA_TRY(cudaMemcpyAsync(bt->z, O_inout, zbytes, cudaMemcpyDeviceToDevice, bt->stream));
    // PLM problems (D = Dg(G), lambda = mu, Jacobi PCG; reading C10) next to LM ones (D = I)
    std::vector<int> scaled_h(B);
    std::vector<float> floors_h(B, 0.0f);
    bool any_scaled = false;
    for (int b = 0; b < B; ++b) {
        scaled_h[b] = prm[b].scaled ? 1 : 0;
        floors_h[b] = prm[b].scaled ? (float)prm[b].diag_floor : 0.0f;
        any_scaled |= scaled_h[b] != 0;
    }
    BSTATUS_TRY(upload_mask(bt, bt->scaled, scaled_h));
    BCUDA_TRY(cudaMemsetAsync(bt->x, 0, zbytes, bt->stream));
    if (want_err) {
        if (!bt->ref) {
            ptylm_status s;
            if ((s = balloc_t(bt, &bt->ref, bt->total, "reference objects")) != PTYLM_OK) return s;
            if ((s = balloc_t(bt, &bt->pix, bt->total, "error masks")) != PTYLM_OK) return s;
        }
        for (int b = 0; b < B; ++b) {
            const long N = bt->off[b + 1] - bt->off[b];
            if (prm[b].O_ref)
                BCUDA_TRY(cudaMemcpyAsync(bt->ref + bt->off[b], prm[b].O_ref, sizeof(float2) * N, cudaMemcpyDeviceToDevice,
                                          bt->stream));
            else
                BCUDA_TRY(cudaMemsetAsync(bt->ref + bt->off[b], 0, sizeof(float2) * N, bt->stream));
            if (prm[b].mask)
                BCUDA_TRY(cudaMemcpyAsync(bt->pix + bt->off[b], prm[b].mask, N, cudaMemcpyDeviceToDevice, bt->stream));
            else
                BCUDA_TRY(cudaMemsetAsync(bt->pix + bt->off[b], 1, N, bt->stream));
        }
    }
    if (!bt->tuned) {
        // the first linearisation is needed to time the schedules on this batch's own work
        BSTATUS_TRY(batch_forward(bt, bt->z, 1, nullptr));
        bt->has_lin = true;
        BCUDA_TRY(cudaStreamSynchronize(bt->stream));
        BSTATUS_TRY(leave(bt));
        BSTATUS_TRY(ptylm_batch_tune(bt, nullptr, nullptr, 0));
        BSTATUS_TRY(enter(bt));
    }
    if (!bt->graph_exec) BSTATUS_TRY(capture_graph(bt));

    // per-problem host state
    std::vector<double> mu(B), f(B, NAN), dl2(B, 0.0), gg(B, 0.0), lambda(B, 0.0), err(B, NAN), f_cur(B, NAN);
    std::vector<int> t(B, 0), done(B, 0), relin(B, 1), cg_total(B, 0), matvecs(B, 0), cg_this(B, 0), hit_max(B, 0);
    std::vector<ptylm_status> st(B, PTYLM_OK);
    for (int b = 0; b < B; ++b) {
        mu[b] = prm[b].mu0;
        if (prm[b].max_outer == 0 || bt->d[b].K == 0) done[b] = 1;
    }
    std::vector<float> hl(B);
    std::vector<double> ht(B);
    std::vector<int> hm(B), active(B), acc(B);
    int max_cg_all = 0;
    for (int b = 0; b < B; ++b) max_cg_all = std::max(max_cg_all, prm[b].fixed_cg > 0 ? prm[b].fixed_cg : prm[b].max_cg);

    for (;;) {
        bool any = false;
        for (int b = 0; b < B; ++b) {
            active[b] = !done[b];
            any |= active[b] != 0;
        }
        if (!any) break;
        // ---- linearise the problems that moved (Algorithm 1, first step) ----
        bool any_relin = false;
        for (int b = 0; b < B; ++b) {
            relin[b] = active[b] && relin[b];
            any_relin |= relin[b] != 0;
            bt->hprobs[b].b = (float)(bt->d[b].background + (active[b] ? surrogate_level(&prm[b], t[b]) : 0.0));
        }
        BSTATUS_TRY(upload_probs(bt));
        BSTATUS_TRY(upload_mask(bt, bt->lm_active, active));
        if (any_relin) {
            BSTATUS_TRY(upload_mask(bt, bt->relin, relin));
            BSTATUS_TRY(batch_forward(bt, bt->z, 1, bt->relin));
            kb_dots<1><<<bt->n_chunks, BVEC_THREADS, 0, bt->stream>>>(dot_args(bt, bt->relin, S_GG, OP_STORE), bt->grad,
                                                                      bt->grad, nullptr, nullptr, nullptr, nullptr);
            BSTATUS_TRY(vec_ok(bt));
            if (any_scaled) {
                std::vector<int> rs(B);
                bool any_rs = false;
                for (int b = 0; b < B; ++b) {
                    rs[b] = relin[b] && scaled_h[b];
                    any_rs |= rs[b] != 0;
                }
                if (any_rs) {   // Dg(G) at the new linearisation point (the accept mask is free here)
                    BSTATUS_TRY(upload_mask(bt, bt->accept, rs));
                    BSTATUS_TRY(batch_diag(bt, bt->accept, floors_h));
                }
            }
            BSTATUS_TRY(read_f_and_scalars(bt));
            for (int b = 0; b < B; ++b) {
                if (!relin[b]) continue;
                f[b] = bt->h_f[2 * b];
                dl2[b] = bt->h_f[2 * b + 1];
                gg[b] = bt->h_scal[(size_t)b * S_COUNT + S_GG];
                if (!std::isfinite(f[b]) || !std::isfinite(gg[b])) {
                    st[b] = PTYLM_ERR_NAN;
                    done[b] = 1;
                    active[b] = 0;
                    continue;
                }
                f_cur[b] = f[b];
                if (stats && stats[b].hist_len > t[b]) {
                    if (stats[b].hist_f) stats[b].hist_f[t[b]] = f[b];
                    if (stats[b].hist_gnorm) stats[b].hist_gnorm[t[b]] = std::sqrt(gg[b]);
                }
                cg_this[b] = 0;
            }
            bt->has_lin = true;
        }
        // ---- damping, CG tolerance (Eqs. lma_termination_eta / _magnitude) ----
        for (int b = 0; b < B; ++b) {
            if (!active[b]) {
                hl[b] = 0.0f;
                ht[b] = 0.0;
                hm[b] = 0;
                continue;
            }
            // lambda = mu ||grad_zeta l||^nu (D = I) or mu (D = Dg(G)), Algorithm 1
            lambda[b] = scaled_h[b] ? mu[b] : mu[b] * std::pow(std::sqrt(dl2[b]), prm[b].nu);
            hl[b] = (float)lambda[b];
            const double gnorm = std::sqrt(gg[b]);
            const double tol = std::min(prm[b].beta, std::sqrt(gnorm)) * gnorm;
            ht[b] = prm[b].fixed_cg > 0 ? -1.0 : tol * tol;
            hm[b] = prm[b].fixed_cg > 0 ? prm[b].fixed_cg : prm[b].max_cg;
        }
        BSTATUS_TRY(upload_mask(bt, bt->lm_active, active));
        BCUDA_TRY(cudaMemcpyAsync(bt->lam, hl.data(), sizeof(float) * B, cudaMemcpyHostToDevice, bt->stream));
        BCUDA_TRY(cudaMemcpyAsync(bt->tol2, ht.data(), sizeof(double) * B, cudaMemcpyHostToDevice, bt->stream));
        BCUDA_TRY(cudaMemcpyAsync(bt->max_cg, hm.data(), sizeof(int) * B, cudaMemcpyHostToDevice, bt->stream));
        // ---- truncated CG on (G + lambda I) x = -g, warm-started from x (C8) ----
        kb_damp<<<bt->n_chunks, BVEC_THREADS, 0, bt->stream>>>(bt->chunks, bt->lm_active, bt->lam, bt->x, bt->q,
                                                               scale_of(bt));
        BSTATUS_TRY(vec_ok(bt));
        BSTATUS_TRY(launch_batch(bt, BK_MATVEC, bt->x, bt->q, bt->lm_active));              // q = (G + lambda) x
        for (int b = 0; b < B; ++b) matvecs[b] += active[b];
        kb_cg_start<<<bt->n_chunks, BVEC_THREADS, 0, bt->stream>>>(dot_args(bt, bt->cg_active, 0, OP_START, POST_START),
                                                                   bt->grad, bt->q, bt->r, bt->p, bt->lam, scale_of(bt));
        BSTATUS_TRY(vec_ok(bt));
        for (int it = 0; it < max_cg_all;) {
            BCUDA_TRY(cudaMemcpyAsync(bt->h_int, bt->any_active, sizeof(int), cudaMemcpyDeviceToHost, bt->stream));
            BCUDA_TRY(cudaStreamSynchronize(bt->stream));
            if (bt->h_int[0] == 0) break;
            const int reps = std::min(4, max_cg_all - it);   // replays between host checks
            for (int k = 0; k < reps; ++k) BCUDA_TRY(cudaGraphLaunch(bt->graph_exec, bt->stream));
            bt->launches += 4LL * reps;
            it += reps;
        }
        BCUDA_TRY(cudaMemcpyAsync(bt->h_int, bt->cg_it, sizeof(int) * B, cudaMemcpyDeviceToHost, bt->stream));
        BCUDA_TRY(cudaStreamSynchronize(bt->stream));
        for (int b = 0; b < B; ++b) {
            if (!active[b]) continue;
            const int n = bt->h_int[b];
            cg_this[b] += n;
            cg_total[b] += n;
            matvecs[b] += n;
            if (prm[b].fixed_cg <= 0 && n >= prm[b].max_cg) hit_max[b] = 1;
        }
        // ---- trial point, its error metric and the gain ratio (Algorithm 1) ----
        kb_axpy<<<bt->n_chunks, BVEC_THREADS, 0, bt->stream>>>(bt->chunks, bt->lm_active, bt->z, bt->x, bt->trial);
        BSTATUS_TRY(vec_ok(bt));
        BSTATUS_TRY(batch_forward(bt, bt->trial, 0, bt->lm_active));
        DotArgs dd_args = dot_args(bt, bt->lm_active, S_DD, OP_STORE);
        dd_args.w0 = scale_of(bt);   // Delta^T D Delta for the scaled problems
        kb_dots<3><<<bt->n_chunks, BVEC_THREADS, 0, bt->stream>>>(dd_args, bt->x,
                                                                  bt->x, bt->x, bt->grad, bt->x, bt->r);
        BSTATUS_TRY(vec_ok(bt));
        BSTATUS_TRY(read_f_and_scalars(bt));
        bool any_acc = false;
        for (int b = 0; b < B; ++b) {
            acc[b] = 0;
            relin[b] = 0;
            if (!active[b]) continue;
            const double* sc = bt->h_scal + (size_t)b * S_COUNT;
            const double f_trial = bt->h_f[2 * b];
            const double dfp = 0.5 * (lambda[b] * sc[S_DD] - sc[S_DG]) + 0.5 * sc[S_DR];
            const double rho = (dfp > 0.0 && std::isfinite(f_trial)) ? (f[b] - f_trial) / dfp : -1.0;
            if (rho > 0.75) mu[b] = std::max(mu[b] / prm[b].kappa, prm[b].mu_min);
            else if (rho > 0.25) { /* keep mu */ }
            else mu[b] = prm[b].kappa * mu[b];
            if (rho > prm[b].rho_min) {
                acc[b] = 1;
                any_acc = true;
                relin[b] = 1;
                f_cur[b] = f_trial;
            } else if (mu[b] > prm[b].mu_max) {
                st[b] = PTYLM_ERR_STALLED;
                done[b] = 1;
                ++t[b];
            }
        }
        if (any_acc) {
            BSTATUS_TRY(upload_mask(bt, bt->accept, acc));
            kb_axpy<<<bt->n_chunks, BVEC_THREADS, 0, bt->stream>>>(bt->chunks, bt->accept, bt->trial, nullptr, bt->z);
            BSTATUS_TRY(vec_ok(bt));
            if (want_err) {
                kb_err_sums<<<bt->n_chunks, BVEC_THREADS, 0, bt->stream>>>(dot_args(bt, bt->accept, S_ER, OP_STORE), bt->z,
                                                                           bt->ref, bt->pix);
                BSTATUS_TRY(vec_ok(bt));
                BSTATUS_TRY(read_f_and_scalars(bt));
            }
        }
        for (int b = 0; b < B; ++b) {
            if (!acc[b]) continue;
            if (stats && stats[b].hist_len > t[b]) {
                if (stats[b].hist_mu) stats[b].hist_mu[t[b]] = mu[b];
                if (stats[b].hist_cg) stats[b].hist_cg[t[b]] = cg_this[b];
            }
            if (want_err && prm[b].O_ref) {
                const double* sc = bt->h_scal + (size_t)b * S_COUNT;
                const double ac = std::hypot(sc[S_ER], sc[S_EI]);
                const double e2 = std::max(0.0, sc[S_NO] + sc[S_NR] - 2.0 * ac);
                err[b] = std::sqrt(e2 / sc[S_NR]);
                if (stats && stats[b].hist_len > t[b] && stats[b].hist_err) stats[b].hist_err[t[b]] = err[b];
            } else if (stats && stats[b].hist_len > t[b] && stats[b].hist_err) {
                stats[b].hist_err[t[b]] = NAN;
            }
            ++t[b];
            if (t[b] >= prm[b].max_outer || (prm[b].O_ref && prm[b].target_err > 0.0 && err[b] <= prm[b].target_err)) done[b] = 1;
        }
    }
    // restore the true backgrounds; a linearisation under a surrogate level is dropped
    bool surrogate_used = false;
    for (int b = 0; b < B; ++b) {
        surrogate_used |= bt->hprobs[b].b != bt->d[b].background;
        bt->hprobs[b].b = bt->d[b].background;
    }
    BSTATUS_TRY(upload_probs(bt));
    if (surrogate_used) bt->has_lin = false;
    BCUDA_TRY(cudaMemcpyAsync(O_inout, bt->z, zbytes, cudaMemcpyDeviceToDevice, bt->stream));
    BCUDA_TRY(cudaStreamSynchronize(bt->stream));
    ptylm_status worst = PTYLM_OK;
    for (int b = 0; b < B; ++b) {
        if (stats) {
            stats[b].n_outer = t[b];
            stats[b].cg_total = cg_total[b];
            stats[b].matvecs_total = matvecs[b];
            stats[b].f_final = f_cur[b];
            stats[b].err_final = err[b];
        }
        if (st[b] != PTYLM_OK && worst == PTYLM_OK) worst = st[b];
    }
    BSTATUS_TRY(leave(bt));
    if (worst != PTYLM_OK) return bfail(worst, "at least one problem ended with status %d (per-problem stats hold the rest)",
                                        (int)worst);
    for (int b = 0; b < B; ++b)
        if (hit_max[b]) return PTYLM_WARN_CG_MAXIT;
    return PTYLM_OK;
}

ptylm_status ptylm_batch_profile_read(ptylm_batch* bt, long long* launches) {
    if (!bt) return bfail(PTYLM_ERR_ARG, "batch must be non-NULL");
    if (launches) *launches = bt->launches;
    return PTYLM_OK;
}

ptylm_status ptylm_batch_destroy(ptylm_batch* bt) {
    if (!bt) return PTYLM_OK;
    cudaStreamSynchronize(bt->stream);
    bfree_all(bt);
    delete bt;
    return PTYLM_OK;
}

}  // extern "C"
