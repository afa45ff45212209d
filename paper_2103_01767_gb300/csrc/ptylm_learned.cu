// ptylm_learned.cu -- C-ABI of the learned initialisation (include/ptylm.h): the network
// object (parameters, Adam state, activation buffers), its forward / gradient / training
// entry points and the initial-object builder for a single-problem context.
//
// Training draws its samples with a host splitmix64 generator from the caller's seed:
// (object, row, column) triples over a pool of objects; the pairs themselves (physics input,
// target patch) are produced on the device by the forward model.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/ptylm.h"
#include "kernels.h"
#include "conv_tc.h"
#include "learned.h"

using namespace ptylm;

namespace {

ptylm_status lfail(ptylm_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    set_last_error(buf);
    return s;
}

#define LCUDA_TRY(expr)                                                                          \
    do {                                                                                         \
        cudaError_t e_ = (expr);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return lfail(PTYLM_ERR_CUDA, "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), \
                         __FILE__, __LINE__);                                                    \
    } while (0)

#define LSTATUS_TRY(expr)               \
    do {                                \
        ptylm_status s_ = (expr);       \
        if (s_ != PTYLM_OK) return s_;  \
    } while (0)

constexpr int NL = 6;
constexpr float EPS_REL = 1e-3f;   // the physics input divides by |P|^2 + EPS_REL max|P|^2

uint64_t splitmix64(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace

struct ptylm_net {
    int m = 0, widths[3] = {0, 0, 0}, max_batch = 0, num_sms = 0;
    TcLayer L[NL];
    bool last_cuda_cores = false;      // the last layer runs on the CUDA cores (conv_last.cu)
    long w_off[NL], b_off[NL], n_params = 0;
    cudaStream_t stream = nullptr;
    std::vector<void*> allocs;
    float* params = nullptr;           // FP32 master: W1 b1 W2 b2 ... (W as [co][ci][3][3])
    float* grads = nullptr;            // same layout
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    int adam_t = 0;
    __nv_bfloat16* wf[NL] = {};        // forward weight copies [9][Co][Ci_pad]
    __nv_bfloat16* wb[NL] = {};        // input-gradient weight copies [9][Ci][Co_pad]
    float* xin = nullptr;              // [max_batch][2][m][m]
    float* target = nullptr;           // [max_batch][2][m][m]
    float* out = nullptr;              // network output [max_batch][2][m][m]
    Act2 x0{};                         // packed input pair, 8 channels
    Act2 act[NL - 1] = {};             // hidden layer outputs (chunk-major pairs)
    Act2 g[NL] = {};                   // gradient w.r.t. each layer's output (g[NL-1]: 8 channels)
    float* db_part = nullptr;          // partial sums of the bias gradients
    float* db_tmp = nullptr;           // their slice sums (kBiasSlices x 256)
    float* ws = nullptr;               // weight-gradient partial sums
    unsigned* err = nullptr;           // bounded-wait failures of the convolution kernels
    float* mask = nullptr;             // [m][m] probe support
    double* loss = nullptr;            // [1]
    float2* tw = nullptr;              // W_m^j
    float2* u = nullptr;               // F(P)/|F(P)| in team order
    float2* P = nullptr;
};

namespace {

constexpr unsigned kConvSpin = 1u << 24;   // polls per bounded wait of a convolution kernel

ptylm_status nalloc(ptylm_net* n, void** p, size_t bytes) {
    if (cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) {
        cudaGetLastError();
        return lfail(PTYLM_ERR_NOMEM, "cudaMalloc(%zu) for the network failed", bytes);
    }
    n->allocs.push_back(*p);
    return PTYLM_OK;
}
template <class T>
ptylm_status nalloc_t(ptylm_net* n, T** p, size_t count) {
    void* q = nullptr;
    ptylm_status s = nalloc(n, &q, count * sizeof(T));
    *p = static_cast<T*>(q);
    return s;
}
// pair tensor of max_batch maps H x H x C in layout `par`, with a parity-split copy if asked
ptylm_status nalloc_act(ptylm_net* n, Act2* a, int H, int C, int par, bool parity_copy) {
    *a = Act2{nullptr, nullptr, n->max_batch, H, H, C, par};
    const size_t count = (size_t)n->max_batch * H * H * C;
    ptylm_status s;
    if ((s = nalloc_t(n, &a->hi, count)) != PTYLM_OK || (s = nalloc_t(n, &a->lo, count)) != PTYLM_OK) return s;
    if (parity_copy && ((s = nalloc_t(n, &a->phi, count)) != PTYLM_OK || (s = nalloc_t(n, &a->plo, count)) != PTYLM_OK))
        return s;
    return PTYLM_OK;
}
Act2 batch(Act2 a, int N) {
    a.N = N;
    return a;
}

ptylm_status refresh_bf16(ptylm_net* n) {
    for (int l = 0; l < NL; ++l) LCUDA_TRY(tc_weights(n->L[l], n->params + n->w_off[l], n->wf[l], n->wb[l], n->stream));
    return PTYLM_OK;
}

// a bounded wait inside a convolution kernel gave up: report it and clear the flag
ptylm_status check_conv_wait(ptylm_net* n) {
    unsigned h = 0;
    LCUDA_TRY(cudaMemcpyAsync(&h, n->err, sizeof(unsigned), cudaMemcpyDeviceToHost, n->stream));
    LCUDA_TRY(cudaStreamSynchronize(n->stream));
    if (h) {
        LCUDA_TRY(cudaMemset(n->err, 0, sizeof(unsigned)));
        return lfail(PTYLM_ERR_TIMEOUT, "a bounded wait of a convolution kernel gave up (flags 0x%x)", h);
    }
    return PTYLM_OK;
}

ptylm_status forward(ptylm_net* n, const float* X, int N) {
    const Act2 x0 = batch(n->x0, N);
    LCUDA_TRY(tc_pack_input(X, x0, n->stream));
    Act2 in = x0;
    for (int l = 0; l < NL; ++l) {
        const Act2 y = l < NL - 1 ? batch(n->act[l], N) : Act2{};
        if (l == NL - 1 && n->last_cuda_cores)
            LCUDA_TRY(tc_last_forward(n->L[l], in, n->wf[l], n->params + n->b_off[l], n->out, n->stream));
        else
            LCUDA_TRY(tc_conv_forward(n->L[l], in, n->wf[l], n->params + n->b_off[l], l < NL - 1 ? &y : nullptr, n->out,
                                      n->err, kConvSpin, n->num_sms, n->stream));
        in = y;
    }
    return PTYLM_OK;
}

// loss and gradients (into n->grads) for the batch X -> target T
ptylm_status loss_grad(ptylm_net* n, const float* X, const float* T, int N, double n_terms, double* loss_dev) {
    LSTATUS_TRY(forward(n, X, N));
    int parts = 0;
    LCUDA_TRY(tc_mse(n->out, T, n->mask, batch(n->g[NL - 1], N), n_terms, n->db_part, &parts, loss_dev, n->stream));
    LCUDA_TRY(tc_bias_reduce(n->db_part, parts, n->L[NL - 1].Co, n->db_tmp, n->grads + n->b_off[NL - 1], n->stream));
    for (int l = NL - 1; l >= 0; --l) {
        const Act2 in = l == 0 ? batch(n->x0, N) : batch(n->act[l - 1], N);
        const Act2 g = batch(n->g[l], N);
        const bool cc = l == NL - 1 && n->last_cuda_cores;
        if (cc) LCUDA_TRY(tc_last_wgrad(n->L[l], in, g, n->ws, n->grads + n->w_off[l], n->stream));
        else LCUDA_TRY(tc_conv_wgrad(n->L[l], in, g, n->ws, n->grads + n->w_off[l], n->err, kConvSpin, n->num_sms, n->stream));
        if (l > 0) {
            if (cc)
                LCUDA_TRY(tc_last_backward_data(n->L[l], g, n->wf[l], in, batch(n->g[l - 1], N), n->db_part, &parts,
                                                n->stream));
            else
                LCUDA_TRY(tc_conv_backward_data(n->L[l], g, n->wb[l], in, batch(n->g[l - 1], N), n->db_part, &parts,
                                                n->err, kConvSpin, n->num_sms, n->stream));
            LCUDA_TRY(tc_bias_reduce(n->db_part, parts, n->L[l].Ci, n->db_tmp, n->grads + n->b_off[l - 1], n->stream));
        }
    }
    return PTYLM_OK;
}

// FP32 master parameters -> host copy of the probe's eps and the support-mask sum
ptylm_status set_probe(ptylm_net* n, const ptylm_c64* P, float* eps_abs, double* mask_sum) {
    const int M = n->m * n->m;
    std::vector<float2> h(M);
    LCUDA_TRY(cudaMemcpy(h.data(), P, sizeof(float2) * M, cudaMemcpyDefault));
    double mx = 0.0, cnt = 0.0;
    for (auto& p : h) {
        const double a = (double)p.x * p.x + (double)p.y * p.y;
        mx = std::max(mx, a);
        cnt += (p.x != 0.0f || p.y != 0.0f) ? 1.0 : 0.0;
    }
    if (!(mx > 0.0)) return lfail(PTYLM_ERR_ARG, "the probe is zero");
    LCUDA_TRY(cudaMemcpyAsync(n->P, h.data(), sizeof(float2) * M, cudaMemcpyHostToDevice, n->stream));
    LCUDA_TRY(probe_phasor(n->P, n->tw, n->u, n->stream));
    LCUDA_TRY(support_mask(n->P, n->mask, M, n->stream));
    LCUDA_TRY(cudaStreamSynchronize(n->stream));
    *eps_abs = (float)(EPS_REL * mx);
    if (mask_sum) *mask_sum = cnt;
    return PTYLM_OK;
}

}  // namespace

extern "C" {

ptylm_status ptylm_net_create(ptylm_net** out, int m, const int* widths, int max_batch, uint64_t seed, void* stream) {
    set_last_error("");
    if (!out || !widths) return lfail(PTYLM_ERR_ARG, "net and widths must be non-NULL");
    *out = nullptr;
    if (m != 128) return lfail(PTYLM_ERR_ARG, "the learned initialisation is built for 128 x 128 patterns");
    if (max_batch < 1) return lfail(PTYLM_ERR_ARG, "max_batch must be >= 1");
    for (int i = 0; i < 3; ++i)
        if (widths[i] < 32 || widths[i] > 256 || widths[i] % 32)
            return lfail(PTYLM_ERR_ARG, "widths must be multiples of 32 in [32, 256]");
    ptylm_net* n = new ptylm_net();
    auto bail = [&](ptylm_status s) {
        for (void* p : n->allocs) cudaFree(p);
        delete n;
        return s;
    };
    n->m = m;
    n->max_batch = max_batch;
    n->stream = static_cast<cudaStream_t>(stream);
    std::copy(widths, widths + 3, n->widths);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return bail(lfail(PTYLM_ERR_CUDA, "no usable CUDA device"));
    }
    if (tc_prepare() != cudaSuccess) {
        cudaGetLastError();
        return bail(lfail(PTYLM_ERR_CUDA, "the tensor-core convolutions need the tensor-map encoder of the driver"));
    }
    const int c1 = widths[0], c2 = widths[1], c3 = widths[2];
    const int ci[NL] = {2, c1, c2, c3, c2, c1}, co[NL] = {c1, c2, c3, c2, c1, 2};
    const int upv[NL] = {0, 0, 0, 1, 1, 1}, rl[NL] = {1, 1, 1, 1, 1, 0};
    const int hin[NL] = {m, m / 2, m / 4, m / 8, m / 4, m / 2};
    long off = 0;
    for (int l = 0; l < NL; ++l) {
        n->L[l] = TcLayer{ci[l], co[l], (ci[l] + 15) / 16 * 16, (co[l] + 15) / 16 * 16, upv[l], rl[l], hin[l]};
        n->w_off[l] = off;
        off += (long)co[l] * ci[l] * 9;
        n->b_off[l] = off;
        off += co[l];
    }
    n->n_params = off;
    n->last_cuda_cores = tc_last_supported(n->L[NL - 1]);
    ptylm_status s;
    const size_t img = (size_t)max_batch * 2 * m * m;
    size_t ws = 1, parts = (size_t)kMseBlocks * 2;
    for (int l = 0; l < NL; ++l) {
        ws = std::max(ws, tc_wgrad_workspace(n->L[l], max_batch, n->num_sms));
        if (l > 0) parts = std::max(parts, (size_t)tc_bias_parts(n->L[l], max_batch, n->num_sms) * ci[l]);
        if (l == NL - 1 && n->last_cuda_cores) {
            ws = std::max(ws, tc_last_wgrad_workspace(n->L[l], max_batch));
            parts = std::max(parts, (size_t)tc_last_bias_parts(n->L[l], max_batch) * ci[l]);
        }
    }
    if ((s = nalloc_t(n, &n->params, off)) || (s = nalloc_t(n, &n->grads, off)) || (s = nalloc_t(n, &n->adam_m, off)) ||
        (s = nalloc_t(n, &n->adam_v, off)) || (s = nalloc_t(n, &n->xin, img)) || (s = nalloc_t(n, &n->target, img)) ||
        (s = nalloc_t(n, &n->out, img)) || (s = nalloc_t(n, &n->db_part, parts)) || (s = nalloc_t(n, &n->db_tmp, (size_t)kBiasSlices * 256)) || (s = nalloc_t(n, &n->ws, ws)) ||
        (s = nalloc_t(n, &n->err, 1)) || (s = nalloc_t(n, &n->mask, (size_t)m * m)) || (s = nalloc_t(n, &n->loss, 1)) ||
        (s = nalloc_t(n, &n->tw, m)) || (s = nalloc_t(n, &n->u, (size_t)m * m)) || (s = nalloc_t(n, &n->P, (size_t)m * m)) ||
        (s = nalloc_act(n, &n->x0, m, 8, 1, false)) || (s = nalloc_act(n, &n->g[NL - 1], m, 8, 0, true)))
        return bail(s);
    for (int l = 0; l < NL; ++l) {
        if ((s = nalloc_t(n, &n->wf[l], (size_t)9 * co[l] * n->L[l].Ci_pad)) ||
            (s = nalloc_t(n, &n->wb[l], (size_t)9 * ci[l] * n->L[l].Co_pad)))
            return bail(s);
        // the input of a stride-2 layer is stored split by parity; the output gradient of an
        // upsampling layer also gets a parity-split copy (its weight gradient reads the four
        // output phases)
        if (l < NL - 1 && ((s = nalloc_act(n, &n->act[l], n->L[l].Hout(), co[l], n->L[l + 1].up ? 0 : 1, false)) ||
                           (s = nalloc_act(n, &n->g[l], n->L[l].Hout(), co[l], 0, n->L[l].up != 0))))
            return bail(s);
    }
    if (cudaMemset(n->err, 0, sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        return bail(lfail(PTYLM_ERR_CUDA, "initialising the network"));
    }
    // He-normal initial weights (std sqrt(2 / (9 c_in))) by Box-Muller on splitmix64, zero biases
    std::vector<float> h(off, 0.0f);
    uint64_t state = seed;
    for (int l = 0; l < NL; ++l) {
        const double sd = std::sqrt(2.0 / (9.0 * ci[l]));
        for (long i = 0; i < (long)co[l] * ci[l] * 9; ++i) {
            const double u1 = ((splitmix64(state) >> 11) + 1.0) * (1.0 / 9007199254740993.0);
            const double u2 = (splitmix64(state) >> 11) * (1.0 / 9007199254740992.0);
            h[n->w_off[l] + i] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * M_PI * u2));
        }
    }
    std::vector<float2> htw(m);
    for (int j = 0; j < m; ++j) {
        const double ang = 2.0 * M_PI * (double)j / (double)m;
        htw[j] = make_float2((float)std::cos(ang), (float)-std::sin(ang));
    }
    if (cudaMemcpy(n->params, h.data(), sizeof(float) * off, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(n->tw, htw.data(), sizeof(float2) * m, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(n->adam_m, 0, sizeof(float) * off) != cudaSuccess || cudaMemset(n->adam_v, 0, sizeof(float) * off) != cudaSuccess) {
        cudaGetLastError();
        return bail(lfail(PTYLM_ERR_CUDA, "initialising the network"));
    }
    if ((s = refresh_bf16(n)) != PTYLM_OK) return bail(s);
    if (cudaStreamSynchronize(n->stream) != cudaSuccess) {
        cudaGetLastError();
        return bail(lfail(PTYLM_ERR_CUDA, "initialising the network"));
    }
    *out = n;
    return PTYLM_OK;
}

long ptylm_net_num_params(const ptylm_net* n) { return n ? n->n_params : -1; }

ptylm_status ptylm_net_set_params(ptylm_net* n, const float* host) {
    set_last_error("");
    if (!n || !host) return lfail(PTYLM_ERR_ARG, "net and params must be non-NULL");
    LCUDA_TRY(cudaMemcpy(n->params, host, sizeof(float) * n->n_params, cudaMemcpyHostToDevice));
    LSTATUS_TRY(refresh_bf16(n));
    LCUDA_TRY(cudaStreamSynchronize(n->stream));
    return PTYLM_OK;
}

ptylm_status ptylm_net_get_params(ptylm_net* n, float* host, float* grads_host) {
    set_last_error("");
    if (!n) return lfail(PTYLM_ERR_ARG, "net must be non-NULL");
    LCUDA_TRY(cudaStreamSynchronize(n->stream));
    if (host) LCUDA_TRY(cudaMemcpy(host, n->params, sizeof(float) * n->n_params, cudaMemcpyDeviceToHost));
    if (grads_host) LCUDA_TRY(cudaMemcpy(grads_host, n->grads, sizeof(float) * n->n_params, cudaMemcpyDeviceToHost));
    return PTYLM_OK;
}

ptylm_status ptylm_net_activation(ptylm_net* n, int layer, int N, float* out) {
    set_last_error("");
    if (!n || !out) return lfail(PTYLM_ERR_ARG, "net and out must be non-NULL");
    if (layer < 1 || layer > NL - 1) return lfail(PTYLM_ERR_ARG, "layer must be in [1, %d]", NL - 1);
    if (N < 1 || N > n->max_batch) return lfail(PTYLM_ERR_ARG, "N must be in [1, max_batch]");
    LCUDA_TRY(tc_unpack(batch(n->act[layer - 1], N), n->L[layer - 1].Co, out, n->stream));
    LCUDA_TRY(cudaStreamSynchronize(n->stream));
    return PTYLM_OK;
}

ptylm_status ptylm_net_forward(ptylm_net* n, const float* X, int N, float* out) {
    set_last_error("");
    if (!n || !X || !out) return lfail(PTYLM_ERR_ARG, "net, X and out must be non-NULL");
    if (N < 1 || N > n->max_batch) return lfail(PTYLM_ERR_ARG, "N must be in [1, max_batch]");
    LSTATUS_TRY(forward(n, X, N));
    LCUDA_TRY(cudaMemcpyAsync(out, n->out, sizeof(float) * N * 2 * n->m * n->m, cudaMemcpyDeviceToDevice, n->stream));
    return check_conv_wait(n);
}

ptylm_status ptylm_net_loss_grad(ptylm_net* n, const float* X, const float* T, const float* mask, int N, double* loss) {
    set_last_error("");
    if (!n || !X || !T || !mask) return lfail(PTYLM_ERR_ARG, "net, X, T and mask must be non-NULL");
    if (N < 1 || N > n->max_batch) return lfail(PTYLM_ERR_ARG, "N must be in [1, max_batch]");
    const int M = n->m * n->m;
    std::vector<float> hm(M);
    LCUDA_TRY(cudaMemcpy(hm.data(), mask, sizeof(float) * M, cudaMemcpyDefault));
    double msum = 0.0;
    for (float v : hm) msum += v;
    if (!(msum > 0.0)) return lfail(PTYLM_ERR_ARG, "the mask is empty");
    LCUDA_TRY(cudaMemcpyAsync(n->mask, hm.data(), sizeof(float) * M, cudaMemcpyHostToDevice, n->stream));
    LCUDA_TRY(cudaMemsetAsync(n->loss, 0, sizeof(double), n->stream));
    LSTATUS_TRY(loss_grad(n, X, T, N, 2.0 * N * msum, n->loss));
    double h = 0.0;
    LCUDA_TRY(cudaMemcpyAsync(&h, n->loss, sizeof(double), cudaMemcpyDeviceToHost, n->stream));
    LCUDA_TRY(cudaStreamSynchronize(n->stream));
    LSTATUS_TRY(check_conv_wait(n));
    if (loss) *loss = h;
    return PTYLM_OK;
}

ptylm_status ptylm_net_pairs(ptylm_net* n, const ptylm_c64* pool, int side, const int32_t* samples, int N,
                             const ptylm_c64* P, float* X, float* T) {
    set_last_error("");
    if (!n || !pool || !samples || !P || !X || !T || N < 0) return lfail(PTYLM_ERR_ARG, "invalid arguments");
    if (side < n->m) return lfail(PTYLM_ERR_ARG, "objects smaller than the probe");
    std::vector<int32_t> hs(3 * (size_t)std::max(1, N));
    if (N > 0) LCUDA_TRY(cudaMemcpy(hs.data(), samples, sizeof(int32_t) * 3 * N, cudaMemcpyDefault));
    std::vector<int4> h4(std::max(1, N));
    for (int i = 0; i < N; ++i) {
        if (hs[3 * i] < 0 || hs[3 * i + 1] < 0 || hs[3 * i + 2] < 0 || hs[3 * i + 1] + n->m > side || hs[3 * i + 2] + n->m > side)
            return lfail(PTYLM_ERR_ARG, "sample %d outside its object", i);
        h4[i] = make_int4(hs[3 * i], hs[3 * i + 1], hs[3 * i + 2], 0);
    }
    float eps_abs = 0.0f;
    LSTATUS_TRY(set_probe(n, P, &eps_abs, nullptr));
    int4* d4 = nullptr;
    LCUDA_TRY(cudaMalloc(&d4, sizeof(int4) * h4.size()));
    cudaError_t e = cudaMemcpy(d4, h4.data(), sizeof(int4) * h4.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = learn_pairs(reinterpret_cast<const float2*>(pool), side, d4, N, n->P, n->u, n->tw, eps_abs, X, T, n->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
    cudaFree(d4);
    LCUDA_TRY(e);
    return PTYLM_OK;
}

ptylm_status ptylm_net_train(ptylm_net* n, const ptylm_c64* pool, int n_obj, int side, const ptylm_c64* P, int steps,
                             int batch, double lr, uint64_t seed, double* loss_hist) {
    set_last_error("");
    if (!n || !pool || !P || n_obj < 1 || steps < 0) return lfail(PTYLM_ERR_ARG, "invalid arguments");
    if (batch < 1 || batch > n->max_batch) return lfail(PTYLM_ERR_ARG, "batch must be in [1, max_batch]");
    if (side < n->m) return lfail(PTYLM_ERR_ARG, "objects smaller than the probe");
    float eps_abs = 0.0f;
    double msum = 0.0;
    LSTATUS_TRY(set_probe(n, P, &eps_abs, &msum));
    if (steps == 0) return PTYLM_OK;
    // all samples up front: (object, row, column) per pattern
    std::vector<int4> h((size_t)steps * batch);
    uint64_t state = seed;
    const uint64_t span = (uint64_t)(side - n->m + 1);
    for (auto& q : h) {
        q.x = (int)(splitmix64(state) % (uint64_t)n_obj);
        q.y = (int)(splitmix64(state) % span);
        q.z = (int)(splitmix64(state) % span);
        q.w = 0;
    }
    int4* d4 = nullptr;
    double* dl = nullptr;
    LCUDA_TRY(cudaMalloc(&d4, sizeof(int4) * h.size()));
    if (cudaMalloc(&dl, sizeof(double) * steps) != cudaSuccess) {
        cudaFree(d4);
        cudaGetLastError();
        return lfail(PTYLM_ERR_NOMEM, "loss history");
    }
    ptylm_status s = PTYLM_OK;
    cudaError_t e = cudaMemcpy(d4, h.data(), sizeof(int4) * h.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemsetAsync(dl, 0, sizeof(double) * steps, n->stream);
    if (e != cudaSuccess) s = lfail(PTYLM_ERR_CUDA, "uploading the samples: %s", cudaGetErrorString(e));
    const double n_terms = 2.0 * batch * msum;
    for (int t = 0; t < steps && s == PTYLM_OK; ++t) {
        // learning rate falls linearly to a tenth over the run
        const float lr_t = (float)(lr * (1.0 - 0.9 * (double)t / (double)steps));
        e = learn_pairs(reinterpret_cast<const float2*>(pool), side, d4 + (size_t)t * batch, batch, n->P, n->u, n->tw,
                        eps_abs, n->xin, n->target, n->stream);
        if (e != cudaSuccess) { s = lfail(PTYLM_ERR_CUDA, "training pairs: %s", cudaGetErrorString(e)); break; }
        if ((s = loss_grad(n, n->xin, n->target, batch, n_terms, dl + t)) != PTYLM_OK) break;
        e = adam_step(n->params, n->adam_m, n->adam_v, n->grads, n->n_params, lr_t, 0.9f, 0.999f, 1e-8f, ++n->adam_t, n->stream);
        if (e != cudaSuccess) { s = lfail(PTYLM_ERR_CUDA, "Adam: %s", cudaGetErrorString(e)); break; }
        s = refresh_bf16(n);
    }
    if (s == PTYLM_OK) {
        e = cudaStreamSynchronize(n->stream);
        if (e == cudaSuccess && loss_hist) e = cudaMemcpy(loss_hist, dl, sizeof(double) * steps, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) s = lfail(PTYLM_ERR_CUDA, "training: %s", cudaGetErrorString(e));
        else s = check_conv_wait(n);
    }
    cudaFree(d4);
    cudaFree(dl);
    return s;
}

ptylm_status ptylm_learned_inputs(ptylm_ctx* ctx, ptylm_net* n, const ptylm_c64* P, const int32_t* idx, int count,
                                  float* X) {
    set_last_error("");
    CtxView cv;
    if (!ctx || !n || !P || !X || (count > 0 && !idx) || !ctx_view(ctx, &cv)) return lfail(PTYLM_ERR_ARG, "invalid arguments");
    if (cv.m != n->m) return lfail(PTYLM_ERR_ARG, "context and network pattern sizes differ");
    LCUDA_TRY(cudaStreamSynchronize(cv.stream));
    if (count > 0) {
        std::vector<int32_t> hi(count);
        LCUDA_TRY(cudaMemcpy(hi.data(), idx, sizeof(int32_t) * count, cudaMemcpyDefault));
        for (int i = 0; i < count; ++i)
            if (hi[i] < 0 || hi[i] >= cv.K) return lfail(PTYLM_ERR_ARG, "position index %d out of range", hi[i]);
    }
    float eps_abs = 0.0f;
    LSTATUS_TRY(set_probe(n, P, &eps_abs, nullptr));
    LCUDA_TRY(physics_inputs(cv.y_team, cv.loss == PTYLM_LOSS_POISSON, reinterpret_cast<const int*>(idx), count, n->P,
                             n->u, n->tw, eps_abs, X, n->stream));
    LCUDA_TRY(cudaStreamSynchronize(n->stream));
    return PTYLM_OK;
}

ptylm_status ptylm_learned_init(ptylm_ctx* ctx, ptylm_net* n, const ptylm_c64* P, const int32_t* idx, int count,
                                ptylm_c64* O0) {
    set_last_error("");
    CtxView cv;
    if (!ctx || !n || !P || !O0 || count < 0 || (count > 0 && !idx) || !ctx_view(ctx, &cv))
        return lfail(PTYLM_ERR_ARG, "invalid arguments");
    if (cv.m != n->m) return lfail(PTYLM_ERR_ARG, "context and network pattern sizes differ");
    LCUDA_TRY(cudaStreamSynchronize(cv.stream));   // the context's measurements are in place
    std::vector<int32_t> hi(std::max(1, count));
    if (count > 0) LCUDA_TRY(cudaMemcpy(hi.data(), idx, sizeof(int32_t) * count, cudaMemcpyDefault));
    for (int i = 0; i < count; ++i)
        if (hi[i] < 0 || hi[i] >= cv.K) return lfail(PTYLM_ERR_ARG, "position index %d out of range", hi[i]);
    float eps_abs = 0.0f;
    LSTATUS_TRY(set_probe(n, P, &eps_abs, nullptr));
    const long N = (long)cv.ny * cv.nx;
    float2* num = nullptr;
    float* den = nullptr;
    int* didx = nullptr;
    cudaError_t e = cudaMalloc(&num, sizeof(float2) * N);
    if (e == cudaSuccess) e = cudaMalloc(&den, sizeof(float) * N);
    if (e == cudaSuccess) e = cudaMalloc(&didx, sizeof(int) * std::max(1, count));
    if (e == cudaSuccess) e = cudaMemcpy(didx, hi.data(), sizeof(int) * std::max(1, count), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemsetAsync(num, 0, sizeof(float2) * N, n->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(den, 0, sizeof(float) * N, n->stream);
    ptylm_status s = PTYLM_OK;
    for (int i0 = 0; i0 < count && e == cudaSuccess && s == PTYLM_OK; i0 += n->max_batch) {
        const int nb = std::min(n->max_batch, count - i0);
        e = physics_inputs(cv.y_team, cv.loss == PTYLM_LOSS_POISSON, didx + i0, nb, n->P, n->u, n->tw, eps_abs, n->xin,
                           n->stream);
        if (e == cudaSuccess) s = forward(n, n->xin, nb);
        if (e == cudaSuccess && s == PTYLM_OK)
            e = stitch_accumulate(n->out, didx + i0, nb, cv.pos, n->P, cv.nx, num, den, n->stream);
    }
    if (e == cudaSuccess && s == PTYLM_OK) e = stitch_finish(num, den, N, reinterpret_cast<float2*>(O0), n->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
    cudaFree(num);
    cudaFree(den);
    cudaFree(didx);
    if (s != PTYLM_OK) return s;
    LCUDA_TRY(e);
    return check_conv_wait(n);
}

ptylm_status ptylm_net_destroy(ptylm_net* n) {
    if (!n) return PTYLM_OK;
    cudaStreamSynchronize(n->stream);
    for (void* p : n->allocs) cudaFree(p);
    delete n;
    return PTYLM_OK;
}

}  // extern "C"
