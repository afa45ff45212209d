// learned.h -- kernels of the learned initialisation (a data-driven initial object for
// Algorithm 1; not part of the paper): the 3x3 convolution layers of the encoder-decoder
// in forward and backward form (bfloat16 weights, FP32 activations and accumulation), the
// loss, Adam, the physics input computed with the team FFT, and the overlap stitching.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace ptylm {

struct ConvShape {
    int N, Ci, Co, Hin, Win;  // input batch, channels and side (before any upsampling)
    int stride, up, relu;     // stride 1 or 2; up: x2 nearest upsampling of the input first
    int Ho() const { return (up ? 2 * Hin : Hin) / stride; }
    int Wo() const { return (up ? 2 * Win : Win) / stride; }
};

// y = conv(x) + bias (ReLU if relu), NCHW FP32, weights bfloat16 [Co][Ci][3][3].
cudaError_t conv_forward(const ConvShape& s, const float* x, const __nv_bfloat16* w, const float* bias, float* y,
                         cudaStream_t st);
// dx (input side, low resolution for upsampled layers) from dy; wt: the weights transposed
// and flipped ([Ci][Co][3][3], bfloat16), scratch: N*Ci*(2 Hin)*(2 Win) floats for up layers.
cudaError_t conv_backward_data(const ConvShape& s, const float* dy, const __nv_bfloat16* w,
                               const __nv_bfloat16* wt, float* dx, float* scratch, cudaStream_t st);
// dw (FP32, accumulated into: zero it first) and db (written) from x and dy.
cudaError_t conv_backward_weights(const ConvShape& s, const float* x, const float* dy, float* dw, float* db,
                                  int num_sms, cudaStream_t st);
// w16 = bf16(w32) and wt = transposed, flipped bf16 copy.
cudaError_t weights_to_bf16(const ConvShape& s, const float* w32, __nv_bfloat16* w16, __nv_bfloat16* wt,
                            cudaStream_t st);
// g *= (a > 0)
cudaError_t relu_backward(float* g, const float* a, long n, cudaStream_t st);
// loss += sum mask (out - t)^2 / n_terms (FP64), g = 2 mask (out - t) / n_terms
cudaError_t mse_loss(const float* out, const float* t, const float* mask, int N, int HW, double n_terms, float* g,
                     double* loss, cudaStream_t st);
// Adam step t (>= 1) on n parameters, then w16 = bf16(w) when w16 != NULL.
cudaError_t adam_step(float* w, float* m, float* v, const float* g, long n, float lr, float b1, float b2, float eps,
                      int t, cudaStream_t st);
// mask[p] = |P[p]| > 0 as 1/0 floats
cudaError_t support_mask(const float2* P, float* mask, int M, cudaStream_t st);

// Physics input and training pairs (probe side 128): u = F(P)/|F(P)| in team order;
// pairs: for samples (obj, r, c) of a pool of objects [n_obj][side][side], X = physics
// input of the noiseless pattern of P . O[r:, c:], T = the object patch (Re, Im channels);
// inputs: X from measured magnitudes (team order, sqrt taken when take_sqrt) at positions
// pos[idx[i]].
cudaError_t probe_phasor(const float2* P, const float2* tw, float2* u, cudaStream_t st);
cudaError_t learn_pairs(const float2* pool, int side, const int4* samples, int N, const float2* P, const float2* u,
                        const float2* tw, float eps_rel, float* X, float* T, cudaStream_t st);
cudaError_t physics_inputs(const float* y_team, int take_sqrt, const int* idx, int n, const float2* P,
                           const float2* u, const float2* tw, float eps_rel, float* X, cudaStream_t st);
// Stitching: num/den accumulate |P|^2-weighted patches (Re, Im channels of est) at pos[idx[i]];
// finish writes O = num/den where den > 0, else 1.
cudaError_t stitch_accumulate(const float* est, const int* idx, int n, const int2* pos, const float2* P, int nx,
                              float2* num, float* den, cudaStream_t st);
cudaError_t stitch_finish(const float2* num, const float* den, long N, float2* O, cudaStream_t st);

}  // namespace ptylm
