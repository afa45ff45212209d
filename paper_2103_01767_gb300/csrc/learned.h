// learned.h -- kernels of the learned initialisation (a data-driven initial object for
// Algorithm 1; not part of the paper) besides its convolutions (conv_tc.h): Adam, the
// probe-support mask, the physics input computed with the team FFT, and the overlap
// stitching.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace ptylm {

// Adam step t (>= 1) on n parameters.
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
