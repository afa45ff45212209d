// conv_tc.h -- tensor-core 3x3 convolutions of the learned initialisation (tcgen05 MMA with
// BF16 operands and FP32 accumulation in TMEM, operands staged by TMA tiled loads).
//
// Feature maps live in HBM as pairs of bfloat16 tensors (hi, lo) with x = hi + lo,
// hi = bf16(x), lo = bf16(x - hi): the pair carries an FP32 activation to 2^-18 relative
// (two MMAs per product against BF16 weights), so the network computes with BF16 weights and
// FP32-accurate activations.  Weight gradients take the three products hi.hi + hi.lo + lo.hi.
//
// Layout: channel-chunk major, [N][C/8][H][W][8] ("plain"), or split by pixel parity,
// [N][C/8][2][2][H/2][W/2][8] ("parity"), so that 16 neighbouring pixels of one 8-channel chunk
// (of the map or of one of its stride-2 sub-lattices) are 256 contiguous bytes: the row of a
// TMA box.  A tensor may carry a second, parity-split copy (phi, plo) for the kernels that
// read its stride-2 sub-lattices.
//
// Weight copies (bfloat16) are tap- and chunk-major: forward wf[9][Ci_pad/8][Co][8], input
// gradient wb[9][Co_pad/8][Ci][8] (wb[t][o/8][c][o%8] = w[o][c][t]), channels zero-padded to
// multiples of 16.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>

namespace ptylm {

struct Act2 {
    __nv_bfloat16* hi;
    __nv_bfloat16* lo;
    int N, H, W, C;  // batch, height, width, stored channels (multiple of 8)
    int par;         // layout of (hi, lo): 0 plain, 1 parity
    __nv_bfloat16* phi = nullptr;  // optional parity-split copy
    __nv_bfloat16* plo = nullptr;
};

struct TcLayer {
    int Ci, Co;          // channels
    int Ci_pad, Co_pad;  // multiples of 16 >= Ci, Co (K extents of wf and wb)
    int up;              // 0: stride 2; 1: x2 nearest upsampling, then stride 1
    int relu;
    int Hin;             // input side (the low-resolution side for up layers); square maps
    int Hout() const { return up ? 2 * Hin : Hin / 2; }
};

// one-time setup (tensor-map encoder entry point, kernel attributes)
cudaError_t tc_prepare();

// y = relu?(conv(x) + bias): hidden layers write the pair y (NHWC, C = Co); the last layer
// writes y32 as FP32 planes [N][Co][Hout][Hout].
cudaError_t tc_conv_forward(const TcLayer& L, const Act2& x, const __nv_bfloat16* wf, const float* bias, const Act2* y,
                            float* y32, unsigned* err, unsigned spin, int num_sms, cudaStream_t st);

// dx = (d conv / d x)^T dy masked by act > 0 (act: the layer's input, same shape as dx);
// db_part[i][c] (i < *n_part) are partial sums over pixels of dx (the bias gradient of the
// layer that produced act).  db_part needs tc_bias_parts(L, N) * Ci floats.
cudaError_t tc_conv_backward_data(const TcLayer& L, const Act2& dy, const __nv_bfloat16* wb, const Act2& act,
                                  const Act2& dx, float* db_part, int* n_part, unsigned* err, unsigned spin, int num_sms,
                                  cudaStream_t st);
int tc_bias_parts(const TcLayer& L, int N, int num_sms);

// dw[o][c][3][3] = sum over the batch and pixels of dy (.) x at the tap, written (not
// accumulated); ws: tc_wgrad_workspace(L, N, num_sms) floats.
cudaError_t tc_conv_wgrad(const TcLayer& L, const Act2& x, const Act2& dy, float* ws, float* dw, unsigned* err,
                          unsigned spin, int num_sms, cudaStream_t st);
size_t tc_wgrad_workspace(const TcLayer& L, int N, int num_sms);

// The decoder's last layer (x2 nearest upsampling, 3x3 convolution to Co <= 2 channels) on
// the CUDA cores, with the same operands and results as the tc_conv_* calls above: forward
// into FP32 planes y32[N][Co][2H][2W]; input gradient dx (plain pair, plus its parity copy
// when dx.phi is set) masked by act > 0, with tc_last_bias_parts(L, N) partial sums of dx
// per channel in db_part[i][Ci]; weight gradient dw[Co][Ci][3][3] through ws
// (tc_last_wgrad_workspace(L, N) floats).  tc_last_supported: the shapes these kernels take
// (Co <= 2, Ci a power of two in 8 .. 256, input side a multiple of 16).
bool tc_last_supported(const TcLayer& L);
cudaError_t tc_last_forward(const TcLayer& L, const Act2& x, const __nv_bfloat16* wf, const float* bias, float* y32,
                            cudaStream_t st);
cudaError_t tc_last_backward_data(const TcLayer& L, const Act2& dy, const __nv_bfloat16* wf, const Act2& act,
                                  const Act2& dx, float* db_part, int* n_part, cudaStream_t st);
int tc_last_bias_parts(const TcLayer& L, int N);
cudaError_t tc_last_wgrad(const TcLayer& L, const Act2& x, const Act2& dy, float* ws, float* dw, cudaStream_t st);
size_t tc_last_wgrad_workspace(const TcLayer& L, int N);

// db[c] = sum_i part[i][c] in a fixed order; tmp: kBiasSlices * C floats
constexpr int kBiasSlices = 64;
cudaError_t tc_bias_reduce(const float* part, int n_part, int C, float* tmp, float* db, cudaStream_t st);
// wf / wb from the FP32 master weights w[Co][Ci][3][3]
cudaError_t tc_weights(const TcLayer& L, const float* w32, __nv_bfloat16* wf, __nv_bfloat16* wb, cudaStream_t st);
// pair x0 (C = 8, channels 2..7 zero, layout x0.par) from FP32 planes X[N][2][H][W]
cudaError_t tc_pack_input(const float* X, const Act2& x0, cudaStream_t st);
// out[n][c][y][x] = hi + lo of the first C_real channels of the pair a (FP32, [N][C_real][H][W])
cudaError_t tc_unpack(const Act2& a, int C_real, float* out, cudaStream_t st);
// loss += sum mask (out - t)^2 / n_terms (FP64); g = 2 mask (out - t) / n_terms as the pair
// g (C = 8, channels 2..7 zero; plain, plus the parity copy when g.phi is set) and
// db_part[i][2] partial sums of g (FP32).
cudaError_t tc_mse(const float* out, const float* t, const float* mask, const Act2& g, double n_terms, float* db_part,
                   int* n_part, double* loss, cudaStream_t st);
constexpr int kMseBlocks = 256;

}  // namespace ptylm
