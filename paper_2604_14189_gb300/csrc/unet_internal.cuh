// Internal interfaces of the learned gradient preconditioner (a U-Net run
// in BF16 with FP32 accumulation): the tcgen05 convolution kernels
// (unet_conv.cu), the element-wise and reduction kernels (unet_ops.cu) and
// the network driver (unet_api.cu).
//
// Tensors are NHWC BF16: element (b, y, x, c) of a view with pixel stride
// ps (channels of the underlying buffer; a view may start at a channel
// offset, e.g. one half of a concatenation buffer) sits at
// base[((b H + y) W + x) ps + c].
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace sweep {

typedef __nv_bfloat16 bf16;

// One 3 x 3 convolution as an implicit GEMM on the tensor cores:
//   out[p][n] = op( sum_{tap, k} in[p + off(tap)][k] * w[n][tap][k] + bias[n] )
// over 128-pixel tiles (M = 128 pixels, N = all output channels, K = 9
// taps x input channels in chunks of kc).  The data gradient of a
// convolution is the same operation on the output gradient with the
// weights transposed and mirrored (w'[ci][8 - tap][co] = w[co][tap][ci]).
enum ConvOp { kOpNone = 0, kOpRelu = 1, kOpMask = 2 };
struct ConvArgs {
  CUtensorMap tin;   // input view {cin, W, H, B}, box {kc, bw, bh, 1}
  CUtensorMap tw;    // weights {cin, 9, cout}, box {kc, 1, cout}
  int B, H, W;
  int cin, cout, kc;  // kc = 64 (128-byte swizzle) or 32 (64-byte)
  int bw, bh;         // pixel tile: bw x bh = 128
  int stages;
  const float* bias;  // [cout] or NULL
  int op;             // ConvOp
  const bf16* mask;   // kOpMask: out *= (mask > 0), same pixel/channel
  int mask_ps;
  bf16* out;
  int out_ps;
  int* status;        // latched on a wait that gives up
};

// Weight gradient of one 3 x 3 convolution on the tensor cores:
//   D[(tap, ci)][co] = sum_p in[p + off(tap)][ci] * dy[p][co]
// (M = 128 rows of (tap, ci) per CTA, N = cout, K = pixels in 64-pixel
// steps, both operands MN-major), one partial sum per pixel split.
struct WgradArgs {
  CUtensorMap tin;   // input view {cin, W, H, B}, box {ka, pw, ph, 1}
  CUtensorMap tdy;   // output-gradient view {cout, W, H, B}, box {kb, pw, ph, 1}
  int B, H, W;
  int cin, cout, ka, kb;  // ka, kb: 64 or 32 channels per box
  int pw, ph;             // pixel box: pw x ph = 64
  int mtiles, splits, stages;
  float* partial;         // [splits][mtiles * 128][cout]
  int* status;
};

void launch_conv(const ConvArgs& a, cudaStream_t st);
void launch_wgrad(const WgradArgs& a, cudaStream_t st);
size_t conv_smem_bytes(int cout, int kc, int stages);
size_t wgrad_smem_bytes(int cout, int stages);

// ---- element-wise and reduction kernels (unet_ops.cu)
struct WeightPrep {  // one 3 x 3 layer of the flat parameter vector
  long long off;     // W[cout][3][3][cin] in the flat FP32 vector
  int cin, cout;
  bf16* w;           // out [cout][9][cin]
  bf16* wt;          // out [cin][9][cout], taps mirrored (data gradient)
};
constexpr int kUnetLayers = 17;
struct WeightPrepAll {
  WeightPrep l[kUnetLayers];
};
void launch_prep_weights(const float* theta, const WeightPrepAll& p, long long total_w,
                         cudaStream_t st);
void launch_pack_input(const float* in, int in_ch, bf16* x0, long long npix, cudaStream_t st);
void launch_pool(const bf16* s, int s_ps, bf16* out, int B, int H, int W, int C,
                 cudaStream_t st);
void launch_upsample(const bf16* x, bf16* out, int B, int h, int w, int C, cudaStream_t st);
// d[p][c] = bf16( (sum over the 2 x 2 children of p of g[child][c]) * (x[p][c] > 0) )
void launch_up_backward_mask(const bf16* g, int g_ps, const bf16* x, bf16* d, int B, int h,
                             int w, int C, cudaStream_t st);
// d[p][c] = bf16( 0.25 gp[parent(p)][c] * (s[p][c] > 0) + gskip[p][c] )
void launch_pool_backward_combine(const bf16* gp, const bf16* s, int s_ps, const bf16* gskip,
                                  int gskip_ps, bf16* d, int B, int H, int W, int C,
                                  cudaStream_t st);
// out[p] = sum_c x[p][c] wh[c] + bh; with a target also the loss partials
void launch_head_forward(const bf16* x, const float* theta_head, float* out, long long npix,
                         cudaStream_t st);
// loss = mean (out - t)^2 (FP64); dout = 2 (out - t) / N;
// dpre[p][c] = bf16(dout[p] wh[c] (x[p][c] > 0)); head gradients
void launch_head_backward(const bf16* x, const float* theta_head, const float* out,
                          const float* target, long long npix, bf16* dpre, double* partial,
                          int nblocks, double* loss, float* grad_head, cudaStream_t st);
// db[co] = sum_p dy[p][co] (FP32, fixed order)
void launch_bias_grad(const bf16* dy, int dy_ps, int cout, long long npix, float* partial,
                      int nblocks, float* db, cudaStream_t st);
// dW[co][tap][ci] = sum_s partial[s][tap cin + ci][co]
void launch_wgrad_reduce(const float* partial, int splits, int rows_padded, int cin, int cout,
                         float* dW, cudaStream_t st);
void launch_adam(float* theta, const float* grad, float* m, float* v, long long n, int step,
                 float lr, float b1, float b2, float eps, cudaStream_t st);

}  // namespace sweep
