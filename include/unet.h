/*
 * unet.h -- C ABI of the learned gradient preconditioner in libsweep.so: a
 * U-Net run on the GB300 tensor cores (tcgen05) in BF16 with FP32
 * accumulation, with hand-written inference and training kernels.
 *
 * The paper (Sec. 1, Sec. 2.1) integrates neural networks with its solvers
 * through the same tensor operations but fixes no network.  This one maps a
 * raw FWI gradient (and the current model) to an estimate of the
 * illumination-compensated gradient; the FWI loop uses it only where the
 * solver's misfit confirms the step, with the plain preconditioned gradient
 * as fallback.
 *
 * Network (fixed): 4 resolution levels, 32/64/128/256 channels.  Every
 * convolution is 3 x 3, zero padded, cross-correlation, followed by ReLU:
 *   encoder level l = 1..3: conv, conv (output s_l), 2 x 2 average pool;
 *   bottleneck: conv 128 -> 256, conv 256 -> 256;
 *   decoder level l = 3..1: nearest 2x upsample, conv ("up") to the level's
 *     channels, concatenate [up output, s_l], conv, conv;
 *   head: 1 x 1 convolution 32 -> 1, no activation.
 * The input's in_ch channels are zero-padded to 32.
 *
 * Parameters: one flat FP32 vector of SWEEP_UNET_PARAMS values: for each of
 * the 17 convolutions in the order enc1a enc1b enc2a enc2b enc3a enc3b bota
 * botb up3 dec3a dec3b up2 dec2a dec2b up1 dec1a dec1b, the weights
 * W[cout][3][3][cin] then the bias[cout]; then the head's w[32], bias[1].
 * The kernels compute with the weights rounded to BF16 (round to nearest
 * even); biases, the head, the loss, gradients and Adam stay FP32 (FP64 for
 * the loss).  Activations are stored as BF16 NHWC; the backward pass stores
 * the gradient of every activation as BF16.
 *
 * Memory: every array is a DEVICE pointer; the caller owns all memory
 * including the workspace (256-byte aligned; its first word is the status
 * word that sweep_status() reads).  Calls are asynchronous on `stream`.
 * Host-visible errors (sizes, NULL pointers, workspace too small) return
 * before any launch; a device-side wait that gives up latches
 * SWEEP_ETIMEOUT in the status word.
 */
#ifndef SWEEP_UNET_H
#define SWEEP_UNET_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SWEEP_UNET_PARAMS 2148993LL

typedef struct {
  int32_t batch;  /* images per call, >= 1                                */
  int32_t height; /* H, a multiple of 128                                 */
  int32_t width;  /* W, a power of two >= 128                             */
  int32_t in_ch;  /* input channels, 1..32                                */
} sweep_unet_shape;

/* Number of parameters (SWEEP_UNET_PARAMS). */
long long sweep_unet_param_count(void);

/* Workspace bytes of sweep_unet_forward (training = 0) or
 * sweep_unet_gradient (training = 1) for `shape`; 0 on an invalid shape. */
size_t sweep_unet_workspace_bytes(const sweep_unet_shape* shape, int training);

/* Inference: output[b][y][x] (FP32) of the network for
 * input[b][y][x][in_ch] (FP32) with parameters theta. */
int sweep_unet_forward(const sweep_unet_shape* shape, const float* theta, const float* input,
                       float* output, void* ws, size_t ws_bytes, void* stream);

/* Training step without the update: forward, loss = mean over the
 * batch's pixels of (output - target)^2 into the device double *loss, and
 * its gradient with respect to theta (FP32, the flat layout) into grad.
 * output (FP32 [batch][H][W]) receives the forward output. */
int sweep_unet_gradient(const sweep_unet_shape* shape, const float* theta, const float* input,
                        const float* target, float* output, double* loss, float* grad, void* ws,
                        size_t ws_bytes, void* stream);

/* Adam (Kingma & Ba, bias-corrected) on n FP32 parameters:
 * m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
 * theta -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps);
 * step counts from 1. */
int sweep_unet_adam(float* theta, const float* grad, float* m, float* v, long long n,
                    int32_t step, float lr, float beta1, float beta2, float eps, void* stream);

/* Single 3 x 3 convolution (the tensor-core kernel the network runs), for
 * tests and reuse: out[b][y][x][co] = op(sum_{tap, ci} x[..shifted..][ci]
 * w[co][tap][ci] + bias[co]) with BF16 x [B][H][W][cin], w [cout][9][cin],
 * FP32 bias (or NULL), op 0 = none, 1 = ReLU, 2 = multiply by
 * (mask[b][y][x][co] > 0) (BF16 mask [B][H][W][cout]); BF16 out
 * [B][H][W][cout].  cin a multiple of 32, cout in 32..256 a multiple of 32,
 * W a power of two >= 16, H a multiple of 128 / min(W, 128).  BF16 arrays
 * are passed as uint16_t bit patterns.  ws: >= 256 bytes (status word). */
int sweep_unet_conv3x3(int32_t B, int32_t H, int32_t W, int32_t cin, int32_t cout,
                       const uint16_t* x, const uint16_t* w, const float* bias, int32_t op,
                       const uint16_t* mask, uint16_t* out, void* ws, size_t ws_bytes,
                       void* stream);

/* Weight gradient of the same convolution:
 * dw[co][tap][ci] = sum_{b, y, x} x[b][y + ky - 1][x + kx - 1][ci] dy[b][y][x][co]
 * (FP32 dw [cout][9][cin], tap = 3 ky + kx), with the workspace of
 * sweep_unet_wgrad_workspace_bytes(); same size rules as the convolution
 * (W a power of two >= 16, H a multiple of 64 / min(W, 64)). */
size_t sweep_unet_wgrad_workspace_bytes(int32_t B, int32_t H, int32_t W, int32_t cin,
                                        int32_t cout);
int sweep_unet_conv3x3_wgrad(int32_t B, int32_t H, int32_t W, int32_t cin, int32_t cout,
                             const uint16_t* x, const uint16_t* dy, float* dw, void* ws,
                             size_t ws_bytes, void* stream);

#ifdef __cplusplus
}
#endif
#endif
