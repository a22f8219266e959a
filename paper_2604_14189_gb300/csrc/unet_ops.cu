// Element-wise and reduction kernels of the U-Net preconditioner: weight
// conversion to BF16 (and the mirrored transpose the data gradient uses),
// input packing, 2 x 2 average pooling, nearest 2x upsampling and their
// backward passes fused with the ReLU masks, the 1 x 1 head with the MSE
// loss, bias and weight-gradient reductions, and the Adam update.
//
// BF16 tensors are NHWC with channel counts that are multiples of 8, so a
// thread moves 8 channels (16 bytes) at a time.  Reductions are FP32 (FP64
// for the loss) with partial sums in a fixed order: the same inputs give the
// same bits.
#include "sweep_internal.cuh"
#include "unet_internal.cuh"

namespace sweep {
namespace {

constexpr int kT = 256;

__device__ __forceinline__ void unpack8(const uint4& u, float* f) {
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 t = __bfloat1622float2(h[i]);
    f[2 * i] = t.x;
    f[2 * i + 1] = t.y;
  }
}

__device__ __forceinline__ uint4 pack8(const float* f) {
  uint4 u;
  __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&u);
#pragma unroll
  for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
  return u;
}

__device__ __forceinline__ uint4 ld8(const bf16* p) { return *reinterpret_cast<const uint4*>(p); }
__device__ __forceinline__ void st8(bf16* p, uint4 v) { *reinterpret_cast<uint4*>(p) = v; }

int blocks_for(long long n, int per_block = kT) {
  long long b = (n + per_block - 1) / per_block;
  return (int)(b < 1 ? 1 : (b > 1048576 ? 1048576 : b));
}

__global__ void prep_weights_kernel(const float* __restrict__ theta, WeightPrepAll p,
                                    long long total) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    long long j = i;
    int l = 0;
    while (l < kUnetLayers - 1 && j >= (long long)p.l[l].cout * 9 * p.l[l].cin) {
      j -= (long long)p.l[l].cout * 9 * p.l[l].cin;
      ++l;
    }
    const WeightPrep& L = p.l[l];
    const float w = theta[L.off + j];
    const int ci = (int)(j % L.cin);
    const int tap = (int)((j / L.cin) % 9);
    const int co = (int)(j / ((long long)L.cin * 9));
    const bf16 h = __float2bfloat16_rn(w);
    L.w[j] = h;
    L.wt[((long long)ci * 9 + (8 - tap)) * L.cout + co] = h;
  }
}

__global__ void pack_input_kernel(const float* __restrict__ in, int in_ch, bf16* __restrict__ x0,
                                  long long npix) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npix;
       p += (long long)gridDim.x * blockDim.x) {
    float f[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) f[c] = c < in_ch ? in[p * in_ch + c] : 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) st8(x0 + p * 32 + 8 * q, pack8(f + 8 * q));
  }
}

// out[b][y][x][c] = 1/4 sum of the 2 x 2 block (8 channels per thread)
__global__ void pool_kernel(const bf16* __restrict__ s, int s_ps, bf16* __restrict__ out, int B,
                            int H, int W, int C) {
  const int h = H / 2, w = W / 2, g = C / 8;
  const long long n = (long long)B * h * w * g;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % g) * 8;
    long long p = i / g;
    const int x = (int)(p % w);
    p /= w;
    const int y = (int)(p % h);
    const int b = (int)(p / h);
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        float f[8];
        unpack8(ld8(s + (((long long)b * H + 2 * y + dy) * W + 2 * x + dx) * s_ps + c), f);
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] += f[k];
      }
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] *= 0.25f;
    st8(out + (((long long)b * h + y) * w + x) * C + c, pack8(acc));
  }
}

__global__ void upsample_kernel(const bf16* __restrict__ x, bf16* __restrict__ out, int B, int h,
                                int w, int C) {
  const int H = 2 * h, W = 2 * w, g = C / 8;
  const long long n = (long long)B * H * W * g;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % g) * 8;
    long long p = i / g;
    const int X = (int)(p % W);
    p /= W;
    const int Y = (int)(p % H);
    const int b = (int)(p / H);
    st8(out + (((long long)b * H + Y) * W + X) * C + c,
        ld8(x + (((long long)b * h + Y / 2) * w + X / 2) * C + c));
  }
}

__global__ void up_backward_mask_kernel(const bf16* __restrict__ g, int g_ps,
                                        const bf16* __restrict__ x, bf16* __restrict__ d, int B,
                                        int h, int w, int C) {
  const int H = 2 * h, W = 2 * w, ng = C / 8;
  const long long n = (long long)B * h * w * ng;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % ng) * 8;
    long long p = i / ng;
    const int xx = (int)(p % w);
    p /= w;
    const int y = (int)(p % h);
    const int b = (int)(p / h);
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        float f[8];
        unpack8(ld8(g + (((long long)b * H + 2 * y + dy) * W + 2 * xx + dx) * g_ps + c), f);
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] += f[k];
      }
    const long long o = (((long long)b * h + y) * w + xx) * C + c;
    float m[8];
    unpack8(ld8(x + o), m);
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (!(m[k] > 0.f)) acc[k] = 0.f;
    st8(d + o, pack8(acc));
  }
}

__global__ void pool_backward_combine_kernel(const bf16* __restrict__ gp,
                                             const bf16* __restrict__ s, int s_ps,
                                             const bf16* __restrict__ gskip, int gskip_ps,
                                             bf16* __restrict__ d, int B, int H, int W, int C) {
  const int ng = C / 8;
  const long long n = (long long)B * H * W * ng;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % ng) * 8;
    const long long p = i / ng;
    const int x = (int)(p % W);
    const int y = (int)((p / W) % H);
    const int b = (int)(p / ((long long)W * H));
    float a[8], m[8], k2[8];
    unpack8(ld8(gp + (((long long)b * (H / 2) + y / 2) * (W / 2) + x / 2) * C + c), a);
    unpack8(ld8(s + p * s_ps + c), m);
    unpack8(ld8(gskip + p * gskip_ps + c), k2);
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = (m[k] > 0.f ? 0.25f * a[k] : 0.f) + k2[k];
    st8(d + p * C + c, pack8(a));
  }
}

__global__ void head_forward_kernel(const bf16* __restrict__ x, const float* __restrict__ th,
                                    float* __restrict__ out, long long npix) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npix;
       p += (long long)gridDim.x * blockDim.x) {
    float acc = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float f[8];
      unpack8(ld8(x + p * 32 + 8 * q), f);
#pragma unroll
      for (int k = 0; k < 8; ++k) acc = fmaf(f[k], th[8 * q + k], acc);
    }
    out[p] = acc + th[32];
  }
}

// Per block: FP64 loss partial, FP32 partials of the 33 head gradients.
__global__ void __launch_bounds__(kT) head_backward_kernel(
    const bf16* __restrict__ x, const float* __restrict__ th, const float* __restrict__ out,
    const float* __restrict__ tgt, long long npix, bf16* __restrict__ dpre,
    double* __restrict__ lpart, float* __restrict__ hpart) {
  __shared__ double sl[kT];
  __shared__ float sh[kT / 32][33];
  const float scale = 2.0f / (float)npix;
  double l = 0.0;
  float gw[33];
#pragma unroll
  for (int k = 0; k < 33; ++k) gw[k] = 0.f;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npix;
       p += (long long)gridDim.x * blockDim.x) {
    const float r = out[p] - tgt[p];
    l += (double)r * (double)r;
    const float dout = scale * r;
    gw[32] += dout;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float f[8], o[8];
      unpack8(ld8(x + p * 32 + 8 * q), f);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        gw[8 * q + k] = fmaf(dout, f[k], gw[8 * q + k]);
        o[k] = f[k] > 0.f ? dout * th[8 * q + k] : 0.f;
      }
      st8(dpre + p * 32 + 8 * q, pack8(o));
    }
  }
  // block sums in a fixed order
  sl[threadIdx.x] = l;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 33; ++k) {
    float v = gw[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < kT; ++i) t += sl[i];
    lpart[blockIdx.x] = t;
  }
  if (threadIdx.x < 33) {
    float t = 0.f;
    for (int w = 0; w < kT / 32; ++w) t += sh[w][threadIdx.x];
    hpart[(long long)blockIdx.x * 33 + threadIdx.x] = t;
  }
}

__global__ void head_backward_total_kernel(const double* lpart, const float* hpart, int nb,
                                           long long npix, double* loss, float* grad_head) {
  if (threadIdx.x == 0 && loss) {
    double t = 0.0;
    for (int i = 0; i < nb; ++i) t += lpart[i];
    *loss = t / (double)npix;
  }
  if (threadIdx.x < 33) {
    float t = 0.f;
    for (int i = 0; i < nb; ++i) t += hpart[(long long)i * 33 + threadIdx.x];
    grad_head[threadIdx.x] = t;
  }
}

// partial[block][co] = sum over the block's pixels of dy[p][co]: a thread
// owns 8 channels (one 16-byte load per pixel) and every (256 / (cout / 8))-th
// pixel of the block's range; the block then adds its rows in a fixed order.
__global__ void __launch_bounds__(256) bias_grad_kernel(const bf16* __restrict__ dy, int ps,
                                                        int cout, long long npix,
                                                        float* __restrict__ partial) {
  __shared__ float red[256][9];
  const int groups = cout / 8;                  // 4 .. 32
  const int rows = blockDim.x / groups;         // pixels in flight per block
  const int g = threadIdx.x % groups, r = threadIdx.x / groups;
  const long long per = (npix + gridDim.x - 1) / gridDim.x;
  const long long p0 = blockIdx.x * per;
  const long long p1 = p0 + per < npix ? p0 + per : npix;
  float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (r < rows)
    for (long long p = p0 + r; p < p1; p += rows) {
      float f[8];
      unpack8(ld8(dy + p * ps + 8 * g), f);
#pragma unroll
      for (int k = 0; k < 8; ++k) acc[k] += f[k];
    }
#pragma unroll
  for (int k = 0; k < 8; ++k) red[threadIdx.x][k] = acc[k];
  __syncthreads();
  if (threadIdx.x < cout) {
    const int gg = threadIdx.x / 8, k = threadIdx.x % 8;
    float t = 0.f;
    for (int rr = 0; rr < rows; ++rr) t += red[rr * groups + gg][k];
    partial[(long long)blockIdx.x * cout + threadIdx.x] = t;
  }
}

// db[c] = sum_j partial[j][c]: warp w of the block adds the partials
// j = w, w + 8, ... for 32 channels (one per lane); the 8 warp sums are then
// added in a fixed order.
__global__ void __launch_bounds__(256) bias_grad_total_kernel(const float* partial, int nb,
                                                              int cout, float* db) {
  __shared__ float red[8][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + lane;
  float t0 = 0.f, t1 = 0.f;
  int j = w;
  for (; j + 8 < nb; j += 16) {
    t0 += partial[(long long)j * cout + c];
    t1 += partial[(long long)(j + 8) * cout + c];
  }
  if (j < nb) t0 += partial[(long long)j * cout + c];
  red[w][lane] = t0 + t1;
  __syncthreads();
  if (w == 0) {
    float t = 0.f;
    for (int k = 0; k < 8; ++k) t += red[k][lane];
    db[c] = t;
  }
}

// dW[co][row] = sum_s partial[s][row][co], row = tap cin + ci.  Block
// (row, 32 output channels): warp w adds the splits s = w, w + 8, ... with
// one coalesced 128-byte load per split; the 8 warp sums are added in a
// fixed order.
__global__ void __launch_bounds__(256) wgrad_reduce_kernel(const float* __restrict__ partial,
                                                           int splits, int rows_pad, int rows,
                                                           int cout, float* __restrict__ dW) {
  __shared__ float red[8][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int r = blockIdx.x, c = blockIdx.y * 32 + lane;
  const float* p = partial + (long long)r * cout + c;
  const long long stride = (long long)rows_pad * cout;
  float t0 = 0.f, t1 = 0.f;
  int s = w;
  for (; s + 8 < splits; s += 16) {
    t0 += p[s * stride];
    t1 += p[(s + 8) * stride];
  }
  if (s < splits) t0 += p[s * stride];
  red[w][lane] = t0 + t1;
  __syncthreads();
  if (w == 0) {
    float t = 0.f;
    for (int k = 0; k < 8; ++k) t += red[k][lane];
    dW[(long long)c * rows + r] = t;
  }
}

__global__ void adam_kernel(float* __restrict__ th, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, long long n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

}  // namespace

void launch_prep_weights(const float* theta, const WeightPrepAll& p, long long total_w,
                         cudaStream_t st) {
  prep_weights_kernel<<<blocks_for(total_w), kT, 0, st>>>(theta, p, total_w);
  note_launches(1);
}

void launch_pack_input(const float* in, int in_ch, bf16* x0, long long npix, cudaStream_t st) {
  pack_input_kernel<<<blocks_for(npix), kT, 0, st>>>(in, in_ch, x0, npix);
  note_launches(1);
}

void launch_pool(const bf16* s, int s_ps, bf16* out, int B, int H, int W, int C,
                 cudaStream_t st) {
  pool_kernel<<<blocks_for((long long)B * (H / 2) * (W / 2) * (C / 8)), kT, 0, st>>>(
      s, s_ps, out, B, H, W, C);
  note_launches(1);
}

void launch_upsample(const bf16* x, bf16* out, int B, int h, int w, int C, cudaStream_t st) {
  upsample_kernel<<<blocks_for((long long)B * 4 * h * w * (C / 8)), kT, 0, st>>>(x, out, B, h,
                                                                                w, C);
  note_launches(1);
}

void launch_up_backward_mask(const bf16* g, int g_ps, const bf16* x, bf16* d, int B, int h,
                             int w, int C, cudaStream_t st) {
  up_backward_mask_kernel<<<blocks_for((long long)B * h * w * (C / 8)), kT, 0, st>>>(
      g, g_ps, x, d, B, h, w, C);
  note_launches(1);
}

void launch_pool_backward_combine(const bf16* gp, const bf16* s, int s_ps, const bf16* gskip,
                                  int gskip_ps, bf16* d, int B, int H, int W, int C,
                                  cudaStream_t st) {
  pool_backward_combine_kernel<<<blocks_for((long long)B * H * W * (C / 8)), kT, 0, st>>>(
      gp, s, s_ps, gskip, gskip_ps, d, B, H, W, C);
  note_launches(1);
}

void launch_head_forward(const bf16* x, const float* theta_head, float* out, long long npix,
                         cudaStream_t st) {
  head_forward_kernel<<<blocks_for(npix), kT, 0, st>>>(x, theta_head, out, npix);
  note_launches(1);
}

void launch_head_backward(const bf16* x, const float* theta_head, const float* out,
                          const float* target, long long npix, bf16* dpre, double* partial,
                          int nblocks, double* loss, float* grad_head, cudaStream_t st) {
  // float partials of the head gradients follow the FP64 loss partials
  float* hpart = reinterpret_cast<float*>(partial + nblocks);
  head_backward_kernel<<<nblocks, kT, 0, st>>>(x, theta_head, out, target, npix, dpre, partial,
                                               hpart);
  head_backward_total_kernel<<<1, 64, 0, st>>>(partial, hpart, nblocks, npix, loss, grad_head);
  note_launches(2);
}

void launch_bias_grad(const bf16* dy, int dy_ps, int cout, long long npix, float* partial,
                      int nblocks, float* db, cudaStream_t st) {
  bias_grad_kernel<<<nblocks, 256, 0, st>>>(dy, dy_ps, cout, npix, partial);
  bias_grad_total_kernel<<<cout / 32, 256, 0, st>>>(partial, nblocks, cout, db);
  note_launches(2);
}

void launch_wgrad_reduce(const float* partial, int splits, int rows_padded, int cin, int cout,
                         float* dW, cudaStream_t st) {
  const int rows = 9 * cin;
  wgrad_reduce_kernel<<<dim3(rows, cout / 32), 256, 0, st>>>(partial, splits, rows_padded, rows,
                                                             cout, dW);
  note_launches(1);
}

void launch_adam(float* theta, const float* grad, float* m, float* v, long long n, int step,
                 float lr, float b1, float b2, float eps, cudaStream_t st) {
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  adam_kernel<<<blocks_for(n), kT, 0, st>>>(theta, grad, m, v, n, lr, b1, b2, eps, c1, c2);
  note_launches(1);
}

}  // namespace sweep
