// 3 x 3 convolutions of the U-Net preconditioner on the 5th-generation
// tensor cores (tcgen05, BF16 operands, FP32 accumulator in tensor memory).
//
// conv_kernel: one CTA per 128-pixel output tile computes all output
// channels: an implicit GEMM with M = 128 pixels, N = cout (<= 256), and
// K = 9 taps x cin, walked in (tap, channel chunk) steps.  Warp 0 stages the
// shifted input tile (a TMA box of the NHWC tensor at the tap's offset; the
// zero padding is the box's out-of-bounds fill) and the weights' (tap,
// chunk) slice into a 4-stage ring; warp 1 issues the MMAs of a stage
// (one per 16 channels) and releases it with a commit; then all four warps
// read the accumulator out of TMEM (one pixel per thread), add the bias,
// apply ReLU or the ReLU mask of the backward pass, and store BF16.
//
// wgrad_kernel: D[(tap, ci)][co] = sum over pixels of in[p + off(tap)][ci]
// dy[p][co]; a CTA owns 128 rows of (tap, ci) and a contiguous range of
// 64-pixel steps (split K); both operands are staged pixel-major by TMA,
// i.e. MN-major for the MMA.  Each CTA writes its FP32 partial sums; a
// reduction kernel adds the splits in a fixed order.
//
// Every mbarrier wait is bounded (tma.cuh); a wait that gives up latches
// SWEEP_ETIMEOUT, the CTA skips its stores, waits for its own copies in
// flight and frees its tensor memory before it exits.
#include <algorithm>
#include <mutex>

#include "sweep_internal.cuh"
#include "tcgen05.cuh"
#include "unet_internal.cuh"

namespace sweep {
namespace {

constexpr int kThreads = 128;
constexpr int kMaxStages = 4;
constexpr size_t kSmemPerSm = 228 * 1024;  // per SM, of which 1 KB per CTA is reserved
// dynamic shared memory the kernels may ask for: 4 stages of at most 48 KB
// and the 1 KB alignment slack (below the 227 KB opt-in limit, which also
// counts the kernels' static barriers)
constexpr int kMaxDynSmem = 4 * 48 * 1024 + 1024;

__host__ __device__ inline uint32_t tmem_cols(int n) {
  uint32_t c = 32;
  while (c < (uint32_t)n) c <<= 1;
  return c;
}

// whole-warp bounded wait (lane 0's outcome is the warp's)
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity) {
  bool got = mbar_wait(bar, parity);
  return __shfl_sync(0xffffffffu, got ? 1 : 0, 0) != 0;
}

__device__ __forceinline__ uint32_t pack2(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

__global__ void __launch_bounds__(kThreads, 1) conv_kernel(const __grid_constant__ ConvArgs a) {
  __shared__ __align__(8) uint64_t full[kMaxStages];
  __shared__ __align__(8) uint64_t empty[kMaxStages];
  __shared__ __align__(8) uint64_t done;
  __shared__ uint32_t tmem_holder;
  __shared__ int failed;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw_u = smem_u32(smem_raw);
  const uint32_t base_u = (raw_u + 1023u) & ~1023u;
  uint8_t* base = smem_raw + (base_u - raw_u);
  const int a_bytes = 128 * a.kc * 2;
  const int stage_bytes = a_bytes + a.cout * a.kc * 2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t ncols = tmem_cols(a.cout);
  const int S = a.stages;

  const int ntx = a.W / a.bw, nty = a.H / a.bh;
  int t = blockIdx.x;
  const int b = t / (ntx * nty);
  t -= b * ntx * nty;
  const int y0 = (t / ntx) * a.bh, x0 = (t % ntx) * a.bw;

  if (warp == 0) {
    tmem_alloc(&tmem_holder, ncols);
    tmem_relinquish();
  }
  if (threadIdx.x == 32) {
    for (int i = 0; i < S; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(&done, 1);
    failed = 0;
    fence_barrier_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_holder;

  const int nch = a.cin / a.kc;
  const int kiters = 9 * nch;
  if (warp == 0) {  // TMA producer
    int k = 0;
    for (; k < kiters; ++k) {
      const int s = k % S;
      if (k >= S && !warp_wait(&empty[s], ((k / S) - 1) & 1)) {
        if (lane == 0) {
          latch(a.status, SWEEP_ETIMEOUT);
          failed = 1;
        }
        break;
      }
      if (lane == 0) {
        const int tap = k / nch, ch = k - tap * nch;
        uint8_t* sa = base + (size_t)s * stage_bytes;
        mbar_arrive_expect_tx(&full[s], stage_bytes);
        tma_load_4d(sa, &a.tin, &full[s], ch * a.kc, x0 + tap % 3 - 1, y0 + tap / 3 - 1, b);
        tma_load_3d(sa + a_bytes, &a.tw, &full[s], ch * a.kc, tap, 0);
      }
      __syncwarp();
    }
    // the last copy into each stage has landed before the CTA may exit
    for (int j = k > S ? k - S : 0; j < k; ++j) warp_wait(&full[j % S], (j / S) & 1);
  } else if (warp == 1) {  // MMA issuer
    const uint32_t idesc = idesc_bf16_f32(128, a.cout, 0, 0);
    const uint32_t swz = a.kc == 64 ? kSwizzle128 : kSwizzle64;
    const uint32_t sbo = 8u * a.kc * 2u;
    for (int k = 0; k < kiters; ++k) {
      const int s = k % S;
      if (!warp_wait(&full[s], (k / S) & 1)) {
        if (lane == 0) {
          latch(a.status, SWEEP_ETIMEOUT);
          failed = 1;
        }
        break;
      }
      tc_fence_after();
      if (lane == 0) {
        const uint32_t sa = base_u + (uint32_t)(s * stage_bytes);
        const uint32_t sb = sa + (uint32_t)a_bytes;
        for (int j = 0; j < a.kc / 16; ++j)
          mma_bf16(tmem, smem_desc(sa + 32u * j, 16u, sbo, swz),
                   smem_desc(sb + 32u * j, 16u, sbo, swz), idesc, (k | j) != 0);
        mma_commit(&empty[s]);  // the stage is free once these MMAs have read it
      }
      __syncwarp();
    }
    if (lane == 0) mma_commit(&done);  // every MMA issued has completed
    __syncwarp();
  }

  const bool got = mbar_wait(&done, 0);
  const bool bad = __syncthreads_or(!got) || failed;
  tc_fence_after();
  if (!bad && kiters > 0) {
    const int r = warp * 32 + lane;  // accumulator lane = output pixel of the tile
    const long long pix = ((long long)b * a.H + (y0 + r / a.bw)) * a.W + (x0 + r % a.bw);
    bf16* op = a.out + pix * a.out_ps;
    const bf16* mp = a.op == kOpMask ? a.mask + pix * a.mask_ps : nullptr;
    for (int c0 = 0; c0 < a.cout; c0 += 32) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (a.bias) {
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] += a.bias[c0 + i];
      }
      if (a.op == kOpRelu) {
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = fmaxf(v[i], 0.f);
      } else if (a.op == kOpMask) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint4 m = *reinterpret_cast<const uint4*>(mp + c0 + 8 * q);
          const bf16* mb = reinterpret_cast<const bf16*>(&m);
#pragma unroll
          for (int i = 0; i < 8; ++i)
            if (!(__bfloat162float(mb[i]) > 0.f)) v[8 * q + i] = 0.f;
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint4 w;
        w.x = pack2(v[8 * q + 0], v[8 * q + 1]);
        w.y = pack2(v[8 * q + 2], v[8 * q + 3]);
        w.z = pack2(v[8 * q + 4], v[8 * q + 5]);
        w.w = pack2(v[8 * q + 6], v[8 * q + 7]);
        *reinterpret_cast<uint4*>(op + c0 + 8 * q) = w;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, ncols);
  }
}

__global__ void __launch_bounds__(kThreads, 1) wgrad_kernel(const __grid_constant__ WgradArgs a) {
  __shared__ __align__(8) uint64_t full[kMaxStages];
  __shared__ __align__(8) uint64_t empty[kMaxStages];
  __shared__ __align__(8) uint64_t done;
  __shared__ uint32_t tmem_holder;
  __shared__ int failed;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw_u = smem_u32(smem_raw);
  const uint32_t base_u = (raw_u + 1023u) & ~1023u;
  uint8_t* base = smem_raw + (base_u - raw_u);
  constexpr int kPix = 64;                // K per stage (pixels)
  constexpr int a_bytes = 128 * kPix * 2;  // 128 rows of (tap, ci) x 64 pixels
  const int stage_bytes = a_bytes + a.cout * kPix * 2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t ncols = tmem_cols(a.cout);
  const int S = a.stages;

  const int mt = blockIdx.x % a.mtiles, split = blockIdx.x / a.mtiles;
  const int ntx = a.W / a.pw, nty = a.H / a.ph;
  const long long T = (long long)a.B * ntx * nty;
  const long long t0 = T * split / a.splits, t1 = T * (split + 1) / a.splits;
  const int kiters = (int)(t1 - t0);
  const int rows = 9 * a.cin;

  if (warp == 0) {
    tmem_alloc(&tmem_holder, ncols);
    tmem_relinquish();
  }
  if (threadIdx.x == 32) {
    for (int i = 0; i < S; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(&done, 1);
    failed = 0;
    fence_barrier_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_holder;

  if (warp == 0) {  // TMA producer
    int k = 0;
    for (; k < kiters; ++k) {
      const int s = k % S;
      if (k >= S && !warp_wait(&empty[s], ((k / S) - 1) & 1)) {
        if (lane == 0) {
          latch(a.status, SWEEP_ETIMEOUT);
          failed = 1;
        }
        break;
      }
      if (lane == 0) {
        long long tt = t0 + k;
        const int b = (int)(tt / (ntx * nty));
        tt -= (long long)b * ntx * nty;
        const int y0 = (int)(tt / ntx) * a.ph, x0 = (int)(tt % ntx) * a.pw;
        uint8_t* sa = base + (size_t)s * stage_bytes;
        mbar_arrive_expect_tx(&full[s], stage_bytes);
        for (int q = 0; q < 128 / a.ka; ++q) {  // runs of ka rows: one (tap, ci chunk) each
          const int r0 = mt * 128 + q * a.ka;
          int tap = r0 / a.cin, ci0 = r0 - tap * a.cin;
          if (tap > 8) {  // rows past 9 cin: any valid tap; their sums are not stored
            tap = 8;
            ci0 = 0;
          }
          tma_load_4d(sa + q * (kPix * a.ka * 2), &a.tin, &full[s], ci0, x0 + tap % 3 - 1,
                      y0 + tap / 3 - 1, b);
        }
        for (int q = 0; q < a.cout / a.kb; ++q)
          tma_load_4d(sa + a_bytes + q * (kPix * a.kb * 2), &a.tdy, &full[s], q * a.kb, x0, y0,
                      b);
      }
      __syncwarp();
    }
    for (int j = k > S ? k - S : 0; j < k; ++j) warp_wait(&full[j % S], (j / S) & 1);
  } else if (warp == 1) {  // MMA issuer: both operands MN-major
    const uint32_t idesc = idesc_bf16_f32(128, a.cout, 1, 1);
    const uint32_t swa = a.ka == 64 ? kSwizzle128 : kSwizzle64;
    const uint32_t swb = a.kb == 64 ? kSwizzle128 : kSwizzle64;
    const uint32_t la = kPix * a.ka * 2, sba = 8u * a.ka * 2u;  // run stride, 8-line stride
    const uint32_t lb = kPix * a.kb * 2, sbb = 8u * a.kb * 2u;
    for (int k = 0; k < kiters; ++k) {
      const int s = k % S;
      if (!warp_wait(&full[s], (k / S) & 1)) {
        if (lane == 0) {
          latch(a.status, SWEEP_ETIMEOUT);
          failed = 1;
        }
        break;
      }
      tc_fence_after();
      if (lane == 0) {
        const uint32_t sa = base_u + (uint32_t)(s * stage_bytes);
        const uint32_t sb = sa + (uint32_t)a_bytes;
        for (int j = 0; j < kPix / 16; ++j)  // 16 pixels (K lines) per MMA
          mma_bf16(tmem, smem_desc(sa + 16u * j * a.ka * 2u, la, sba, swa),
                   smem_desc(sb + 16u * j * a.kb * 2u, lb, sbb, swb), idesc, (k | j) != 0);
        mma_commit(&empty[s]);
      }
      __syncwarp();
    }
    if (lane == 0) mma_commit(&done);
    __syncwarp();
  }

  const bool got = mbar_wait(&done, 0);
  const bool bad = __syncthreads_or(!got) || failed;
  tc_fence_after();
  if (!bad) {
    const int r = warp * 32 + lane;
    const int R = mt * 128 + r;
    float* out = a.partial + ((size_t)split * a.mtiles * 128 + R) * a.cout;
    for (int c0 = 0; c0 < a.cout; c0 += 32) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);  // all lanes
      if (R < rows) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          float4 w = kiters > 0 ? make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3])
                                : make_float4(0.f, 0.f, 0.f, 0.f);
          *reinterpret_cast<float4*>(out + c0 + 4 * q) = w;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, ncols);
  }
}

// Shared memory of a launch, raised if needed so that the CTAs that fit on
// one SM by shared memory never ask for more than the 512 TMEM columns.
size_t fit_tmem(size_t smem, int cout) {
  const size_t max_ctas = 512 / tmem_cols(cout);
  // with at least this much each, max_ctas + 1 CTAs do not fit on one SM
  const size_t floor_bytes = kSmemPerSm / (max_ctas + 1) + 1;
  return std::max(smem, floor_bytes);
}

}  // namespace

size_t conv_smem_bytes(int cout, int kc, int stages) {
  const size_t s = (size_t)stages * (128 * kc * 2 + (size_t)cout * kc * 2) + 1024;
  return fit_tmem(s, cout);
}

size_t wgrad_smem_bytes(int cout, int stages) {
  const size_t s = (size_t)stages * (128 * 64 * 2 + (size_t)cout * 64 * 2) + 1024;
  return fit_tmem(s, cout);
}

void launch_conv(const ConvArgs& a, cudaStream_t st) {
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(conv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
  });
  const int tiles = a.B * (a.H / a.bh) * (a.W / a.bw);
  if (tiles <= 0) return;
  conv_kernel<<<tiles, kThreads, conv_smem_bytes(a.cout, a.kc, a.stages), st>>>(a);
  note_launches(1);
}

void launch_wgrad(const WgradArgs& a, cudaStream_t st) {
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
  });
  wgrad_kernel<<<a.mtiles * a.splits, kThreads, wgrad_smem_bytes(a.cout, a.stages), st>>>(a);
  note_launches(1);
}

}  // namespace sweep
