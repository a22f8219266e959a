// Host side of include/unet.h: shape checks, workspace layout, tensor
// maps, and the launch sequences of the U-Net's forward pass, backward pass
// and Adam update.  No device memory is allocated here.
#include <algorithm>
#include <cstring>

#include "sweep.h"
#include "sweep_internal.cuh"
#include "tcgen05.cuh"
#include "unet.h"
#include "unet_internal.cuh"

namespace sweep {
namespace {

struct LayerDef {
  int cin, cout;
};
enum {
  ENC1A, ENC1B, ENC2A, ENC2B, ENC3A, ENC3B, BOTA, BOTB,
  UP3, DEC3A, DEC3B, UP2, DEC2A, DEC2B, UP1, DEC1A, DEC1B
};
constexpr LayerDef kLayer[kUnetLayers] = {
    {32, 32},   {32, 32},   {32, 64},   {64, 64},   {64, 128}, {128, 128},
    {128, 256}, {256, 256}, {256, 128}, {256, 128}, {128, 128}, {128, 64},
    {128, 64},  {64, 64},   {64, 32},   {64, 32},   {32, 32}};

long long layer_off(int l) {  // start of layer l's weights in the flat vector
  long long o = 0;
  for (int k = 0; k < l; ++k) o += (long long)kLayer[k].cout * 9 * kLayer[k].cin + kLayer[k].cout;
  return o;
}
long long head_off() { return layer_off(kUnetLayers); }
long long total_weights() {
  long long n = 0;
  for (int k = 0; k < kUnetLayers; ++k) n += (long long)kLayer[k].cout * 9 * kLayer[k].cin;
  return n;
}

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }
struct Bump {
  size_t off = 0;
  size_t take(size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes);
    return o;
  }
};

constexpr int kRedBlocks = 256;       // partial sums of the loss / head / bias reductions
constexpr int kMaxWgradCtas = 512;    // split-K CTAs of one weight-gradient launch
constexpr int kStages = 4;

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

bool valid_shape(const sweep_unet_shape* s) {
  if (!s) return false;
  if (s->batch < 1 || s->in_ch < 1 || s->in_ch > 32) return false;
  if (s->height < 128 || s->height % 128 != 0) return false;
  if (s->width < 128 || !pow2(s->width)) return false;
  if ((long long)s->batch * s->height * s->width * 256 >= (1LL << 40)) return false;
  return true;
}

// Buffers of one call (offsets into the workspace).
struct UnetLayout {
  size_t status = 0, lpart = 0, bpart = 0, wpart = 0;
  size_t w[kUnetLayers] = {}, wt[kUnetLayers] = {};
  // level 1 (H x W), 2 (H/2), 3 (H/4), 4 (H/8)
  size_t x0 = 0, a1 = 0, cat1 = 0, U1 = 0, da1 = 0, x1 = 0;
  size_t p1 = 0, a2 = 0, cat2 = 0, U2 = 0, da2 = 0, x2 = 0;
  size_t p2 = 0, a3 = 0, cat3 = 0, U3 = 0, da3 = 0, x3 = 0;
  size_t p3 = 0, ba = 0, bt = 0;
  // training: gradients of the activations (BF16)
  size_t G1 = 0, G2 = 0, Gc1 = 0, GU1 = 0, G13 = 0, G14 = 0;
  size_t G3 = 0, G4 = 0, Gc2 = 0, GU2 = 0, Gp1 = 0, G11 = 0, G12 = 0;
  size_t G5 = 0, G6 = 0, Gc3 = 0, GU3 = 0, Gp2 = 0, G9 = 0, G10 = 0;
  size_t G7 = 0, G8 = 0, Gp3 = 0;
  size_t total = 0;
};

UnetLayout layout(const sweep_unet_shape* s, bool training) {
  UnetLayout L;
  Bump b;
  const size_t B = s->batch, H = s->height, W = s->width;
  auto act = [&](int level, int C) {
    const size_t h = H >> (level - 1), w = W >> (level - 1);
    return b.take(B * h * w * (size_t)C * sizeof(bf16));
  };
  L.status = b.take(sizeof(int) * 4);
  L.lpart = b.take(sizeof(double) * kRedBlocks + sizeof(float) * 33 * kRedBlocks);
  L.bpart = b.take(sizeof(float) * kRedBlocks * 256);
  L.wpart = training ? b.take(sizeof(float) * (size_t)kMaxWgradCtas * 128 * 256) : 0;
  for (int l = 0; l < kUnetLayers; ++l) {
    const size_t n = (size_t)kLayer[l].cout * 9 * kLayer[l].cin * sizeof(bf16);
    L.w[l] = b.take(n);
    L.wt[l] = b.take(n);
  }
  L.x0 = act(1, 32); L.a1 = act(1, 32); L.cat1 = act(1, 64); L.U1 = act(1, 64);
  L.da1 = act(1, 32); L.x1 = act(1, 32);
  L.p1 = act(2, 32); L.a2 = act(2, 64); L.cat2 = act(2, 128); L.U2 = act(2, 128);
  L.da2 = act(2, 64); L.x2 = act(2, 64);
  L.p2 = act(3, 64); L.a3 = act(3, 128); L.cat3 = act(3, 256); L.U3 = act(3, 256);
  L.da3 = act(3, 128); L.x3 = act(3, 128);
  L.p3 = act(4, 128); L.ba = act(4, 256); L.bt = act(4, 256);
  if (training) {
    L.G1 = act(1, 32); L.G2 = act(1, 32); L.Gc1 = act(1, 64); L.GU1 = act(1, 64);
    L.G13 = act(1, 32); L.G14 = act(1, 32);
    L.G3 = act(2, 64); L.G4 = act(2, 64); L.Gc2 = act(2, 128); L.GU2 = act(2, 128);
    L.Gp1 = act(2, 32); L.G11 = act(2, 64); L.G12 = act(2, 64);
    L.G5 = act(3, 128); L.G6 = act(3, 128); L.Gc3 = act(3, 256); L.GU3 = act(3, 256);
    L.Gp2 = act(3, 64); L.G9 = act(3, 128); L.G10 = act(3, 128);
    L.G7 = act(4, 256); L.G8 = act(4, 256); L.Gp3 = act(4, 128);
  }
  L.total = b.off;
  return L;
}

template <typename T>
T* at(void* ws, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(ws) + off);
}

// A BF16 NHWC view: C channels of a buffer with pixel stride ps.
struct View {
  const bf16* p;
  int ps, C;
};

int kchunk(int c) { return c >= 64 ? 64 : 32; }

// Pipeline depth of a convolution: as many stages (2..4) as let two CTAs
// share an SM, so that one CTA's epilogue overlaps the other's main loop.
int conv_stages(int cout, int kc) {
  const int stage = 128 * kc * 2 + cout * kc * 2;
  const int budget = 112 * 1024 - 1024;  // half an SM's shared memory
  return std::max(2, std::min(kStages, budget / stage));
}

bool act_map(CUtensorMap* m, const View& v, int B, int H, int W, int kc, int bw, int bh) {
  const uint64_t dims[4] = {(uint64_t)v.C, (uint64_t)W, (uint64_t)H, (uint64_t)B};
  const uint64_t str[3] = {(uint64_t)v.ps, (uint64_t)W * v.ps, (uint64_t)H * W * v.ps};
  const uint32_t box[4] = {(uint32_t)kc, (uint32_t)bw, (uint32_t)bh, 1};
  return make_tensor_map_bf16(m, v.p, 4, dims, str, box, kc * 2);
}

bool weight_map(CUtensorMap* m, const bf16* w, int cin, int cout, int kc) {
  const uint64_t dims[3] = {(uint64_t)cin, 9, (uint64_t)cout};
  const uint64_t str[2] = {(uint64_t)cin, (uint64_t)cin * 9};
  const uint32_t box[3] = {(uint32_t)kc, 1, (uint32_t)cout};
  return make_tensor_map_bf16(m, w, 3, dims, str, box, kc * 2);
}

// One convolution on an H x W level: in (cin channels) * w [cout][9][cin].
int run_conv(int B, int H, int W, const View& in, const bf16* w, int cin, int cout,
             const float* bias, int op, const bf16* mask, int mask_ps, bf16* out, int out_ps,
             int* status, cudaStream_t st) {
  ConvArgs a{};
  a.B = B;
  a.H = H;
  a.W = W;
  a.cin = cin;
  a.cout = cout;
  a.kc = kchunk(cin);
  a.bw = std::min(W, 128);
  a.bh = 128 / a.bw;
  a.stages = conv_stages(cout, a.kc);
  a.bias = bias;
  a.op = op;
  a.mask = mask;
  a.mask_ps = mask_ps;
  a.out = out;
  a.out_ps = out_ps;
  a.status = status;
  if (H % a.bh != 0) return SWEEP_EINVAL;
  if (!act_map(&a.tin, in, B, H, W, a.kc, a.bw, a.bh)) return SWEEP_ECUDA;
  if (!weight_map(&a.tw, w, cin, cout, a.kc)) return SWEEP_ECUDA;
  launch_conv(a, st);
  return SWEEP_OK;
}

int wgrad_splits(int mtiles, long long T) {
  const int ctas = std::min(2 * device_sms(), kMaxWgradCtas);
  long long s = std::max(1, ctas / mtiles);
  s = std::min<long long>(s, T);
  return (int)std::max<long long>(s, 1);
}

// dW (FP32 [cout][9][cin]) of one convolution; partial: the split sums.
int run_wgrad(int B, int H, int W, const View& x, const View& dy, int cin, int cout, float* dW,
              float* partial, int* status, cudaStream_t st) {
  WgradArgs a{};
  a.B = B;
  a.H = H;
  a.W = W;
  a.cin = cin;
  a.cout = cout;
  a.ka = kchunk(cin);
  a.kb = kchunk(cout);
  a.pw = std::min(W, 64);
  a.ph = 64 / a.pw;
  if (H % a.ph != 0) return SWEEP_EINVAL;
  a.mtiles = (9 * cin + 127) / 128;
  const long long T = (long long)B * (H / a.ph) * (W / a.pw);
  a.splits = wgrad_splits(a.mtiles, T);
  a.stages = kStages;
  a.partial = partial;
  a.status = status;
  if (!act_map(&a.tin, x, B, H, W, a.ka, a.pw, a.ph)) return SWEEP_ECUDA;
  if (!act_map(&a.tdy, dy, B, H, W, a.kb, a.pw, a.ph)) return SWEEP_ECUDA;
  launch_wgrad(a, st);
  launch_wgrad_reduce(partial, a.splits, a.mtiles * 128, cin, cout, dW, st);
  return SWEEP_OK;
}

struct Net {
  const sweep_unet_shape* s;
  void* ws;
  UnetLayout L;
  cudaStream_t st;
  int* status;
  int B, H, W;

  bf16* p(size_t off) const { return at<bf16>(ws, off); }
  int h(int level) const { return H >> (level - 1); }
  int w(int level) const { return W >> (level - 1); }
  long long npix(int level) const { return (long long)B * h(level) * w(level); }

  int conv(int level, const View& in, int l, int op, const float* theta, bf16* out, int out_ps) {
    return run_conv(B, h(level), w(level), in, p(L.w[l]), kLayer[l].cin, kLayer[l].cout,
                    theta + layer_off(l) + (long long)kLayer[l].cout * 9 * kLayer[l].cin, op,
                    nullptr, 0, out, out_ps, status, st);
  }
  // data gradient of layer l: dpre (cout channels) -> its input's gradient
  int dgrad(int level, const View& dpre, int l, const bf16* mask, int mask_ps, bf16* out,
            int out_ps) {
    return run_conv(B, h(level), w(level), dpre, p(L.wt[l]), kLayer[l].cout, kLayer[l].cin,
                    nullptr, mask ? kOpMask : kOpNone, mask, mask_ps, out, out_ps, status, st);
  }
  int wgrad(int level, const View& x, const View& dpre, int l, float* grad) {
    float* dW = grad + layer_off(l);
    const int cin = kLayer[l].cin, cout = kLayer[l].cout;
    int rc = run_wgrad(B, h(level), w(level), x, dpre, cin, cout, dW, at<float>(ws, L.wpart),
                       status, st);
    if (rc) return rc;
    launch_bias_grad(dpre.p, dpre.ps, cout, npix(level), at<float>(ws, L.bpart), kRedBlocks,
                     dW + (long long)cout * 9 * cin, st);
    return SWEEP_OK;
  }
};

#define UNET_TRY(x)            \
  do {                         \
    const int rc_ = (x);       \
    if (rc_) return rc_;       \
  } while (0)

int prep(Net& n, const float* theta) {
  WeightPrepAll wp{};
  for (int l = 0; l < kUnetLayers; ++l) {
    wp.l[l].off = layer_off(l);
    wp.l[l].cin = kLayer[l].cin;
    wp.l[l].cout = kLayer[l].cout;
    wp.l[l].w = n.p(n.L.w[l]);
    wp.l[l].wt = n.p(n.L.wt[l]);
  }
  cudaMemsetAsync(n.status, 0, sizeof(int), n.st);
  launch_prep_weights(theta, wp, total_weights(), n.st);
  return SWEEP_OK;
}

int forward(Net& n, const float* theta, const float* input, float* output) {
  const UnetLayout& L = n.L;
  const int B = n.B;
  UNET_TRY(prep(n, theta));
  launch_pack_input(input, n.s->in_ch, n.p(L.x0), n.npix(1), n.st);
  // encoder
  UNET_TRY(n.conv(1, {n.p(L.x0), 32, 32}, ENC1A, kOpRelu, theta, n.p(L.a1), 32));
  UNET_TRY(n.conv(1, {n.p(L.a1), 32, 32}, ENC1B, kOpRelu, theta, n.p(L.cat1) + 32, 64));
  launch_pool(n.p(L.cat1) + 32, 64, n.p(L.p1), B, n.h(1), n.w(1), 32, n.st);
  UNET_TRY(n.conv(2, {n.p(L.p1), 32, 32}, ENC2A, kOpRelu, theta, n.p(L.a2), 64));
  UNET_TRY(n.conv(2, {n.p(L.a2), 64, 64}, ENC2B, kOpRelu, theta, n.p(L.cat2) + 64, 128));
  launch_pool(n.p(L.cat2) + 64, 128, n.p(L.p2), B, n.h(2), n.w(2), 64, n.st);
  UNET_TRY(n.conv(3, {n.p(L.p2), 64, 64}, ENC3A, kOpRelu, theta, n.p(L.a3), 128));
  UNET_TRY(n.conv(3, {n.p(L.a3), 128, 128}, ENC3B, kOpRelu, theta, n.p(L.cat3) + 128, 256));
  launch_pool(n.p(L.cat3) + 128, 256, n.p(L.p3), B, n.h(3), n.w(3), 128, n.st);
  // bottleneck
  UNET_TRY(n.conv(4, {n.p(L.p3), 128, 128}, BOTA, kOpRelu, theta, n.p(L.ba), 256));
  UNET_TRY(n.conv(4, {n.p(L.ba), 256, 256}, BOTB, kOpRelu, theta, n.p(L.bt), 256));
  // decoder
  launch_upsample(n.p(L.bt), n.p(L.U3), B, n.h(4), n.w(4), 256, n.st);
  UNET_TRY(n.conv(3, {n.p(L.U3), 256, 256}, UP3, kOpRelu, theta, n.p(L.cat3), 256));
  UNET_TRY(n.conv(3, {n.p(L.cat3), 256, 256}, DEC3A, kOpRelu, theta, n.p(L.da3), 128));
  UNET_TRY(n.conv(3, {n.p(L.da3), 128, 128}, DEC3B, kOpRelu, theta, n.p(L.x3), 128));
  launch_upsample(n.p(L.x3), n.p(L.U2), B, n.h(3), n.w(3), 128, n.st);
  UNET_TRY(n.conv(2, {n.p(L.U2), 128, 128}, UP2, kOpRelu, theta, n.p(L.cat2), 128));
  UNET_TRY(n.conv(2, {n.p(L.cat2), 128, 128}, DEC2A, kOpRelu, theta, n.p(L.da2), 64));
  UNET_TRY(n.conv(2, {n.p(L.da2), 64, 64}, DEC2B, kOpRelu, theta, n.p(L.x2), 64));
  launch_upsample(n.p(L.x2), n.p(L.U1), B, n.h(2), n.w(2), 64, n.st);
  UNET_TRY(n.conv(1, {n.p(L.U1), 64, 64}, UP1, kOpRelu, theta, n.p(L.cat1), 64));
  UNET_TRY(n.conv(1, {n.p(L.cat1), 64, 64}, DEC1A, kOpRelu, theta, n.p(L.da1), 32));
  UNET_TRY(n.conv(1, {n.p(L.da1), 32, 32}, DEC1B, kOpRelu, theta, n.p(L.x1), 32));
  launch_head_forward(n.p(L.x1), theta + head_off(), output, n.npix(1), n.st);
  return SWEEP_OK;
}

int backward(Net& n, const float* theta, const float* target, const float* output,
             double* loss, float* grad) {
  const UnetLayout& L = n.L;
  const int B = n.B;
  launch_head_backward(n.p(L.x1), theta + head_off(), output, target, n.npix(1), n.p(L.G1),
                       at<double>(n.ws, L.lpart), kRedBlocks, loss, grad + head_off(), n.st);
  // decoder level 1
  UNET_TRY(n.wgrad(1, {n.p(L.da1), 32, 32}, {n.p(L.G1), 32, 32}, DEC1B, grad));
  UNET_TRY(n.dgrad(1, {n.p(L.G1), 32, 32}, DEC1B, n.p(L.da1), 32, n.p(L.G2), 32));
  UNET_TRY(n.wgrad(1, {n.p(L.cat1), 64, 64}, {n.p(L.G2), 32, 32}, DEC1A, grad));
  UNET_TRY(n.dgrad(1, {n.p(L.G2), 32, 32}, DEC1A, n.p(L.cat1), 64, n.p(L.Gc1), 64));
  UNET_TRY(n.wgrad(1, {n.p(L.U1), 64, 64}, {n.p(L.Gc1), 64, 32}, UP1, grad));
  UNET_TRY(n.dgrad(1, {n.p(L.Gc1), 64, 32}, UP1, nullptr, 0, n.p(L.GU1), 64));
  launch_up_backward_mask(n.p(L.GU1), 64, n.p(L.x2), n.p(L.G3), B, n.h(2), n.w(2), 64, n.st);
  // decoder level 2
  UNET_TRY(n.wgrad(2, {n.p(L.da2), 64, 64}, {n.p(L.G3), 64, 64}, DEC2B, grad));
  UNET_TRY(n.dgrad(2, {n.p(L.G3), 64, 64}, DEC2B, n.p(L.da2), 64, n.p(L.G4), 64));
  UNET_TRY(n.wgrad(2, {n.p(L.cat2), 128, 128}, {n.p(L.G4), 64, 64}, DEC2A, grad));
  UNET_TRY(n.dgrad(2, {n.p(L.G4), 64, 64}, DEC2A, n.p(L.cat2), 128, n.p(L.Gc2), 128));
  UNET_TRY(n.wgrad(2, {n.p(L.U2), 128, 128}, {n.p(L.Gc2), 128, 64}, UP2, grad));
  UNET_TRY(n.dgrad(2, {n.p(L.Gc2), 128, 64}, UP2, nullptr, 0, n.p(L.GU2), 128));
  launch_up_backward_mask(n.p(L.GU2), 128, n.p(L.x3), n.p(L.G5), B, n.h(3), n.w(3), 128, n.st);
  // decoder level 3
  UNET_TRY(n.wgrad(3, {n.p(L.da3), 128, 128}, {n.p(L.G5), 128, 128}, DEC3B, grad));
  UNET_TRY(n.dgrad(3, {n.p(L.G5), 128, 128}, DEC3B, n.p(L.da3), 128, n.p(L.G6), 128));
  UNET_TRY(n.wgrad(3, {n.p(L.cat3), 256, 256}, {n.p(L.G6), 128, 128}, DEC3A, grad));
  UNET_TRY(n.dgrad(3, {n.p(L.G6), 128, 128}, DEC3A, n.p(L.cat3), 256, n.p(L.Gc3), 256));
  UNET_TRY(n.wgrad(3, {n.p(L.U3), 256, 256}, {n.p(L.Gc3), 256, 128}, UP3, grad));
  UNET_TRY(n.dgrad(3, {n.p(L.Gc3), 256, 128}, UP3, nullptr, 0, n.p(L.GU3), 256));
  launch_up_backward_mask(n.p(L.GU3), 256, n.p(L.bt), n.p(L.G7), B, n.h(4), n.w(4), 256, n.st);
  // bottleneck
  UNET_TRY(n.wgrad(4, {n.p(L.ba), 256, 256}, {n.p(L.G7), 256, 256}, BOTB, grad));
  UNET_TRY(n.dgrad(4, {n.p(L.G7), 256, 256}, BOTB, n.p(L.ba), 256, n.p(L.G8), 256));
  UNET_TRY(n.wgrad(4, {n.p(L.p3), 128, 128}, {n.p(L.G8), 256, 256}, BOTA, grad));
  UNET_TRY(n.dgrad(4, {n.p(L.G8), 256, 256}, BOTA, nullptr, 0, n.p(L.Gp3), 128));
  // encoder level 3
  launch_pool_backward_combine(n.p(L.Gp3), n.p(L.cat3) + 128, 256, n.p(L.Gc3) + 128, 256,
                               n.p(L.G9), B, n.h(3), n.w(3), 128, n.st);
  UNET_TRY(n.wgrad(3, {n.p(L.a3), 128, 128}, {n.p(L.G9), 128, 128}, ENC3B, grad));
  UNET_TRY(n.dgrad(3, {n.p(L.G9), 128, 128}, ENC3B, n.p(L.a3), 128, n.p(L.G10), 128));
  UNET_TRY(n.wgrad(3, {n.p(L.p2), 64, 64}, {n.p(L.G10), 128, 128}, ENC3A, grad));
  UNET_TRY(n.dgrad(3, {n.p(L.G10), 128, 128}, ENC3A, nullptr, 0, n.p(L.Gp2), 64));
  // encoder level 2
  launch_pool_backward_combine(n.p(L.Gp2), n.p(L.cat2) + 64, 128, n.p(L.Gc2) + 64, 128,
                               n.p(L.G11), B, n.h(2), n.w(2), 64, n.st);
  UNET_TRY(n.wgrad(2, {n.p(L.a2), 64, 64}, {n.p(L.G11), 64, 64}, ENC2B, grad));
  UNET_TRY(n.dgrad(2, {n.p(L.G11), 64, 64}, ENC2B, n.p(L.a2), 64, n.p(L.G12), 64));
  UNET_TRY(n.wgrad(2, {n.p(L.p1), 32, 32}, {n.p(L.G12), 64, 64}, ENC2A, grad));
  UNET_TRY(n.dgrad(2, {n.p(L.G12), 64, 64}, ENC2A, nullptr, 0, n.p(L.Gp1), 32));
  // encoder level 1
  launch_pool_backward_combine(n.p(L.Gp1), n.p(L.cat1) + 32, 64, n.p(L.Gc1) + 32, 64,
                               n.p(L.G13), B, n.h(1), n.w(1), 32, n.st);
  UNET_TRY(n.wgrad(1, {n.p(L.a1), 32, 32}, {n.p(L.G13), 32, 32}, ENC1B, grad));
  UNET_TRY(n.dgrad(1, {n.p(L.G13), 32, 32}, ENC1B, n.p(L.a1), 32, n.p(L.G14), 32));
  UNET_TRY(n.wgrad(1, {n.p(L.x0), 32, 32}, {n.p(L.G14), 32, 32}, ENC1A, grad));
  return SWEEP_OK;
}

bool ws_ok(void* ws, size_t ws_bytes, size_t need) {
  return ws && (reinterpret_cast<uintptr_t>(ws) % kAlign) == 0 && ws_bytes >= need;
}

int single_conv_shape_ok(int B, int H, int W, int cin, int cout, int pix_box) {
  if (B < 1 || cin < 32 || cin % 32 || cout < 32 || cout > 256 || cout % 32) return 0;
  if (W < 16 || !pow2(W) || H < 1) return 0;
  const int bw = std::min(W, pix_box), bh = pix_box / bw;
  if (H % bh) return 0;
  if ((long long)B * H * W * std::max(cin, cout) >= (1LL << 40)) return 0;
  return 1;
}

}  // namespace
}  // namespace sweep

using namespace sweep;

extern "C" long long sweep_unet_param_count(void) { return head_off() + 33; }

extern "C" size_t sweep_unet_workspace_bytes(const sweep_unet_shape* s, int training) {
  if (!valid_shape(s)) return 0;
  return layout(s, training != 0).total;
}

extern "C" int sweep_unet_forward(const sweep_unet_shape* s, const float* theta,
                                  const float* input, float* output, void* ws, size_t ws_bytes,
                                  void* stream) {
  if (!valid_shape(s)) return SWEEP_EINVAL;
  if (!theta || !input || !output) return SWEEP_EINVAL;
  Net n{s, ws, layout(s, false), static_cast<cudaStream_t>(stream), nullptr, s->batch,
        s->height, s->width};
  if (!ws_ok(ws, ws_bytes, n.L.total)) return SWEEP_EWORKSPACE;
  n.status = at<int>(ws, n.L.status);
  UNET_TRY(forward(n, theta, input, output));
  return cudaGetLastError() == cudaSuccess ? SWEEP_OK : SWEEP_ECUDA;
}

extern "C" int sweep_unet_gradient(const sweep_unet_shape* s, const float* theta,
                                   const float* input, const float* target, float* output,
                                   double* loss, float* grad, void* ws, size_t ws_bytes,
                                   void* stream) {
  if (!valid_shape(s)) return SWEEP_EINVAL;
  if (!theta || !input || !target || !output || !grad) return SWEEP_EINVAL;
  Net n{s, ws, layout(s, true), static_cast<cudaStream_t>(stream), nullptr, s->batch,
        s->height, s->width};
  if (!ws_ok(ws, ws_bytes, n.L.total)) return SWEEP_EWORKSPACE;
  n.status = at<int>(ws, n.L.status);
  UNET_TRY(forward(n, theta, input, output));
  UNET_TRY(backward(n, theta, target, output, loss, grad));
  return cudaGetLastError() == cudaSuccess ? SWEEP_OK : SWEEP_ECUDA;
}

extern "C" int sweep_unet_adam(float* theta, const float* grad, float* m, float* v, long long n,
                               int32_t step, float lr, float beta1, float beta2, float eps,
                               void* stream) {
  if (n < 0 || step < 1 || (n > 0 && (!theta || !grad || !m || !v))) return SWEEP_EINVAL;
  if (n == 0) return SWEEP_OK;
  launch_adam(theta, grad, m, v, n, step, lr, beta1, beta2, eps,
              static_cast<cudaStream_t>(stream));
  return cudaGetLastError() == cudaSuccess ? SWEEP_OK : SWEEP_ECUDA;
}

extern "C" int sweep_unet_conv3x3(int32_t B, int32_t H, int32_t W, int32_t cin, int32_t cout,
                                  const uint16_t* x, const uint16_t* w, const float* bias,
                                  int32_t op, const uint16_t* mask, uint16_t* out, void* ws,
                                  size_t ws_bytes, void* stream) {
  if (!single_conv_shape_ok(B, H, W, cin, cout, 128)) return SWEEP_EINVAL;
  if (!x || !w || !out || op < 0 || op > 2 || (op == kOpMask && !mask)) return SWEEP_EINVAL;
  if (!ws_ok(ws, ws_bytes, 16)) return SWEEP_EWORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int* status = static_cast<int*>(ws);
  cudaMemsetAsync(status, 0, sizeof(int), st);
  const View in{reinterpret_cast<const bf16*>(x), cin, cin};
  UNET_TRY(run_conv(B, H, W, in, reinterpret_cast<const bf16*>(w), cin, cout, bias, op,
                    reinterpret_cast<const bf16*>(mask), cout, reinterpret_cast<bf16*>(out), cout,
                    status, st));
  return cudaGetLastError() == cudaSuccess ? SWEEP_OK : SWEEP_ECUDA;
}

extern "C" size_t sweep_unet_wgrad_workspace_bytes(int32_t B, int32_t H, int32_t W,
                                                   int32_t cin, int32_t cout) {
  if (!single_conv_shape_ok(B, H, W, cin, cout, 64)) return 0;
  return kAlign + sizeof(float) * (size_t)kMaxWgradCtas * 128 * 256;
}

extern "C" int sweep_unet_conv3x3_wgrad(int32_t B, int32_t H, int32_t W, int32_t cin,
                                        int32_t cout, const uint16_t* x, const uint16_t* dy,
                                        float* dw, void* ws, size_t ws_bytes, void* stream) {
  if (!single_conv_shape_ok(B, H, W, cin, cout, 64)) return SWEEP_EINVAL;
  if (!x || !dy || !dw) return SWEEP_EINVAL;
  if (!ws_ok(ws, ws_bytes, sweep_unet_wgrad_workspace_bytes(B, H, W, cin, cout)))
    return SWEEP_EWORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int* status = static_cast<int*>(ws);
  cudaMemsetAsync(status, 0, sizeof(int), st);
  float* partial = reinterpret_cast<float*>(static_cast<char*>(ws) + kAlign);
  UNET_TRY(run_wgrad(B, H, W, {reinterpret_cast<const bf16*>(x), cin, cin},
                     {reinterpret_cast<const bf16*>(dy), cout, cout}, cin, cout, dw, partial,
                     status, st));
  return cudaGetLastError() == cudaSuccess ? SWEEP_OK : SWEEP_ECUDA;
}
