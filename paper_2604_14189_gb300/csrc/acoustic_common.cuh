// Stencil coefficients and small device helpers of the acoustic engine.
//
// Scheme (Sec. 3.1.2, Eq. 2, in the update form of the Sec. 2.1 listing):
//   u^{n+1} = 2 u^n - u^{n-1} + K (Lx + Lz) + K f^n delta_s,  K = v^2 dt^2/dx^2
// with, per axis, L = D2 u^n away from the border and, inside the border,
//   W = D2 u^n + D1 psi^{n-1};  zeta^n = a zeta^{n-1} + b W;
//   psi^n = a psi^{n-1} + b D1 u^n;  L = W + zeta^n.
// D2, D1: 8th-order centred differences at unit spacing (1/dx^2 lives in K).
//
// Backward step n, the exact transpose written for mu = K lambda:
//   G  = (1 + b) mu^{n+1} + b zetabar^n            (per axis, per cell)
//   mu^n = 2 mu^{n+1} - mu^{n+2} + K sum_axes [D2 G - D1 (b psibar^n)]
//          + K R^T r^{n-1}
//   psibar^{n-1} = a psibar^n - D1 (m G),  m = 1 inside that axis' border
//   zetabar^{n-1} = a (mu^{n+1} + zetabar^n)
// Away from the border (4 cells or more) this is the forward update itself.
// Imaging on interior cells: graw += mu^{n+1} (D2x u^n + D2z u^n + f^n delta_s)
// and the interior wavefield runs backwards,
//   u^{n-1} = 2 u^n - u^{n+1} + K (Lap u^n + f^n delta_s),
// with the 4-cell ring around the interior restored from the forward save.
#pragma once

#include "sweep_internal.cuh"

namespace sweep {

constexpr float kC0 = -205.0f / 72.0f;
constexpr float kC1 = 8.0f / 5.0f;
constexpr float kC2 = -1.0f / 5.0f;
constexpr float kC3 = 8.0f / 315.0f;
constexpr float kC4 = -1.0f / 560.0f;
constexpr float kD1 = 4.0f / 5.0f;
constexpr float kD2 = -1.0f / 5.0f;
constexpr float kD3 = 4.0f / 105.0f;
constexpr float kD4 = -1.0f / 280.0f;

// second difference centred on c from the 8 neighbours m4..m1, p1..p4
__device__ __forceinline__ float d2(float m4, float m3, float m2, float m1, float c, float p1,
                                    float p2, float p3, float p4) {
  return kC0 * c + kC1 * (p1 + m1) + kC2 * (p2 + m2) + kC3 * (p3 + m3) + kC4 * (p4 + m4);
}
// first difference from the 8 neighbours
__device__ __forceinline__ float d1(float m4, float m3, float m2, float m1, float p1, float p2,
                                    float p3, float p4) {
  return kD1 * (p1 - m1) + kD2 * (p2 - m2) + kD3 * (p3 - m3) + kD4 * (p4 - m4);
}

__device__ __forceinline__ void f4a(const float4 v, float* o) {
  o[0] = v.x;
  o[1] = v.y;
  o[2] = v.z;
  o[3] = v.w;
}

__device__ __forceinline__ bool in_region(const Region& r, int z, int x) {
  return z >= r.z0 && z < r.z1 && x >= r.x0 && x < r.x1;
}

__device__ __forceinline__ bool x_border(const Geom& g, int x) {
  return x < g.P || x >= g.P + g.nx;
}
__device__ __forceinline__ bool z_border(const Geom& g, int z) {
  return z < g.P || z >= g.P + g.nz;
}
__device__ __forceinline__ bool interior(const Geom& g, int z, int x) {
  return z >= g.P && z < g.P + g.nz && x >= g.P && x < g.P + g.nx;
}

// Per-shot values a step kernel needs for every unit (source cell, this
// step's wavelet sample), staged in shared memory once per
// launch so that no unit waits on a dependent global load for them.
constexpr int kShotTable = 128;  // shots held in shared memory; more: global
struct ShotTable {
  int sz[kShotTable], sx[kShotTable];
  float fn[kShotTable];
};

__device__ __forceinline__ void load_shot_table(ShotTable& T, const Geom& g,
                                                const int32_t* src, const float* wavelet,
                                                int n) {
  if (g.nshot > kShotTable) return;
  for (int s = threadIdx.x; s < g.nshot; s += blockDim.x) {
    T.sz[s] = src[2 * s] + g.P;
    T.sx[s] = src[2 * s + 1] + g.P;
    T.fn[s] = (wavelet && n < g.nt) ? wavelet[(long long)s * g.nt + n] : 0.f;
  }
}

struct ShotInfo {
  int sz, sx;
  float fn;
};
__device__ __forceinline__ ShotInfo shot_info(const ShotTable& T, const Geom& g,
                                              const int32_t* src, const float* wavelet, int n,
                                              int s) {
  ShotInfo i;
  if (g.nshot <= kShotTable) {
    i.sz = T.sz[s];
    i.sx = T.sx[s];
    i.fn = T.fn[s];
  } else {
    i.sz = src[2 * s] + g.P;
    i.sx = src[2 * s + 1] + g.P;
    i.fn = (wavelet && n < g.nt) ? wavelet[(long long)s * g.nt + n] : 0.f;
  }
  return i;
}

}  // namespace sweep
