// Elastic adjoint: the exact transpose of one velocity-stress step
// (elastic.cu, Sec. 3.5, Eq. 12), and the chain rule from the step
// coefficients to (vp, vs, rho).
//
// Forward step n (unit-spacing staggered differences D, 1/dx folded into
// the coefficients c* = (dt/dx) x physical coefficient):
//   vx += cbx (Dpx txx + p1' + Dmz txz + p2'),  p1' = axh p1 + bxh Dpx txx ...
//   vz += cbz (Dmx txz + p3' + Dpz tzz + p4')
//   record v^{n+1/2};  Ex = Dmx vx + p5',  Ez = Dmz vz + p6'
//   txx += cl2m Ex + clam Ez;  tzz += clam Ex + cl2m Ez
//   txz += cmu (Dpz vx + p7' + Dpx vz + p8');  txx(s), tzz(s) += (dt/dx^2) f^n
// Its transpose, in reverse order, with T = adjoint of a quantity:
//   wavelet: f^n-bar = (dt/dx^2) (txx-bar + tzz-bar)(s)
//   stress:  Ex-bar = cl2m txx-bar + clam tzz-bar (Ez-bar likewise);
//            P = p5-bar + Ex-bar;  exx-bar = Ex-bar + bx P;  p5-bar = ax P
//            (p6..p8 alike); vx-bar += -Dpx(exx-bar) - Dmz(ezx-bar),
//            vz-bar += -Dpz(ezz-bar) - Dmx(exz-bar)      (Dp^T = -Dm)
//   receivers: v-bar(r) += residual^n(r)
//   velocity: Q = cbx vx-bar;  P = p1-bar + Q;  dxt-bar = Q + bxh P;
//            p1-bar = axh P (p2..p4 alike); txx-bar += -Dmx(dxt-bar), ...
//   coefficients (summed over shots and steps; see below for the precision):
//            d J / d cl2m += txx-bar Ex + tzz-bar Ez, d J / d clam +=
//            txx-bar Ez + tzz-bar Ex, d J / d cmu += txz-bar (shear bracket),
//            d J / d cbx += vx-bar (vx bracket), d J / d cbz likewise.
// Each half is one persistent kernel over (tile, shot group) units: a TMA
// pipeline stages, per shot, the tile with a halo of 2 rows and 4 columns
// (the fields the half reads around a cell and the coefficients); the
// block forms the four adjoint difference terms of the half on the whole
// box in shared memory, then applies their transposed differences to the
// tile's cells and sums the coefficient adjoints of the group's shots in
// registers (one addition per unit to the group's accumulators).  Those
// sums over shots and steps are compensated FP32 sums (double-float,
// about 44 significant bits), converted to FP64 and summed over the
// groups by the chain-rule kernel: FP64 arithmetic runs at a small
// fraction of the FP32 rate on this GPU, and plain FP64 accumulation cost
// a sixth of the elastic gradient's time.
//
// A memory variable and its adjoint stay zero wherever its profile pair
// (a, b) is zero, i.e. off its border strip (both start at zero and are
// only ever replaced by a x (...)); the kernels read and write them only on
// units whose box meets a strip.  A unit reads the adjoint memory variables
// of its halo, which the neighbouring tile's unit replaces in the same
// launch, so each step reads them from one buffer and writes them to the
// other (ap_in, ap_out; the caller swaps the two every step).
#include <algorithm>

#include "elastic_internal.cuh"
#include "tma.cuh"

namespace sweep {
namespace {

constexpr float kS1 = 9.0f / 8.0f;
constexpr float kS2 = -1.0f / 24.0f;

enum { G_L2M = 0, G_LAM = 1, G_MU = 2, G_BX = 3, G_BZ = 4 };

// ------------------------------------------------------------- wavelet
__global__ void el_adj_src_kernel(const ElAdjArgs a) {
  grid_dep_wait();
  grid_dep_trigger();
  if (*a.status) return;
  const Geom& g = a.g;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.nshot) return;
  const size_t c = (size_t)s * g.fstride + (size_t)(a.src[2 * s] + g.P) * g.NXp +
                   (a.src[2 * s + 1] + g.P);
  a.wgrad[(size_t)s * g.nt + a.n] = a.src_scale * (a.atxx[c] + a.atzz[c]);
}

// ------------------------------------------------------------ fused halves
constexpr int TA_Z = 16;         // tile rows: a warp per row
constexpr int TA_X = 128;        // tile columns: a lane per 4 cells
constexpr int A_H = TA_Z + 4;    // box rows: the tile's +- 2
constexpr int A_W = TA_X + 8;    // box columns: the tile's +- 4 (16-byte aligned x)
constexpr int A_BOX = A_H * A_W;
constexpr int A_G4 = A_W / 4;    // float4 groups per box row
constexpr int A_THREADS = 32 * TA_Z;
constexpr int A_STAGES = 2;
constexpr uint32_t kABox = A_BOX * 4;  // bytes of one staged field

struct __align__(128) AStrStage {  // per shot: adjoint stress, coefficients, forward v
  float txx[A_BOX], tzz[A_BOX], txz[A_BOX], l2m[A_BOX], lam[A_BOX], mu[A_BOX];
  float vx[A_BOX], vz[A_BOX];
};
struct __align__(128) AVelStage {  // per shot: adjoint velocity, buoyancies, forward tau
  float vx[A_BOX], vz[A_BOX], cbx[A_BOX], cbz[A_BOX];
  float txx[A_BOX], tzz[A_BOX], txz[A_BOX];
};
struct __align__(128) ATerms {  // the half's four difference terms on the box
  float t[4][A_BOX];
};
static_assert(kABox % 128 == 0, "staged field alignment");
constexpr size_t kATable = 64 * 16;  // unit descriptor table (A_TABLE int4)
static_assert(A_STAGES <= 2, "16 bytes of barriers");
constexpr size_t kAStrSmem = A_STAGES * sizeof(AStrStage) + sizeof(ATerms) + 16 + kATable;
constexpr size_t kAVelSmem = A_STAGES * sizeof(AVelStage) + sizeof(ATerms) + 16 + kATable;
static_assert(kAStrSmem <= 227 * 1024 && kAVelSmem <= 227 * 1024, "shared memory");

enum : int { AU_XS = 1, AU_ZS = 2, AU_PLAIN = 4 };
struct AUnit {
  int s, z0, x0, flags, grp;
  bool valid, first, last;
};

// Unit i of this CTA: unit blockIdx.x + i gridDim.x = (tile, group); its
// sub-units are the group's shots grp sg + k, k < sg (past the last shot:
// an empty sub-unit).  The tile part (s, valid, first, last unset).
__device__ __forceinline__ AUnit a_unit_base(const ElAdjArgs& a, int i) {
  const Geom& g = a.g;
  const int unit = blockIdx.x + i * gridDim.x;
  const int tile = unit / a.ngrp;
  AUnit u;
  u.grp = unit - tile * a.ngrp;
  const int tz = tile / a.ntx;
  u.z0 = tz * TA_Z;
  u.x0 = (tile - tz * a.ntx) * TA_X;
  int f = 0;  // the box meets a CPML strip (an integer or half-point profile is nonzero)
  if (g.P > 0 && (u.x0 - 4 < g.P || u.x0 + TA_X + 4 > g.P + g.nx - 1)) f |= AU_XS;
  if (g.P > 0 && (u.z0 - 2 < g.P || u.z0 + TA_Z + 2 > g.P + g.nz - 1)) f |= AU_ZS;
  // plain: no strip, and the box inside the grid; there every memory
  // variable and profile is zero, so exz-bar = ezx-bar (stress) and the two
  // terms of each velocity component are equal
  if (!f && u.z0 >= 2 && u.z0 + TA_Z + 2 <= g.NZ && u.x0 >= 4 && u.x0 + TA_X + 4 <= g.NX)
    f |= AU_PLAIN;
  u.flags = f;
  return u;
}

// Descriptors of this CTA's first A_TABLE units, made once per launch
// (the tile part, packed: z0, x0, flags, group); later units on the fly.
constexpr int A_TABLE = 64;
static_assert(A_TABLE * 16 == kATable, "descriptor table size");
struct ASub {  // position in this CTA's sub-unit sequence
  int i, k;    // unit, shot within its group
  __device__ __forceinline__ void next(int sg) {
    if (++k == sg) {
      k = 0;
      ++i;
    }
  }
};
__device__ __forceinline__ AUnit a_unit(const ElAdjArgs& a, const int4* tab, ASub q) {
  AUnit u;
  if (q.i < A_TABLE) {
    const int4 t = tab[q.i];
    u.z0 = t.x;
    u.x0 = t.y;
    u.flags = t.z;
    u.grp = t.w;
  } else {
    u = a_unit_base(a, q.i);
  }
  u.s = u.grp * a.sg + q.k;
  u.valid = u.s < a.g.nshot;
  u.first = q.k == 0;
  u.last = q.k == a.sg - 1;
  return u;
}

__device__ __forceinline__ float4 lda4(const float* t, int r, int c) {
  return *reinterpret_cast<const float4*>(t + r * A_W + c);
}
__device__ __forceinline__ void sta4(float* t, int r, int c, const float* v) {
  *reinterpret_cast<float4*>(t + r * A_W + c) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void v4(const float4 q, float* o) {
  o[0] = q.x;
  o[1] = q.y;
  o[2] = q.z;
  o[3] = q.w;
}
__device__ __forceinline__ float4 ld4z(const float* p, bool ok) {
  return ok ? *reinterpret_cast<const float4*>(p) : make_float4(0.f, 0.f, 0.f, 0.f);
}
__device__ __forceinline__ void st4v(float* p, const float* v) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
// 12 values of box row r, columns c0 .. c0+11
__device__ __forceinline__ void row12(const float* t, int r, int c0, float* e) {
  v4(lda4(t, r, c0), e);
  v4(lda4(t, r, c0 + 4), e + 4);
  v4(lda4(t, r, c0 + 8), e + 8);
}
// differences at the 4 cells c = 0..3 of a row window e[12] (cell c at
// e[4 + c]): D+ x and D- x
__device__ __forceinline__ float wdp(const float* e, int c) {
  return kS1 * (e[5 + c] - e[4 + c]) + kS2 * (e[6 + c] - e[3 + c]);
}
__device__ __forceinline__ float wdm(const float* e, int c) {
  return kS1 * (e[4 + c] - e[3 + c]) + kS2 * (e[5 + c] - e[2 + c]);
}
// and along z from rows R-2 .. R+2 of one column group (m2 .. p2)
__device__ __forceinline__ float zdp(float m1, float c0, float p1, float p2) {
  return kS1 * (p1 - c0) + kS2 * (p2 - m1);
}
__device__ __forceinline__ float zdm(float m2, float m1, float c0, float p1) {
  return kS1 * (c0 - m1) + kS2 * (p1 - m2);
}

// Compensated (double-float) sums: a value is hi + lo, two FP32 numbers;
// TwoSum (Knuth) adds an FP32 term with its rounding error kept in lo, so
// a sum keeps about 44 significant bits while every operation runs on the
// FP32 pipe (FP64 is far slower on this GPU).  __fadd_rn keeps the compiler
// from reassociating or contracting the error terms.
__device__ __forceinline__ void df_add(float& hi, float& lo, float x) {
  const float s = __fadd_rn(hi, x);
  const float bp = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
  hi = s;
  lo = __fadd_rn(lo, e);
}
// (H, L) += (hi, lo), renormalised so that |L| <= ulp(H) / 2
__device__ __forceinline__ void df_acc(float& H, float& L, float hi, float lo) {
  const float s = __fadd_rn(H, hi);
  const float bp = __fsub_rn(s, H);
  const float e = __fadd_rn(__fsub_rn(H, __fsub_rn(s, bp)), __fsub_rn(hi, bp));
  const float l = __fadd_rn(__fadd_rn(L, lo), e);
  H = __fadd_rn(s, l);
  L = __fsub_rn(l, __fsub_rn(H, s));
}
// Bring the accumulator planes of this thread's cells into L2 ahead of the
// flush at the end of the group's last shot (hi at G, lo at G + fstride)
__device__ __forceinline__ void df_prefetch(const float* G, long long fstride) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(G));
  asm volatile("prefetch.global.L2 [%0];" ::"l"(G + fstride));
}
__device__ __forceinline__ void pf_l2(const float* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}
// Strip units: bring the memory variables that the terms' phase reads (its
// box groups, adjoint, ap_in[m0], ap_in[m1] on x strips, [m2], [m3] on z
// strips) and the forward ones of this thread's cells (fp, gradient) into
// L2 before the stage wait.
__device__ __forceinline__ void strip_prefetch(const ElAdjArgs& a, const AUnit& u, size_t so,
                                               size_t ci, bool cell, bool grad, int m0, int m1,
                                               int m2, int m3) {
  const Geom& g = a.g;
  const bool xs = u.flags & AU_XS, zs = u.flags & AU_ZS;
  for (int gi = threadIdx.x; gi < A_H * A_G4; gi += A_THREADS) {
    const int br = gi / A_G4, bc = 4 * (gi - br * A_G4);
    const int zz = u.z0 - 2 + br, xx = u.x0 - 4 + bc;
    if (zz < 0 || zz >= g.NZ || xx < 0 || xx >= g.NXp) continue;
    const size_t c = so + (size_t)zz * g.NXp + xx;
    if (xs) {
      pf_l2(a.ap_in[m0] + c);
      pf_l2(a.ap_in[m1] + c);
    }
    if (zs) {
      pf_l2(a.ap_in[m2] + c);
      pf_l2(a.ap_in[m3] + c);
    }
  }
  if (cell && grad) {
    if (xs) {
      pf_l2(a.fp[m0] + ci);
      pf_l2(a.fp[m1] + ci);
    }
    if (zs) {
      pf_l2(a.fp[m2] + ci);
      pf_l2(a.fp[m3] + ci);
    }
  }
}
// Add this thread's 4 cells of one coefficient adjoint to the group's
// accumulator planes (hi at G, lo at G + fstride)
__device__ __forceinline__ void df_flush(float* G, long long fstride, const float* hi,
                                         const float* lo) {
  float H[4], L[4];
  v4(*reinterpret_cast<const float4*>(G), H);
  v4(*reinterpret_cast<const float4*>(G + fstride), L);
#pragma unroll
  for (int k = 0; k < 4; ++k) df_acc(H[k], L[k], hi[k], lo[k]);
  *reinterpret_cast<float4*>(G) = make_float4(H[0], H[1], H[2], H[3]);
  *reinterpret_cast<float4*>(G + fstride) = make_float4(L[0], L[1], L[2], L[3]);
}

// The persistent pipeline of both halves: sub-units in order, D stages.
// body(u, stage, wait) returns false when a transfer never landed.
template <typename Stage, typename Issue, typename Body, typename Ahead>
__device__ __forceinline__ void a_pipeline(const ElAdjArgs& a, unsigned char* smem_raw,
                                           Issue issue, Body body, Ahead ahead) {
  constexpr int D = A_STAGES;
  Stage* stg = reinterpret_cast<Stage*>(smem_raw);
  uint64_t* bar =
      reinterpret_cast<uint64_t*>(smem_raw + D * sizeof(Stage) + sizeof(ATerms));
  int4* tab = reinterpret_cast<int4*>(bar + 2);  // (barriers: 16 bytes reserved)
  const int G = gridDim.x;
  const int nunit = (a.units - (int)blockIdx.x + G - 1) / G;
  const int count = nunit * a.sg;
  if (count <= 0) return;
  for (int i = threadIdx.x; i < nunit && i < A_TABLE; i += A_THREADS) {
    const AUnit u = a_unit_base(a, i);
    tab[i] = make_int4(u.z0, u.x0, u.flags, u.grp);
  }
  // (programmatic launch: the table above overlaps the previous kernel's
  // tail; everything below reads what earlier kernels wrote)
  grid_dep_wait();
  // one reader of the status word, so that the whole block returns together
  if (__syncthreads_or(threadIdx.x == 0 && *a.status != 0)) return;
  ASub qi{0, 0};  // next sub-unit to issue (thread 0)
  if (threadIdx.x == 0) {
    for (int i = 0; i < D; ++i) mbar_init(&bar[i], 1);
    fence_barrier_init();
    for (int k = 0; k < D && k < count; ++k) {
      issue(stg[k], &bar[k], a_unit(a, tab, qi));
      qi.next(a.sg);
    }
  }
  __syncthreads();
  ASub q{0, 0};
  ahead(a_unit(a, tab, q));
  int k = 0;
  for (; k < count; ++k) {
    if (k == count - 1) grid_dep_trigger();  // the next kernel may start
    const AUnit u = a_unit(a, tab, q);
    const bool ok = body(u, stg[k % D], [&]() {
      const bool got = mbar_wait(&bar[k % D], (k / D) & 1);
      return !__syncthreads_or(!got);
    });
    if (!ok) break;  // uniform: a transfer never landed
    if (k + 1 < count) {  // the next sub-unit's global reads, into L2
      ASub qn = q;
      qn.next(a.sg);
      ahead(a_unit(a, tab, qn));
    }
    __syncthreads();  // stage and terms released
    if (threadIdx.x == 0 && k + D < count) {
      fence_proxy_async_smem();
      issue(stg[k % D], &bar[k % D], a_unit(a, tab, qi));
      qi.next(a.sg);
    }
    q.next(a.sg);
  }
  if (k < count && threadIdx.x == 0) {
    latch(const_cast<int*>(a.status), SWEEP_ETIMEOUT);
    for (int j = k; j < count && j < k + D; ++j) mbar_wait(&bar[j % D], (j / D) & 1);
  }
}

// A replayed forward memory variable is valid only on the tiles that meet
// its strip (the replay writes it nowhere else): read it where its profile
// pair is nonzero, 0 elsewhere.  pa, pb: the pair, at cells x .. x+3 (x axis) or row z.
__device__ __forceinline__ void fp_x(const float* f, const float* pa, const float* pb, int x,
                                     bool ok, float* o) {
  float A[4], B[4], v[4];
  v4(ld4z(pa + x, ok), A);
  v4(ld4z(pb + x, ok), B);
  v4(ld4z(f, ok), v);
#pragma unroll
  for (int k = 0; k < 4; ++k) o[k] = (A[k] != 0.f || B[k] != 0.f) ? v[k] : 0.f;
}
__device__ __forceinline__ void fp_z(const float* f, const float* pa, const float* pb, int z,
                                     bool ok, float* o) {
  const bool on = ok && (__ldg(pa + z) != 0.f || __ldg(pb + z) != 0.f);
  v4(ld4z(f, on), o);
}

// profiles of the 4 cells x .. x+3 (zero outside [0, NX)) and of row z
struct XProf {
  float a[4], b[4], ah[4], bh[4];
};
__device__ __forceinline__ void x_prof(const ElAdjArgs& a, int x, XProf& p) {
  const bool ok = x >= 0 && x < a.g.NXp;  // (the arrays are zero on [NX, NXp))
  v4(ld4z(a.ax + x, ok), p.a);
  v4(ld4z(a.bx + x, ok), p.b);
  v4(ld4z(a.axh + x, ok), p.ah);
  v4(ld4z(a.bxh + x, ok), p.bh);
}

// ----------------------------------------------------------------- stress
// The transpose of the stress update: terms exx-bar (t0), ezz-bar (t1),
// ezx-bar (t2), exz-bar (t3) on the box; v-bar -= D^T of them on the tile;
// d J / d (cl2m, clam, cmu) from the forward v^{n+1/2} and p5..p8.
__global__ void __launch_bounds__(A_THREADS, 1)
    el_adj_str_kernel(const __grid_constant__ ElAdjArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const Geom& g = a.g;
  ATerms& T = *reinterpret_cast<ATerms*>(smem_raw + A_STAGES * sizeof(AStrStage));
  const bool grad = a.gacc != nullptr;
  const int lane = threadIdx.x & 31, r = threadIdx.x >> 5, lx = 4 * lane;
  float acc[3][4], acl[3][4];  // coefficient adjoints of the group's shots (hi, lo)
  auto issue = [&](AStrStage& sg, uint64_t* b, const AUnit& u) {
    if (!u.valid) {
      mbar_arrive_expect_tx(b, 0);  // completes the phase: nothing to copy
      return;
    }
    mbar_arrive_expect_tx(b, (grad ? 8 : 6) * kABox);
    const int x = u.x0 - 4, y = u.z0 - 2;
    tma_load_3d(sg.txx, &a.m_atxx, b, x, y, u.s);
    tma_load_3d(sg.tzz, &a.m_atzz, b, x, y, u.s);
    tma_load_3d(sg.txz, &a.m_atxz, b, x, y, u.s);
    tma_load_2d(sg.l2m, &a.m_l2m, b, x, y);
    tma_load_2d(sg.lam, &a.m_lam, b, x, y);
    tma_load_2d(sg.mu, &a.m_mu, b, x, y);
    if (grad) {
      tma_load_3d(sg.vx, &a.m_fvx, b, x, y, u.s);
      tma_load_3d(sg.vz, &a.m_fvz, b, x, y, u.s);
    }
  };
  auto body = [&](const AUnit& u, const AStrStage& sg, auto wait) {
    if (u.first) {
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[k][c] = acl[k][c] = 0.f;
    }
    const size_t so = (size_t)u.s * g.fstride;
    const bool xs = u.flags & AU_XS, zs = u.flags & AU_ZS;
    // this thread's tile cells: adjoint velocities (updated) and the forward
    // memory variables p5..p8 (gradient), loaded before the stage wait
    const int z = u.z0 + r, x = u.x0 + lx;
    const bool cell = u.valid && z < g.NZ && x < g.NXp;
    const size_t ci = so + (size_t)z * g.NXp + x;
    float vx[4], vz[4];
    v4(ld4z(a.avx + ci, cell), vx);
    v4(ld4z(a.avz + ci, cell), vz);
    const bool flush = u.last && grad && z < g.NZ && x < g.NXp;
    float* const ga = a.gacc + (size_t)u.grp * 10 * g.fstride + (size_t)z * g.NXp + x;
    if (!wait()) return false;
    const bool plain = u.flags & AU_PLAIN;
    if (u.valid && plain) {
      // 1. (plain unit) exx-bar, ezz-bar and ezx-bar = exz-bar on the box
      for (int gi = threadIdx.x; gi < A_H * A_G4; gi += A_THREADS) {
        const int br = gi / A_G4, bc = 4 * (gi - br * A_G4);
        float txx[4], tzz[4], txz[4], l2m[4], lam[4], mu[4], e0[4], e1[4], e2[4];
        v4(lda4(sg.txx, br, bc), txx);
        v4(lda4(sg.tzz, br, bc), tzz);
        v4(lda4(sg.txz, br, bc), txz);
        v4(lda4(sg.l2m, br, bc), l2m);
        v4(lda4(sg.lam, br, bc), lam);
        v4(lda4(sg.mu, br, bc), mu);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          e0[k] = l2m[k] * txx[k] + lam[k] * tzz[k];
          e1[k] = lam[k] * txx[k] + l2m[k] * tzz[k];
          e2[k] = mu[k] * txz[k];
        }
        sta4(T.t[0], br, bc, e0);
        sta4(T.t[1], br, bc, e1);
        sta4(T.t[2], br, bc, e2);
      }
    } else if (u.valid) {
      // 1. the terms on the whole box; new p5..p8 on the tile's own cells
      for (int gi = threadIdx.x; gi < A_H * A_G4; gi += A_THREADS) {
        const int br = gi / A_G4, bc = 4 * (gi - br * A_G4);
        const int zz = u.z0 - 2 + br, xx = u.x0 - 4 + bc;
        const bool zin = zz >= 0 && zz < g.NZ;
        const bool gin = zin && xx >= 0 && xx < g.NXp;  // the group lies in the arrays
        const size_t c = so + (size_t)zz * g.NXp + xx;
        float txx[4], tzz[4], txz[4], l2m[4], lam[4], mu[4];
        v4(lda4(sg.txx, br, bc), txx);
        v4(lda4(sg.tzz, br, bc), tzz);
        v4(lda4(sg.txz, br, bc), txz);
        v4(lda4(sg.l2m, br, bc), l2m);
        v4(lda4(sg.lam, br, bc), lam);
        v4(lda4(sg.mu, br, bc), mu);
        XProf px;
        float q5[4], q6[4], q7[4], q8[4];
        x_prof(a, xs ? xx : -4, px);
        v4(ld4z(a.ap_in[4] + c, gin && xs), q5);
        v4(ld4z(a.ap_in[7] + c, gin && xs), q8);
        v4(ld4z(a.ap_in[5] + c, gin && zs), q6);
        v4(ld4z(a.ap_in[6] + c, gin && zs), q7);
        const float A6 = zs && zin ? __ldg(a.az + zz) : 0.f, B6 = zs && zin ? __ldg(a.bz + zz) : 0.f;
        const float A7 = zs && zin ? __ldg(a.azh + zz) : 0.f, B7 = zs && zin ? __ldg(a.bzh + zz) : 0.f;
        float e0[4], e1[4], e2[4], e3[4], n5[4], n6[4], n7[4], n8[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const bool in = zin && xx + k >= 0 && xx + k < g.NX;
          // txz += cmu (ezx + p7' + exz + p8')
          const float Tz = mu[k] * txz[k];
          const float P7 = q7[k] + Tz, P8 = q8[k] + Tz;
          e2[k] = in ? Tz + B7 * P7 : 0.f;        // ezx-bar
          e3[k] = in ? Tz + px.bh[k] * P8 : 0.f;  // exz-bar
          n7[k] = A7 * P7;
          n8[k] = px.ah[k] * P8;
          // txx += cl2m Ex + clam Ez, tzz += clam Ex + cl2m Ez
          const float Ex = l2m[k] * txx[k] + lam[k] * tzz[k];
          const float Ez = lam[k] * txx[k] + l2m[k] * tzz[k];
          const float P5 = q5[k] + Ex, P6 = q6[k] + Ez;
          e0[k] = in ? Ex + px.b[k] * P5 : 0.f;   // exx-bar
          e1[k] = in ? Ez + B6 * P6 : 0.f;        // ezz-bar
          n5[k] = px.a[k] * P5;
          n6[k] = A6 * P6;
        }
        sta4(T.t[0], br, bc, e0);
        sta4(T.t[1], br, bc, e1);
        sta4(T.t[2], br, bc, e2);
        sta4(T.t[3], br, bc, e3);
        const bool own = gin && br >= 2 && br < 2 + TA_Z && bc >= 4 && bc < 4 + TA_X;
        if (own && xs) {
          st4v(a.ap_out[4] + c, n5);
          st4v(a.ap_out[7] + c, n8);
        }
        if (own && zs) {
          st4v(a.ap_out[5] + c, n6);
          st4v(a.ap_out[6] + c, n7);
        }
      }
    }
    if (u.valid) {
      __syncthreads();
      // 2. v-bar -= D^T terms on the tile; coefficient adjoints (the forward
      // memory variables p5..p8 read here: only strip units have them)
      if (cell) {
        float f5[4], f6[4], f7[4], f8[4];
        fp_x(a.fp[4] + ci, a.ax, a.bx, x, grad && xs, f5);
        fp_x(a.fp[7] + ci, a.axh, a.bxh, x, grad && xs, f8);
        fp_z(a.fp[5] + ci, a.az, a.bz, z, grad && zs, f6);
        fp_z(a.fp[6] + ci, a.azh, a.bzh, z, grad && zs, f7);
        const int R = r + 2;
        float e[12], f[12];
        row12(T.t[0], R, lx, e);  // exx-bar
        row12(plain ? T.t[2] : T.t[3], R, lx, f);  // exz-bar
        float m2[4], m1[4], c0[4], p1[4];
        v4(lda4(T.t[2], R - 2, lx + 4), m2);  // ezx-bar rows R-2 .. R+1
        v4(lda4(T.t[2], R - 1, lx + 4), m1);
        v4(lda4(T.t[2], R, lx + 4), c0);
        v4(lda4(T.t[2], R + 1, lx + 4), p1);
        float n1[4], n0[4], q1[4], q2[4];
        v4(lda4(T.t[1], R - 1, lx + 4), n1);  // ezz-bar rows R-1 .. R+2
        v4(lda4(T.t[1], R, lx + 4), n0);
        v4(lda4(T.t[1], R + 1, lx + 4), q1);
        v4(lda4(T.t[1], R + 2, lx + 4), q2);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (x + k >= g.NX) continue;
          vx[k] -= wdp(e, k) + zdm(m2[k], m1[k], c0[k], p1[k]);
          vz[k] -= zdp(n1[k], n0[k], q1[k], q2[k]) + wdm(f, k);
        }
        st4v(a.avx + ci, vx);
        st4v(a.avz + ci, vz);
        if (grad) {
          float w[12], y[12];
          row12(sg.vx, R, lx, w);
          row12(sg.vz, R, lx, y);
          float xm1[4], xp1[4], xp2[4], zm2[4], zm1[4], zp1[4];
          v4(lda4(sg.vx, R - 1, lx + 4), xm1);  // vx rows R-1 .. R+2
          v4(lda4(sg.vx, R + 1, lx + 4), xp1);
          v4(lda4(sg.vx, R + 2, lx + 4), xp2);
          v4(lda4(sg.vz, R - 2, lx + 4), zm2);  // vz rows R-2 .. R+1
          v4(lda4(sg.vz, R - 1, lx + 4), zm1);
          v4(lda4(sg.vz, R + 1, lx + 4), zp1);
          float txx[4], tzz[4], txz[4];
          v4(lda4(sg.txx, R, lx + 4), txx);
          v4(lda4(sg.tzz, R, lx + 4), tzz);
          v4(lda4(sg.txz, R, lx + 4), txz);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            if (x + k >= g.NX) continue;
            const float ex = wdm(w, k) + f5[k];
            const float ez = zdm(zm2[k], zm1[k], y[4 + k], zp1[k]) + f6[k];
            const float sxz = zdp(xm1[k], w[4 + k], xp1[k], xp2[k]) + f7[k] + wdp(y, k) + f8[k];
            df_add(acc[0][k], acl[0][k], txx[k] * ex + tzz[k] * ez);
            df_add(acc[1][k], acl[1][k], txx[k] * ez + tzz[k] * ex);
            df_add(acc[2][k], acl[2][k], txz[k] * sxz);
          }
        }
      }
    }
    if (flush) {
      df_flush(ga + 2 * G_L2M * g.fstride, g.fstride, acc[0], acl[0]);
      df_flush(ga + 2 * G_LAM * g.fstride, g.fstride, acc[1], acl[1]);
      df_flush(ga + 2 * G_MU * g.fstride, g.fstride, acc[2], acl[2]);
    }
    return true;
  };
  // global reads of a sub-unit, brought into L2 while the one before runs
  auto ahead = [&](const AUnit& u) {
    const int z = u.z0 + r, x = u.x0 + lx;
    const size_t so = (size_t)u.s * g.fstride;
    const size_t ci = so + (size_t)z * g.NXp + x;
    const bool cell = u.valid && z < g.NZ && x < g.NXp;
    if (u.last && grad && z < g.NZ && x < g.NXp) {
      const float* ga = a.gacc + (size_t)u.grp * 10 * g.fstride + (size_t)z * g.NXp + x;
      df_prefetch(ga + 2 * G_L2M * g.fstride, g.fstride);
      df_prefetch(ga + 2 * G_LAM * g.fstride, g.fstride);
      df_prefetch(ga + 2 * G_MU * g.fstride, g.fstride);
    }
    if (cell) {  // the adjoint velocities it updates
      pf_l2(a.avx + ci);
      pf_l2(a.avz + ci);
    }
    if (u.valid && !(u.flags & AU_PLAIN)) strip_prefetch(a, u, so, ci, cell, grad, 4, 7, 5, 6);
  };
  a_pipeline<AStrStage>(a, smem_raw, issue, body, ahead);
}

// ---------------------------------------------------------------- receivers
__global__ void el_adj_rec_kernel(const ElAdjArgs a) {
  grid_dep_wait();
  grid_dep_trigger();
  if (*a.status) return;
  const Geom& g = a.g;
  const int r = blockIdx.x * blockDim.x + threadIdx.x, s = blockIdx.y;
  if (r >= g.nrec) return;
  const int32_t* q = a.rec + 2 * ((size_t)s * g.nrec + r);
  const size_t c = (size_t)s * g.fstride + (size_t)(q[0] + g.P) * g.NXp + (q[1] + g.P);
  // atomic: several receivers of a shot may share a cell (their residuals
  // add up, as in the transpose of recording each of them)
  atomicAdd(a.avx + c, a.res[(((size_t)s * 2 + 0) * g.nrec + r) * g.nt + a.n]);
  atomicAdd(a.avz + c, a.res[(((size_t)s * 2 + 1) * g.nrec + r) * g.nt + a.n]);
}

// --------------------------------------------------------------- velocity
// The transpose of the velocity update: terms dxt-bar of Dpx txx (t0), of
// Dmz txz (t1), of Dmx txz (t2), of Dpz tzz (t3) on the box; tau-bar -= D^T
// of them on the tile; d J / d (cbx, cbz) from the forward tau^n and p1..p4.
__global__ void __launch_bounds__(A_THREADS, 1)
    el_adj_vel_kernel(const __grid_constant__ ElAdjArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const Geom& g = a.g;
  ATerms& T = *reinterpret_cast<ATerms*>(smem_raw + A_STAGES * sizeof(AVelStage));
  const bool grad = a.gacc != nullptr;
  const int lane = threadIdx.x & 31, r = threadIdx.x >> 5, lx = 4 * lane;
  float acc[2][4], acl[2][4];
  auto issue = [&](AVelStage& sg, uint64_t* b, const AUnit& u) {
    if (!u.valid) {
      mbar_arrive_expect_tx(b, 0);
      return;
    }
    mbar_arrive_expect_tx(b, (grad ? 7 : 4) * kABox);
    const int x = u.x0 - 4, y = u.z0 - 2;
    tma_load_3d(sg.vx, &a.m_avx, b, x, y, u.s);
    tma_load_3d(sg.vz, &a.m_avz, b, x, y, u.s);
    tma_load_2d(sg.cbx, &a.m_cbx, b, x, y);
    tma_load_2d(sg.cbz, &a.m_cbz, b, x, y);
    if (grad) {
      tma_load_3d(sg.txx, &a.m_ftxx, b, x, y, u.s);
      tma_load_3d(sg.tzz, &a.m_ftzz, b, x, y, u.s);
      tma_load_3d(sg.txz, &a.m_ftxz, b, x, y, u.s);
    }
  };
  auto body = [&](const AUnit& u, const AVelStage& sg, auto wait) {
    if (u.first) {
#pragma unroll
      for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[k][c] = acl[k][c] = 0.f;
    }
    const size_t so = (size_t)u.s * g.fstride;
    const bool xs = u.flags & AU_XS, zs = u.flags & AU_ZS;
    const int z = u.z0 + r, x = u.x0 + lx;
    const bool cell = u.valid && z < g.NZ && x < g.NXp;
    const size_t ci = so + (size_t)z * g.NXp + x;
    float txx[4], tzz[4], txz[4];
    v4(ld4z(a.atxx + ci, cell), txx);
    v4(ld4z(a.atzz + ci, cell), tzz);
    v4(ld4z(a.atxz + ci, cell), txz);
    const bool flush = u.last && grad && z < g.NZ && x < g.NXp;
    float* const ga = a.gacc + (size_t)u.grp * 10 * g.fstride + (size_t)z * g.NXp + x;
    if (!wait()) return false;
    const bool plain = u.flags & AU_PLAIN;
    if (u.valid && plain) {
      // (plain unit) one term per velocity component: d0 = d1, d2 = d3
      for (int gi = threadIdx.x; gi < A_H * A_G4; gi += A_THREADS) {
        const int br = gi / A_G4, bc = 4 * (gi - br * A_G4);
        float vx[4], vz[4], cbx[4], cbz[4], d0[4], d2[4];
        v4(lda4(sg.vx, br, bc), vx);
        v4(lda4(sg.vz, br, bc), vz);
        v4(lda4(sg.cbx, br, bc), cbx);
        v4(lda4(sg.cbz, br, bc), cbz);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          d0[k] = cbx[k] * vx[k];
          d2[k] = cbz[k] * vz[k];
        }
        sta4(T.t[0], br, bc, d0);
        sta4(T.t[2], br, bc, d2);
      }
    } else if (u.valid) {
      for (int gi = threadIdx.x; gi < A_H * A_G4; gi += A_THREADS) {
        const int br = gi / A_G4, bc = 4 * (gi - br * A_G4);
        const int zz = u.z0 - 2 + br, xx = u.x0 - 4 + bc;
        const bool zin = zz >= 0 && zz < g.NZ;
        const bool gin = zin && xx >= 0 && xx < g.NXp;
        const size_t c = so + (size_t)zz * g.NXp + xx;
        float vx[4], vz[4], cbx[4], cbz[4];
        v4(lda4(sg.vx, br, bc), vx);
        v4(lda4(sg.vz, br, bc), vz);
        v4(lda4(sg.cbx, br, bc), cbx);
        v4(lda4(sg.cbz, br, bc), cbz);
        XProf px;
        float q1[4], q2[4], q3[4], q4[4];
        x_prof(a, xs ? xx : -4, px);
        v4(ld4z(a.ap_in[0] + c, gin && xs), q1);
        v4(ld4z(a.ap_in[2] + c, gin && xs), q3);
        v4(ld4z(a.ap_in[1] + c, gin && zs), q2);
        v4(ld4z(a.ap_in[3] + c, gin && zs), q4);
        const float A2 = zs && zin ? __ldg(a.az + zz) : 0.f, B2 = zs && zin ? __ldg(a.bz + zz) : 0.f;
        const float A4 = zs && zin ? __ldg(a.azh + zz) : 0.f, B4 = zs && zin ? __ldg(a.bzh + zz) : 0.f;
        float d0[4], d1[4], d2[4], d3[4], n1[4], n2[4], n3[4], n4[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const bool in = zin && xx + k >= 0 && xx + k < g.NX;
          // vx += cbx (dxt + p1' + dzt + p2')
          const float Q = cbx[k] * vx[k];
          const float P1 = q1[k] + Q, P2 = q2[k] + Q;
          d0[k] = in ? Q + px.bh[k] * P1 : 0.f;  // dxt-bar (Dpx txx)
          d1[k] = in ? Q + B2 * P2 : 0.f;        // dzt-bar (Dmz txz)
          n1[k] = px.ah[k] * P1;
          n2[k] = A2 * P2;
          // vz += cbz (dxt + p3' + dzt + p4')
          const float Qz = cbz[k] * vz[k];
          const float P3 = q3[k] + Qz, P4 = q4[k] + Qz;
          d2[k] = in ? Qz + px.b[k] * P3 : 0.f;  // dxt-bar (Dmx txz)
          d3[k] = in ? Qz + B4 * P4 : 0.f;       // dzt-bar (Dpz tzz)
          n3[k] = px.a[k] * P3;
          n4[k] = A4 * P4;
        }
        sta4(T.t[0], br, bc, d0);
        sta4(T.t[1], br, bc, d1);
        sta4(T.t[2], br, bc, d2);
        sta4(T.t[3], br, bc, d3);
        const bool own = gin && br >= 2 && br < 2 + TA_Z && bc >= 4 && bc < 4 + TA_X;
        if (own && xs) {
          st4v(a.ap_out[0] + c, n1);
          st4v(a.ap_out[2] + c, n3);
        }
        if (own && zs) {
          st4v(a.ap_out[1] + c, n2);
          st4v(a.ap_out[3] + c, n4);
        }
      }
    }
    if (u.valid) {
      __syncthreads();
      if (cell) {
        const int R = r + 2;
        {  // tau-bar -= D^T terms
          float d0[12], d2[12];
          row12(T.t[0], R, lx, d0);
          row12(T.t[2], R, lx, d2);
          float a1[4], a0[4], b1[4], b2[4], m2[4], m1[4], c0[4], p1[4];
          const float* t1 = plain ? T.t[0] : T.t[1];
          const float* t3 = plain ? T.t[2] : T.t[3];
          v4(lda4(t1, R - 1, lx + 4), a1);  // d1 rows R-1 .. R+2
          v4(lda4(t1, R, lx + 4), a0);
          v4(lda4(t1, R + 1, lx + 4), b1);
          v4(lda4(t1, R + 2, lx + 4), b2);
          v4(lda4(t3, R - 2, lx + 4), m2);  // d3 rows R-2 .. R+1
          v4(lda4(t3, R - 1, lx + 4), m1);
          v4(lda4(t3, R, lx + 4), c0);
          v4(lda4(t3, R + 1, lx + 4), p1);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            if (x + k >= g.NX) continue;
            txx[k] -= wdm(d0, k);
            txz[k] -= zdp(a1[k], a0[k], b1[k], b2[k]) + wdp(d2, k);
            tzz[k] -= zdm(m2[k], m1[k], c0[k], p1[k]);
          }
          st4v(a.atxx + ci, txx);
          st4v(a.atzz + ci, tzz);
          st4v(a.atxz + ci, txz);
        }
        if (grad) {
          float f1[4], f2[4], f3[4], f4_[4];  // forward p1..p4 (strip units)
          fp_x(a.fp[0] + ci, a.axh, a.bxh, x, xs, f1);
          fp_x(a.fp[2] + ci, a.ax, a.bx, x, xs, f3);
          fp_z(a.fp[1] + ci, a.az, a.bz, z, zs, f2);
          fp_z(a.fp[3] + ci, a.azh, a.bzh, z, zs, f4_);
          float w[12], y[12];
          row12(sg.txx, R, lx, w);
          row12(sg.txz, R, lx, y);
          float tzm1[4], tz0[4], tzp1[4], tzp2[4], xzm2[4], xzm1[4], xzp1[4], avx[4], avz[4];
          v4(lda4(sg.txz, R - 2, lx + 4), xzm2);  // txz rows R-2 .. R+1
          v4(lda4(sg.txz, R - 1, lx + 4), xzm1);
          v4(lda4(sg.txz, R + 1, lx + 4), xzp1);
          v4(lda4(sg.tzz, R - 1, lx + 4), tzm1);  // tzz rows R-1 .. R+2
          v4(lda4(sg.tzz, R, lx + 4), tz0);
          v4(lda4(sg.tzz, R + 1, lx + 4), tzp1);
          v4(lda4(sg.tzz, R + 2, lx + 4), tzp2);
          v4(lda4(sg.vx, R, lx + 4), avx);
          v4(lda4(sg.vz, R, lx + 4), avz);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            if (x + k >= g.NX) continue;
            const float sx = wdp(w, k) + f1[k] + zdm(xzm2[k], xzm1[k], y[4 + k], xzp1[k]) + f2[k];
            const float sz = wdm(y, k) + f3[k] + zdp(tzm1[k], tz0[k], tzp1[k], tzp2[k]) + f4_[k];
            df_add(acc[0][k], acl[0][k], avx[k] * sx);
            df_add(acc[1][k], acl[1][k], avz[k] * sz);
          }
        }
      }
    }
    if (flush) {
      df_flush(ga + 2 * G_BX * g.fstride, g.fstride, acc[0], acl[0]);
      df_flush(ga + 2 * G_BZ * g.fstride, g.fstride, acc[1], acl[1]);
    }
    return true;
  };
  auto ahead = [&](const AUnit& u) {
    const int z = u.z0 + r, x = u.x0 + lx;
    const size_t so = (size_t)u.s * g.fstride;
    const size_t ci = so + (size_t)z * g.NXp + x;
    const bool cell = u.valid && z < g.NZ && x < g.NXp;
    if (u.last && grad && z < g.NZ && x < g.NXp) {
      const float* ga = a.gacc + (size_t)u.grp * 10 * g.fstride + (size_t)z * g.NXp + x;
      df_prefetch(ga + 2 * G_BX * g.fstride, g.fstride);
      df_prefetch(ga + 2 * G_BZ * g.fstride, g.fstride);
    }
    if (cell) {  // the adjoint stresses it updates
      pf_l2(a.atxx + ci);
      pf_l2(a.atzz + ci);
      pf_l2(a.atxz + ci);
    }
    if (u.valid && !(u.flags & AU_PLAIN)) strip_prefetch(a, u, so, ci, cell, grad, 0, 2, 1, 3);
  };
  a_pipeline<AVelStage>(a, smem_raw, issue, body, ahead);
}

// ------------------------------------------------------------ chain rule
__device__ __forceinline__ double mval(const float* model, const Geom& g, int padded, int par,
                                       int z, int x) {
  z = min(max(z, 0), g.NZ - 1);
  x = min(max(x, 0), g.NX - 1);
  if (padded) return model[((size_t)par * g.NZ + z) * g.NX + x];
  const int zi = min(max(z - g.P, 0), g.nz - 1), xi = min(max(x - g.P, 0), g.nx - 1);
  return model[((size_t)par * g.nz + zi) * g.nx + xi];
}
__device__ __forceinline__ double mu_at(const float* model, const Geom& g, int padded, int z,
                                        int x) {
  const double vs = mval(model, g, padded, 1, z, x);
  return mval(model, g, padded, 2, z, x) * vs * vs;
}
// coefficient adjoint k at padded point (z, x), summed over shots and steps:
// the shot groups' compensated sums [ngrp][5][hi, lo][NZ][NXp], in FP64
// and in group order
__device__ __forceinline__ double gsum(const float* gacc, const Geom& g, int ngrp, int k,
                                       int z, int x) {
  double t = 0.0;
  for (int q = 0; q < ngrp; ++q) {
    const float* G = gacc + ((size_t)q * 10 + 2 * k) * g.fstride + (size_t)z * g.NXp + x;
    t += (double)G[0] + (double)G[g.fstride];
  }
  return t;
}

__global__ void el_grad_kernel(const Geom g, const float* gacc, int ngrp, const float* model,
                               int padded, double sc, float* grad, const int* status) {
  if (*status) return;
  const int i = blockIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= g.nx) return;
  const int Z = i + g.P, X = j + g.P;
  const double vp = mval(model, g, padded, 0, Z, X), vs = mval(model, g, padded, 1, Z, X);
  const double rho = mval(model, g, padded, 2, Z, X), mu = rho * vs * vs;
  // lam = rho (vp^2 - 2 vs^2): cl2m = sc (lam + 2 mu), clam = sc lam
  const double gl2m = gsum(gacc, g, ngrp, G_L2M, Z, X);
  const double glam = sc * (gl2m + gsum(gacc, g, ngrp, G_LAM, Z, X));
  double gmu = 2.0 * sc * gl2m;
  double grho = 0.0;
  // cmu at (pz, px) = sc 4 / sum 1/mu over (pz|pz+1) x (px|px+1), clamped
  for (int dz = -1; dz <= 0; ++dz)
    for (int dx = -1; dx <= 0; ++dx) {
      const int pz = Z + dz, px = X + dx;
      if (pz < 0 || px < 0) continue;
      const int pz1 = min(pz + 1, g.NZ - 1), px1 = min(px + 1, g.NX - 1);
      const int cz[4] = {pz, pz, pz1, pz1}, cx[4] = {px, px1, px, px1};
      int mult = 0;
      double inv = 0.0;
      bool zero = false;
      for (int k = 0; k < 4; ++k) {
        const double m = mu_at(model, g, padded, cz[k], cx[k]);
        if (m == 0.0) zero = true;
        else inv += 1.0 / m;
        if (cz[k] == Z && cx[k] == X) ++mult;
      }
      if (mult == 0 || zero) continue;
      const double mxz = 4.0 / inv;
      gmu += mult * sc * gsum(gacc, g, ngrp, G_MU, pz, px) * mxz * mxz / (4.0 * mu * mu);
    }
  // cbx at (Z, px) = sc 2 / (rho(Z, px) + rho(Z, px+1)), cbz likewise in z
  for (int dx = -1; dx <= 0; ++dx) {
    const int px = X + dx;
    if (px < 0) continue;
    const int px1 = min(px + 1, g.NX - 1);
    const int mult = (px == X) + (px1 == X);
    if (!mult) continue;
    const double r2 = mval(model, g, padded, 2, Z, px) + mval(model, g, padded, 2, Z, px1);
    grho += mult * sc * gsum(gacc, g, ngrp, G_BX, Z, px) * (-2.0 / (r2 * r2));
  }
  for (int dz = -1; dz <= 0; ++dz) {
    const int pz = Z + dz;
    if (pz < 0) continue;
    const int pz1 = min(pz + 1, g.NZ - 1);
    const int mult = (pz == Z) + (pz1 == Z);
    if (!mult) continue;
    const double r2 = mval(model, g, padded, 2, pz, X) + mval(model, g, padded, 2, pz1, X);
    grho += mult * sc * gsum(gacc, g, ngrp, G_BZ, pz, X) * (-2.0 / (r2 * r2));
  }
  const size_t M = (size_t)g.nz * g.nx, o = (size_t)i * g.nx + j;
  grad[o] = (float)(glam * 2.0 * rho * vp);
  grad[M + o] = (float)(glam * (-4.0 * rho * vs) + gmu * 2.0 * rho * vs);
  grad[2 * M + o] = (float)(grho + glam * (vp * vp - 2.0 * vs * vs) + gmu * vs * vs);
}

}  // namespace

int el_adj_shot_group(const Geom& g) {
  // units = tiles x groups; halve the group until there are units enough
  // for about twelve per SM of a GB300 (fewer shots per group: more
  // accumulator traffic, one addition per group and step).  Measured on
  // the 500x1500 + 40 gradient with 8 shots (481 tiles): groups of 8 shots
  // 527.6 ms, 4 shots 486.7, 2 shots 480.5, 1 shot 541.4.
  const long long tiles =
      (long long)((g.NZ + TA_Z - 1) / TA_Z) * ((g.NXp + TA_X - 1) / TA_X);
  int sg = std::max(g.nshot, 1);
  while (sg > 1 && tiles * ((g.nshot + sg - 1) / sg) < 1824) sg = (sg + 1) / 2;
  return sg;
}

bool el_adj_maps(ElAdjArgs& a) {
  const Geom& g = a.g;
  const uint64_t S = (uint64_t)(g.nshot > 0 ? g.nshot : 1);
  auto f3 = [&](CUtensorMap* m, const float* base) {
    return make_tensor_map(m, base, 3, g.NX, g.NZ, S, g.NXp, (uint64_t)g.fstride, A_W, A_H, 1);
  };
  auto f2 = [&](CUtensorMap* m, const float* base) {
    return make_tensor_map(m, base, 2, g.NX, g.NZ, 1, g.NXp, (uint64_t)g.fstride, A_W, A_H, 1);
  };
  a.sg = el_adj_shot_group(g);
  a.ngrp = (g.nshot + a.sg - 1) / a.sg;
  a.ntx = (g.NXp + TA_X - 1) / TA_X;
  a.units = a.ntx * ((g.NZ + TA_Z - 1) / TA_Z) * a.ngrp;
  return f3(&a.m_atxx, a.atxx) && f3(&a.m_atzz, a.atzz) && f3(&a.m_atxz, a.atxz) &&
         f3(&a.m_avx, a.avx) && f3(&a.m_avz, a.avz) && f2(&a.m_l2m, a.cl2m) &&
         f2(&a.m_lam, a.clam) && f2(&a.m_mu, a.cmu) && f2(&a.m_cbx, a.cbx) &&
         f2(&a.m_cbz, a.cbz);
}

bool el_adj_forward_maps(ElAdjArgs& a) {
  const Geom& g = a.g;
  const uint64_t S = (uint64_t)(g.nshot > 0 ? g.nshot : 1);
  auto f3 = [&](CUtensorMap* m, const float* base) {
    return make_tensor_map(m, base, 3, g.NX, g.NZ, S, g.NXp, (uint64_t)g.fstride, A_W, A_H, 1);
  };
  return f3(&a.m_fvx, a.fvx) && f3(&a.m_fvz, a.fvz) && f3(&a.m_ftxx, a.ftxx) &&
         f3(&a.m_ftzz, a.ftzz) && f3(&a.m_ftxz, a.ftxz);
}

void launch_el_adj_step(const ElAdjArgs& a, cudaStream_t st) {
  const Geom& g = a.g;
  if (a.units <= 0) return;
  static const bool attr = [] {  // thread-safe one-time initialisation
    cudaFuncSetAttribute(el_adj_str_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kAStrSmem);
    cudaFuncSetAttribute(el_adj_vel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kAVelSmem);
    return true;
  }();
  (void)attr;
  const int grid = std::min(device_sms(), a.units);
  int k = 0;
  if (a.wgrad) {
    launch_dependent(el_adj_src_kernel, dim3((g.nshot + 127) / 128), dim3(128), 0, st, a);
    ++k;
  }
  void* t = profile_begin(SWEEP_K_EL_ADJ, st);
  launch_dependent(el_adj_str_kernel, dim3(grid), dim3(A_THREADS), kAStrSmem, st, a);
  ++k;
  if (a.res && g.nrec > 0) {
    launch_dependent(el_adj_rec_kernel, dim3((g.nrec + 127) / 128, g.nshot), dim3(128), 0, st,
                     a);
    ++k;
  }
  launch_dependent(el_adj_vel_kernel, dim3(grid), dim3(A_THREADS), kAVelSmem, st, a);
  profile_end(t, st);
  note_launches(k + 1);
}

void launch_el_grad(const Geom& g, const float* gacc, int ngrp, const float* model, int padded,
                    float dx, float dt, float* grad, const int* status, cudaStream_t st) {
  const double sc = (double)dt / (double)dx;
  el_grad_kernel<<<dim3((g.nx + 127) / 128, g.nz), 128, 0, st>>>(g, gacc, ngrp, model, padded,
                                                                 sc, grad, status);
  note_launches(1);
}

}  // namespace sweep
