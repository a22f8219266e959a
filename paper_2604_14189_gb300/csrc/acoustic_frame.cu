// Frame acoustic step kernels: every cell outside the interior kernels'
// rectangles (the absorbing border, plus the interior cells next to it),
// with the full convolutional-PML update, ring save/restore, and source and
// receiver handling.  See acoustic_common.cuh for the equations.
//
// Work is a list of (frame tile, shot) units, FR_TZ x FR_TX tiles laid over
// the (up to four) frame rectangles; persistent CTAs take units round-robin
// and run a multi-stage TMA pipeline: every field a unit needs (wavefield
// with halo, PML memory variables with the halo along their own axis, centre
// values) lands in one shared-memory stage, several units ahead of the one
// being computed.  Loads are skipped per unit when a tile has no x or z
// border cells.  Each thread owns one column of the tile, so warps read
// consecutive shared-memory words and the z stencils run on register
// windows.  The backward kernel first forms G = (1 + b) mu + b zetabar per
// axis in shared memory.
#include "acoustic_common.cuh"
#include "tma.cuh"

namespace sweep {
namespace {

constexpr int FW = FR_HW;
constexpr int FH = FR_HH;
constexpr int CEN = FR_TZ * FR_TX;
constexpr int FR_ROWS = FR_TZ * FR_TX / FR_THREADS;  // rows per thread
static_assert(FR_THREADS % FR_TX == 0 && FR_ROWS * (FR_THREADS / FR_TX) == FR_TZ, "mapping");
constexpr int WIN = FR_ROWS + 8;  // z window

constexpr uint32_t B_HALO = FH * FW * 4;      // 6912
constexpr uint32_t B_CEN = CEN * 4;           // 4096
constexpr uint32_t B_XH = FR_TZ * FW * 4;     // 4608
constexpr uint32_t B_ZH = FH * FR_TX * 4;     // 6144
static_assert(B_HALO % 128 == 0 && B_CEN % 128 == 0 && B_XH % 128 == 0 && B_ZH % 128 == 0,
              "stage alignment");

__device__ __forceinline__ void frame_tile(const FrameRects& fr, int t, int& z0, int& x0,
                                           int& z1, int& x1) {
  int r = 0;
  while (r + 1 < fr.n && t >= fr.first[r + 1]) ++r;
  const int lt = t - fr.first[r];
  const int tz = lt / fr.ntx[r], tx = lt - tz * fr.ntx[r];
  z0 = fr.z0[r] + tz * FR_TZ;
  x0 = fr.x0[r] + tx * FR_TX;
  z1 = min(z0 + FR_TZ, fr.z1[r]);
  x1 = min(x0 + FR_TX, fr.x1[r]);
}

__device__ __forceinline__ bool has_xborder(const Geom& g, int xa, int xb) {
  return (xa < g.P && xb > 0) || (xb > g.P + g.nx && xa < g.NX);
}
__device__ __forceinline__ bool has_zborder(const Geom& g, int za, int zb) {
  return (za < g.P && zb > 0) || (zb > g.P + g.nz && za < g.NZ);
}
__device__ __forceinline__ bool touches_interior(const Geom& g, int z0, int z1, int x0,
                                                 int x1) {
  return z1 > g.P && z0 < g.P + g.nz && x1 > g.P && x0 < g.P + g.nx;
}

struct FrUnit {
  int s, z0, x0, z1, x1;
};
__device__ __forceinline__ FrUnit fr_unit(const FrameRects& fr, int S, int unit) {
  FrUnit u;
  const int t = unit / S;
  u.s = unit - t * S;
  frame_tile(fr, t, u.z0, u.x0, u.z1, u.x1);
  return u;
}

// ------------------------------------------------------------------ forward
struct __align__(128) FrFwdStage {
  float u[FH * FW];       // u^n, halo
  float up[CEN];          // u^{n-1}
  float k[CEN];           // K
  float px[FR_TZ * FW];   // psi_x^{n-1}, x halo
  float pz[FH * FR_TX];   // psi_z^{n-1}, z halo
  float zx[CEN];          // zeta_x
  float zz[CEN];          // zeta_z
};
constexpr int FR_FWD_STAGES = 6;
constexpr size_t kFrFwdSmem = FR_FWD_STAGES * sizeof(FrFwdStage) + 8 * FR_FWD_STAGES;

__global__ void __launch_bounds__(FR_THREADS, 1)
    ac_fr_fwd_kernel(const __grid_constant__ AcFrFwdArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ ShotTable T;
  __shared__ BorderProfiles BP;
  FrFwdStage* stg = reinterpret_cast<FrFwdStage*>(smem_raw);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + FR_FWD_STAGES * sizeof(FrFwdStage));
  constexpr int D = FR_FWD_STAGES;
  if (*a.status) return;
  const Geom& g = a.g;
  const int S = g.nshot;
  const int G = gridDim.x;
  const int count = (a.units - (int)blockIdx.x + G - 1) / G;  // units b, b+G, ...
  if (count <= 0) return;
  load_shot_table(T, g, a.src, a.wavelet, a.rbox, a.n);
  load_profiles(BP, g, a.ax, a.bx, a.az, a.bz);
  if (threadIdx.x == 0) {
    for (int i = 0; i < D; ++i) mbar_init(&bar[i], 1);
    fence_barrier_init();
  }
  __syncthreads();
  auto issue = [&](int k) {
    const FrUnit u = fr_unit(a.fr, S, blockIdx.x + k * G);
    const bool hx = has_xborder(g, u.x0, u.x0 + FR_TX);
    const bool hz = has_zborder(g, u.z0, u.z0 + FR_TZ);
    FrFwdStage& sg = stg[k % D];
    uint64_t* b = &bar[k % D];
    mbar_arrive_expect_tx(b, B_HALO + 2 * B_CEN + (hx ? B_XH + B_CEN : 0) +
                                 (hz ? B_ZH + B_CEN : 0));
    tma_load_3d(sg.u, &a.tu, b, u.x0 - 4, u.z0 - 4, u.s);
    tma_load_3d(sg.up, &a.tup, b, u.x0, u.z0, u.s);
    tma_load_2d(sg.k, &a.tK, b, u.x0, u.z0);
    if (hx) {
      tma_load_3d(sg.px, &a.tpx, b, u.x0 - 4, u.z0, u.s);
      tma_load_3d(sg.zx, &a.tzx, b, u.x0, u.z0, u.s);
    }
    if (hz) {
      tma_load_3d(sg.pz, &a.tpz, b, u.x0, u.z0 - 4, u.s);
      tma_load_3d(sg.zz, &a.tzz, b, u.x0, u.z0, u.s);
    }
  };
  if (threadIdx.x == 0)
    for (int k = 0; k < D && k < count; ++k) issue(k);
  const int c = threadIdx.x % FR_TX, r0 = (threadIdx.x / FR_TX) * FR_ROWS;
  int k = 0;
  for (; k < count; ++k) {
    const FrUnit u = fr_unit(a.fr, S, blockIdx.x + k * G);
    const bool got = mbar_wait(&bar[k % D], (k / D) & 1);
    if (__syncthreads_or(!got)) break;
    const ShotInfo si = shot_info(T, g, a.src, a.wavelet, a.rbox, a.n, u.s);
    const int sz = si.sz, sx = si.sx;
    const float fn = si.fn;
    const FrFwdStage& sg = stg[k % D];
    const bool hz = has_zborder(g, u.z0, u.z0 + FR_TZ);
    const long long so = (long long)u.s * g.fstride;
    const int x = u.x0 + c;
    const bool xb = x < u.x1 && x_border(g, x);
    const float2 abx = xb ? prof_x(BP, g, a.ax, a.bx, x) : make_float2(0.f, 0.f);
    const float Ax = abx.x, Bx = abx.y;
    float wu[WIN], wp[WIN];
#pragma unroll
    for (int j = 0; j < WIN; ++j) {
      wu[j] = sg.u[(r0 + j) * FW + c + 4];
      wp[j] = hz ? sg.pz[(r0 + j) * FR_TX + c] : 0.f;
    }
#pragma unroll
    for (int q = 0; q < FR_ROWS; ++q) {
      const int r = r0 + q, gz = u.z0 + r;
      if (gz >= u.z1 || x >= u.x1) continue;
      const float* row = sg.u + (r + 4) * FW + (c + 4);
      const float* w = wu + q;
      float lapx = d2(row[-4], row[-3], row[-2], row[-1], w[4], row[1], row[2], row[3], row[4]);
      float lapz = d2(w[0], w[1], w[2], w[3], w[4], w[5], w[6], w[7], w[8]);
      const long long ci = so + (long long)gz * g.NXp + x;
      if (xb) {
        const float* pr = sg.px + r * FW + (c + 4);
        const float dp = d1(pr[-4], pr[-3], pr[-2], pr[-1], pr[1], pr[2], pr[3], pr[4]);
        const float du = d1(row[-4], row[-3], row[-2], row[-1], row[1], row[2], row[3], row[4]);
        const float W = lapx + dp;
        const float zn = Ax * sg.zx[r * FR_TX + c] + Bx * W;
        a.psx_out[ci] = Ax * pr[0] + Bx * du;
        a.zex[ci] = zn;
        lapx = W + zn;
      }
      if (hz && z_border(g, gz)) {
        const float* p = wp + q;
        const float dp = d1(p[0], p[1], p[2], p[3], p[5], p[6], p[7], p[8]);
        const float du = d1(w[0], w[1], w[2], w[3], w[5], w[6], w[7], w[8]);
        const float2 abz = prof_z(BP, g, a.az, a.bz, gz);
        const float A = abz.x, B = abz.y;
        const float W = lapz + dp;
        const float zn = A * sg.zz[r * FR_TX + c] + B * W;
        a.psz_out[ci] = A * p[4] + B * du;
        a.zez[ci] = zn;
        lapz = W + zn;
      }
      const float kk = sg.k[r * FR_TX + c];
      float v = 2.f * w[4] - sg.up[r * FR_TX + c] + kk * (lapx + lapz);
      if (gz == sz && x == sx) v += kk * fn;
      a.un[ci] = v;
      if (a.save) {
        const int ri = ring_index(g, gz, x);
        if (ri >= 0) a.save[(long long)u.s * g.nring + ri] = v;
      }
    }
    __syncthreads();  // stage released; this unit's stores visible to the CTA
    if (threadIdx.x == 0 && k + D < count) {
      fence_proxy_async_smem();
      issue(k + D);
    }
    if (a.data && tile_meets(si.box, u.z0, FR_TZ, u.x0, FR_TX)) {
      const long long so2 = (long long)u.s * g.fstride;
      for (int rr = threadIdx.x; rr < g.nrec; rr += FR_THREADS) {
        const int32_t* q = a.rec + 2 * ((long long)u.s * g.nrec + rr);
        const int rz = q[0] + g.P, rx = q[1] + g.P;
        if (rz >= u.z0 && rz < u.z1 && rx >= u.x0 && rx < u.x1)
          a.data[((long long)u.s * g.nrec + rr) * g.nt + a.n] =
              a.un[so2 + (long long)rz * g.NXp + rx];
      }
    }
  }
  if (k < count && threadIdx.x == 0) {
    latch(a.status, SWEEP_ETIMEOUT);
    for (int j = k; j < count && j < k + D; ++j) mbar_wait(&bar[j % D], (j / D) & 1);
  }
}

// ----------------------------------------------------------------- backward
struct __align__(128) FrBwdStage {
  float m[FH * FW];        // mu^{n+1}, halo
  float u[FH * FW];        // u^n, halo
  float k[CEN];            // K
  float m2[CEN];           // mu^{n+2}
  float u1[CEN];           // u^{n+1}
  float gr[CEN];           // imaging accumulator
  float il[CEN];           // illumination accumulator
  float zbx[FR_TZ * FW];   // zetabar_x, x halo
  float pbx[FR_TZ * FW];   // psibar_x, x halo
  float zbz[FH * FR_TX];   // zetabar_z, z halo
  float pbz[FH * FR_TX];   // psibar_z, z halo
};
struct FrBwdWork {
  float gx[FR_TZ * FW];    // G_x on the tile rows with the x halo
  float bpx[FR_TZ * FW];   // b_x psibar_x
  float mgx[FR_TZ * FW];   // G_x masked to the x border
  float gz[FH * FR_TX];    // G_z on the tile columns with the z halo
  float bpz[FH * FR_TX];   // b_z psibar_z
  float mgz[FH * FR_TX];   // G_z masked to the z border
  float bxs[FW];
  float bzs[FH];
};
constexpr int FR_BWD_STAGES = 3;
constexpr size_t kFrBwdSmem =
    FR_BWD_STAGES * sizeof(FrBwdStage) + sizeof(FrBwdWork) + 8 * FR_BWD_STAGES;

__global__ void __launch_bounds__(FR_THREADS, 1)
    ac_fr_bwd_kernel(const __grid_constant__ AcFrBwdArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ ShotTable T;
  __shared__ BorderProfiles BP;
  constexpr int D = FR_BWD_STAGES;
  FrBwdStage* stg = reinterpret_cast<FrBwdStage*>(smem_raw);
  FrBwdWork& W = *reinterpret_cast<FrBwdWork*>(smem_raw + D * sizeof(FrBwdStage));
  uint64_t* bar =
      reinterpret_cast<uint64_t*>(smem_raw + D * sizeof(FrBwdStage) + sizeof(FrBwdWork));
  if (*a.status) return;
  const Geom& g = a.g;
  const int S = g.nshot;
  const int G = gridDim.x;
  const int count = (a.units - (int)blockIdx.x + G - 1) / G;
  if (count <= 0) return;
  const bool adj = a.do_adj != 0, rec = a.do_rec != 0;
  load_shot_table(T, g, a.src, a.do_img ? a.wavelet : nullptr, a.rbox, a.n);
  load_profiles(BP, g, a.ax, a.bx, a.az, a.bz);
  if (threadIdx.x == 0) {
    for (int i = 0; i < D; ++i) mbar_init(&bar[i], 1);
    fence_barrier_init();
  }
  __syncthreads();
  auto issue = [&](int k) {
    const FrUnit u = fr_unit(a.fr, S, blockIdx.x + k * G);
    const bool img = a.do_img && touches_interior(g, u.z0, u.z1, u.x0, u.x1);
    const bool hx = adj && has_xborder(g, u.x0 - 4, u.x0 + FR_TX + 4);
    const bool hz = adj && has_zborder(g, u.z0 - 4, u.z0 + FR_TZ + 4);
    FrBwdStage& sg = stg[k % D];
    uint64_t* b = &bar[k % D];
    const uint32_t bytes = B_HALO + B_CEN + (adj ? B_CEN : 0) +
                           (img ? B_HALO + B_CEN + (a.illum ? B_CEN : 0) + (rec ? B_CEN : 0) : 0) +
                           (hx ? 2 * B_XH : 0) + (hz ? 2 * B_ZH : 0);
    mbar_arrive_expect_tx(b, bytes);
    tma_load_3d(sg.m, &a.tmA, b, u.x0 - 4, u.z0 - 4, u.s);
    tma_load_2d(sg.k, &a.tK, b, u.x0, u.z0);
    if (adj) tma_load_3d(sg.m2, &a.tmB, b, u.x0, u.z0, u.s);
    if (img) {
      tma_load_3d(sg.u, &a.tuA, b, u.x0 - 4, u.z0 - 4, u.s);
      tma_load_3d(sg.gr, &a.tG, b, u.x0, u.z0, u.s);
      if (a.illum) tma_load_3d(sg.il, &a.tI, b, u.x0, u.z0, u.s);
      if (rec) tma_load_3d(sg.u1, &a.tuB, b, u.x0, u.z0, u.s);
    }
    if (hx) {
      tma_load_3d(sg.zbx, &a.tzbx, b, u.x0 - 4, u.z0, u.s);
      tma_load_3d(sg.pbx, &a.tpbx, b, u.x0 - 4, u.z0, u.s);
    }
    if (hz) {
      tma_load_3d(sg.zbz, &a.tzbz, b, u.x0, u.z0 - 4, u.s);
      tma_load_3d(sg.pbz, &a.tpbz, b, u.x0, u.z0 - 4, u.s);
    }
  };
  if (threadIdx.x == 0)
    for (int k = 0; k < D && k < count; ++k) issue(k);
  const int c = threadIdx.x % FR_TX, r0 = (threadIdx.x / FR_TX) * FR_ROWS;
  int k = 0;
  for (; k < count; ++k) {
    const FrUnit u = fr_unit(a.fr, S, blockIdx.x + k * G);
    const bool img = a.do_img && touches_interior(g, u.z0, u.z1, u.x0, u.x1);
    const bool hx = adj && has_xborder(g, u.x0 - 4, u.x0 + FR_TX + 4);
    const bool hz = adj && has_zborder(g, u.z0 - 4, u.z0 + FR_TZ + 4);
    // border profiles of this tile (with halo)
    for (int j = threadIdx.x; j < FW; j += FR_THREADS) {
      const int xx = u.x0 - 4 + j;
      W.bxs[j] = (xx >= 0 && xx < g.NX && x_border(g, xx)) ? prof_x(BP, g, a.ax, a.bx, xx).y
                                                            : 0.f;
    }
    for (int i = threadIdx.x; i < FH; i += FR_THREADS) {
      const int zz = u.z0 - 4 + i;
      W.bzs[i] = (zz >= 0 && zz < g.NZ && z_border(g, zz)) ? prof_z(BP, g, a.az, a.bz, zz).y
                                                            : 0.f;
    }
    const bool got = mbar_wait(&bar[k % D], (k / D) & 1);
    if (__syncthreads_or(!got)) break;
    const ShotInfo si = shot_info(T, g, a.src, a.do_img ? a.wavelet : nullptr, a.rbox, a.n, u.s);
    const int sz = si.sz, sx = si.sx;
    const float fn = img ? si.fn : 0.f;
    const FrBwdStage& sg = stg[k % D];
    const long long so = (long long)u.s * g.fstride;
    if (adj && (hx || hz)) {
      // per-axis adjoint combinations on the tile with halo (zetabar out on
      // the way): each thread fills its own column and rows, edge threads
      // also the halo columns / rows
      if (hx) {
        auto buildx = [&](int j) {
          const int xx = u.x0 - 4 + j;
          const bool bord = xx >= 0 && xx < g.NX && x_border(g, xx);
          const bool out = bord && j >= 4 && xx < u.x1;
          const float b = W.bxs[j];
          const float A = out ? prof_x(BP, g, a.ax, a.bx, xx).x : 0.f;
#pragma unroll
          for (int q = 0; q < FR_ROWS; ++q) {
            const int r = r0 + q, idx = r * FW + j;
            const float m1 = sg.m[(r + 4) * FW + j], zb = sg.zbx[idx];
            const float Gv = m1 + b * (m1 + zb);
            W.gx[idx] = Gv;
            W.bpx[idx] = b * sg.pbx[idx];
            W.mgx[idx] = bord ? Gv : 0.f;
            if (out && u.z0 + r < u.z1)
              a.zbx_out[so + (long long)(u.z0 + r) * g.NXp + xx] = A * (m1 + zb);
          }
        };
        buildx(c + 4);
        if (c < 4) buildx(c);
        else if (c >= FR_TX - 4) buildx(c + 8);
      }
      if (hz) {
        const int xx = u.x0 + c;
        auto buildz = [&](int i) {
          const int zz = u.z0 - 4 + i;
          const bool bord = zz >= 0 && zz < g.NZ && z_border(g, zz);
          const int idx = i * FR_TX + c;
          const float b = W.bzs[i];
          const float m1 = sg.m[i * FW + c + 4], zb = sg.zbz[idx];
          const float Gv = m1 + b * (m1 + zb);
          W.gz[idx] = Gv;
          W.bpz[idx] = b * sg.pbz[idx];
          W.mgz[idx] = bord ? Gv : 0.f;
          if (bord && i >= 4 && i < 4 + FR_TZ && zz < u.z1 && xx < u.x1)
            a.zbz_out[so + (long long)zz * g.NXp + xx] =
                prof_z(BP, g, a.az, a.bz, zz).x * (m1 + zb);
        };
#pragma unroll
        for (int q = 0; q < FR_ROWS; ++q) buildz(r0 + 4 + q);
        if (r0 == 0) {
#pragma unroll
          for (int q = 0; q < 4; ++q) buildz(q);
        }
        if (r0 == FR_TZ - FR_ROWS) {
#pragma unroll
          for (int q = 0; q < 4; ++q) buildz(FR_TZ + 4 + q);
        }
      }
      __syncthreads();
    }
    // G_x is mu^{n+1} itself when the tile and its halo have no x border
    const float* GX = hx ? W.gx : sg.m + 4 * FW;
    const int x = u.x0 + c;
    const bool xb = x < u.x1 && x_border(g, x);
    const float Ax = xb ? prof_x(BP, g, a.ax, a.bx, x).x : 0.f;
    // does this tile hold ring cells to restore?
    const int rw = g.ringw;
    const bool ring_tile = rec && a.save && rw > 0 && u.z0 < g.P + g.nz + rw &&
                           u.z1 > g.P - rw && u.x0 < g.P + g.nx + rw && u.x1 > g.P - rw;
    float wg[WIN], wbp[WIN], wmg[WIN];
    if (adj) {
#pragma unroll
      for (int j = 0; j < WIN; ++j) {
        const int i = (r0 + j) * FR_TX + c;
        wg[j] = hz ? W.gz[i] : sg.m[(r0 + j) * FW + c + 4];
        wbp[j] = hz ? W.bpz[i] : 0.f;
        wmg[j] = hz ? W.mgz[i] : 0.f;
      }
    }
#pragma unroll
    for (int q = 0; q < FR_ROWS; ++q) {
      const int r = r0 + q, gz = u.z0 + r;
      if (gz >= u.z1 || x >= u.x1) continue;
      const long long ci = so + (long long)gz * g.NXp + x;
      const int cc = r * FR_TX + c;
      const float m1 = sg.m[(r + 4) * FW + c + 4];
      const float kk = sg.k[cc];
      if (adj) {
        const float* G1 = GX + r * FW + c + 4;
        const float* G2 = wg + q;
        float acc = d2(G1[-4], G1[-3], G1[-2], G1[-1], G1[0], G1[1], G1[2], G1[3], G1[4]) +
                    d2(G2[0], G2[1], G2[2], G2[3], G2[4], G2[5], G2[6], G2[7], G2[8]);
        if (hx) {
          const float* B1 = W.bpx + r * FW + c + 4;
          acc -= d1(B1[-4], B1[-3], B1[-2], B1[-1], B1[1], B1[2], B1[3], B1[4]);
          if (xb) {
            const float* M1 = W.mgx + r * FW + c + 4;
            a.pbx_out[ci] = Ax * sg.pbx[r * FW + c + 4] -
                            d1(M1[-4], M1[-3], M1[-2], M1[-1], M1[1], M1[2], M1[3], M1[4]);
          }
        }
        if (hz) {
          const float* Wb = wbp + q;
          acc -= d1(Wb[0], Wb[1], Wb[2], Wb[3], Wb[5], Wb[6], Wb[7], Wb[8]);
          if (z_border(g, gz)) {
            const float* M = wmg + q;
            a.pbz_out[ci] = prof_z(BP, g, a.az, a.bz, gz).x * sg.pbz[(r + 4) * FR_TX + c] -
                            d1(M[0], M[1], M[2], M[3], M[5], M[6], M[7], M[8]);
          }
        }
        a.mB[ci] = 2.f * m1 - sg.m2[cc] + kk * acc;
      }
      if (img && interior(g, gz, x)) {
        const float* row = sg.u + (r + 4) * FW + (c + 4);
        float lap = d2(row[-4], row[-3], row[-2], row[-1], row[0], row[1], row[2], row[3],
                       row[4]) +
                    d2(row[-4 * FW], row[-3 * FW], row[-2 * FW], row[-FW], row[0], row[FW],
                       row[2 * FW], row[3 * FW], row[4 * FW]);
        if (gz == sz && x == sx) lap += fn;
        a.graw[ci] = sg.gr[cc] + m1 * lap;
        if (a.illum) a.illum[ci] = sg.il[cc] + row[0] * row[0];
        if (rec) a.uB[ci] = 2.f * row[0] - sg.u1[cc] + kk * lap;
      } else if (ring_tile) {
        const int ri = ring_index(g, gz, x);
        if (ri >= 0) a.uB[ci] = a.save[(long long)u.s * g.nring + ri];
      }
    }
    if (a.wgrad && a.n < g.nt && threadIdx.x == 0 && sz >= u.z0 && sz < u.z1 && sx >= u.x0 &&
        sx < u.x1)
      a.wgrad[(long long)u.s * g.nt + a.n] = sg.m[(sz - u.z0 + 4) * FW + (sx - u.x0 + 4)];
    __syncthreads();  // stage and G arrays released; mu^n stores visible
    if (threadIdx.x == 0 && k + D < count) {
      fence_proxy_async_smem();
      issue(k + D);
    }
    if (adj && a.n >= 1 && tile_meets(si.box, u.z0, FR_TZ, u.x0, FR_TX)) {
      for (int rr = threadIdx.x; rr < g.nrec; rr += FR_THREADS) {
        const int32_t* q = a.rec + 2 * ((long long)u.s * g.nrec + rr);
        const int rz = q[0] + g.P, rx = q[1] + g.P;
        if (rz >= u.z0 && rz < u.z1 && rx >= u.x0 && rx < u.x1) {
          const float rv = a.res[((long long)u.s * g.nrec + rr) * g.nt + (a.n - 1)];
          atomicAdd(a.mB + so + (long long)rz * g.NXp + rx,
                    a.K[(long long)rz * g.NXp + rx] * rv);
        }
      }
    }
  }
  if (k < count && threadIdx.x == 0) {
    latch(a.status, SWEEP_ETIMEOUT);
    for (int j = k; j < count && j < k + D; ++j) mbar_wait(&bar[j % D], (j / D) & 1);
  }
}

}  // namespace

FrameRects frame_rects(const Geom& g, const Region& in) {
  FrameRects fr{};
  auto add = [&](int z0, int z1, int x0, int x1) {
    if (z1 <= z0 || x1 <= x0) return;
    const int k = fr.n++;
    fr.z0[k] = z0;
    fr.z1[k] = z1;
    fr.x0[k] = x0;
    fr.x1[k] = x1;
    fr.ntx[k] = (x1 - x0 + FR_TX - 1) / FR_TX;
    const int ntz = (z1 - z0 + FR_TZ - 1) / FR_TZ;
    fr.first[k + 1] = fr.first[k] + ntz * fr.ntx[k];
  };
  if (in.z1 <= in.z0 || in.x1 <= in.x0) {
    add(0, g.NZ, 0, g.NX);
  } else {
    add(0, in.z0, 0, g.NX);
    add(in.z1, g.NZ, 0, g.NX);
    add(in.z0, in.z1, 0, in.x0);
    add(in.z0, in.z1, in.x1, g.NX);
  }
  return fr;
}

void launch_ac_fr_fwd(const AcFrFwdArgs& a, cudaStream_t st) {
  if (a.units <= 0) return;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(ac_fr_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kFrFwdSmem);
    attr = true;
  }
  int grid = device_sms();
  if (grid > a.units) grid = a.units;
  void* tok = profile_begin(SWEEP_K_AC_FWD_FR, st);
  ac_fr_fwd_kernel<<<grid, FR_THREADS, kFrFwdSmem, st>>>(a);
  profile_end(tok, st);
  note_launches(1);
}

void launch_ac_fr_bwd(const AcFrBwdArgs& a, cudaStream_t st) {
  if (a.units <= 0) return;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(ac_fr_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kFrBwdSmem);
    attr = true;
  }
  int grid = device_sms();
  if (grid > a.units) grid = a.units;
  void* tok = profile_begin(SWEEP_K_AC_BWD_FR, st);
  ac_fr_bwd_kernel<<<grid, FR_THREADS, kFrBwdSmem, st>>>(a);
  profile_end(tok, st);
  note_launches(1);
}

}  // namespace sweep
