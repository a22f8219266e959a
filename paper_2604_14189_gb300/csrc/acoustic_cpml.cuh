// Device code of the acoustic CPML kernel (the second kernel of a time
// step; acoustic_cpml.cu), shared with the time-loop kernels of
// acoustic_loop.cu.  See acoustic_cpml.cu for the equations and the work
// split.  The part functions are templates on NC: true reads the fields
// through the non-coherent path (__ldg), valid when the fields do not
// change during the kernel (one launch per step); false uses coherent
// loads, for kernels that write the fields in an earlier phase of the
// same launch.  A part function runs on FT consecutive threads (one block
// of the per-step kernel, or one FT-thread slice of a larger block).
#pragma once

#include "acoustic_common.cuh"
#include "tma.cuh"

namespace sweep {
namespace {


// Block size and rows per z-part thread: chosen by a sweep on GB300 (ZCH 4,
// 8, 12 x 128, 256 threads; 301x901+40, 20 shots): forward 8 rows, backward
// 4 rows (its thread keeps three windows), 128 threads.  The minimum blocks
// per SM in the kernels' launch bounds (8 forward, 7 backward) hold them at
// 64 and 72 registers without spills; unbounded, the backward kernel takes
// 80 and one block per SM fewer fits.
constexpr int FT = 128;     // threads per block
constexpr int ZCH_F = ZCH_FWD;  // rows per thread, forward z part
constexpr int ZCH_B = ZCH_BWD;  // rows per thread, backward z part

__device__ __forceinline__ float4 ldg4(const float* p) {
  return __ldg(reinterpret_cast<const float4*>(p));
}
// The 9-point weights of d2 and d1 (acoustic_common.cuh) by offset k - 4.
__host__ __device__ constexpr float kD2w(int k) {
  return k == 4 ? kC0 : (k == 3 || k == 5) ? kC1 : (k == 2 || k == 6) ? kC2
       : (k == 1 || k == 7) ? kC3 : kC4;
}
__host__ __device__ constexpr float kD1w(int k) {
  return k == 4 ? 0.f : k == 5 ? kD1 : k == 6 ? kD2 : k == 7 ? kD3 : k == 8 ? kD4
       : k == 3 ? -kD1 : k == 2 ? -kD2 : k == 1 ? -kD3 : -kD4;
}

// field loads: non-coherent (NC) or coherent
template <bool NC>
__device__ __forceinline__ float ldf(const float* p) {
  if constexpr (NC) return __ldg(p);
  else return *p;
}
template <bool NC>
__device__ __forceinline__ float4 ldf4(const float* p) {
  if constexpr (NC) return __ldg(reinterpret_cast<const float4*>(p));
  else return *reinterpret_cast<const float4*>(p);
}
// this thread's index within its FT-thread slice
__device__ __forceinline__ int ftid() { return threadIdx.x % FT; }
__device__ __forceinline__ float4 ld4(const float* p) {
  return *reinterpret_cast<const float4*>(p);
}
__device__ __forceinline__ void st4(float* p, const float* v) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void red4(float* p, const float* v) {
  atomicAdd(reinterpret_cast<float4*>(p), make_float4(v[0], v[1], v[2], v[3]));
}
// Deterministic mode: only the nonzero terms are added.  An atomic float
// addition flushes a subnormal result to zero, so an added 0.0 would change
// a tiny value of a cell that gets no CPML term (an interior cell of a group
// straddling the border), and a receiver read in the same kernel could see
// the cell before or after it.
__device__ __forceinline__ void red4_nonzero(float* p, const float* v) {
  if (v[0] != 0.f && v[1] != 0.f && v[2] != 0.f && v[3] != 0.f) {
    red4(p, v);
    return;
  }
#pragma unroll
  for (int c = 0; c < 4; ++c)
    if (v[c] != 0.f) atomicAdd(p + c, v[c]);
}

// 12 cells x-4 .. x+7 of a row (zero outside [0, NXp))
template <bool NC>
__device__ __forceinline__ void ldrow12(const float* row, int x, int NXp, float* e) {
  const float4 l = x >= 4 ? ldf4<NC>(row + x - 4) : make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 c = ldf4<NC>(row + x);
  const float4 r = x + 4 < NXp ? ldf4<NC>(row + x + 4) : make_float4(0.f, 0.f, 0.f, 0.f);
  f4a(l, e);
  f4a(c, e + 4);
  f4a(r, e + 8);
}

// Row bands of the backward z part and column bands of the backward x part:
// everything within 4 cells of the border, without overlap.
__host__ __device__ __forceinline__ int band_lo_end(int P, int N) { return min(P + 4, N); }
__host__ __device__ __forceinline__ int band_hi_start(int P, int n, int N) {
  return max(P + n - 4, band_lo_end(P, N));
}

__host__ __device__ __forceinline__ XBands x_bands(int lo_end, int hi_start, int NX) {
  XBands b;
  b.gl = (lo_end + 3) / 4;
  b.gr0 = hi_start / 4;
  if (b.gr0 < b.gl) b.gr0 = b.gl;
  b.ngr = b.gl + (NX + 3) / 4 - b.gr0;
  return b;
}

// Columns of the x part's 4-cell groups.  Deterministic mode (OWN; the
// problem flag SWEEP_F_DETERMINISTIC): each border cell has one owner, the x
// part owning every cell of its columns (in the rows of the z band too,
// where it adds both axes' terms) and the z part the other columns of the z
// band, and the backward stencil kernel injects the residual; so every cell
// receives at most one addition per step, and the results do not depend on
// the order in which blocks run.  Otherwise a corner cell of the border
// takes the z and the x part's additions in either order.
__device__ __forceinline__ bool x_group_col(const AcFixArgs& a, int x) {
  return x < 4 * a.xb.gl || x >= 4 * a.xb.gr0;
}

// Work split: block b of the grid belongs to shot b / bps (bps = blocks per
// shot, one division per block); within a shot the blocks are, in order,
// nbz z-part blocks (row chunk = block / zbx, columns (block % zbx) * FT +
// thread), nbx x-part blocks (a thread per (row, 4-cell column group of the
// two bands), row-major, so that no lane idles when a row has fewer than 32
// groups), nbr receiver blocks and nbs ring blocks.

// ------------------------------------------------------------------ forward
// One forward z-part chunk: rows [zs, ze) of column x, window zs-4 ..
// zs+ZCH+3.  FULL: the window lies inside the grid and the chunk is whole, so
// no row needs a bounds test.
template <bool NC, bool FULL>
__device__ __forceinline__ void fwd_z_chunk(const AcFixArgs& a, size_t so, int x, int zs,
                                            int ze) {
  const Geom& g = a.g;
  constexpr int ZCH = ZCH_F, ZW = ZCH + 8;
  float wu[ZW], wp[ZW], zt[ZCH], kk[ZCH];
#pragma unroll
  for (int k = 0; k < ZW; ++k) {
    const int zz = zs - 4 + k;
    const bool ok = FULL || (zz >= 0 && zz < g.NZ);
    const int o = zz * g.NXp;
    wu[k] = ok ? ldf<NC>(a.u + so + o) : 0.f;
    wp[k] = ok ? ldf<NC>(a.pzin + so + o) : 0.f;
  }
#pragma unroll
  for (int q = 0; q < ZCH; ++q) {
    const bool ok = FULL || zs + q < ze;
    const int o = (zs + q) * g.NXp;
    zt[q] = ok ? a.zzin[so + o] : 0.f;
    kk[q] = ok ? __ldg(a.K + x + o) : 0.f;
  }
  float corr[ZCH];
#pragma unroll
  for (int q = 0; q < ZCH; ++q) {
    const int z = zs + q;
    corr[q] = 0.f;
    if (!FULL && z >= ze) break;
    const float A = __ldg(a.az + z), B = __ldg(a.bz + z);
    const float* w = wu + q;
    const float* p = wp + q;
    const float d2u = d2(w[0], w[1], w[2], w[3], w[4], w[5], w[6], w[7], w[8]);
    const float d1u = d1(w[0], w[1], w[2], w[3], w[5], w[6], w[7], w[8]);
    const float dp = d1(p[0], p[1], p[2], p[3], p[5], p[6], p[7], p[8]);
    const float zn = A * zt[q] + B * (d2u + dp);
    const size_t o = so + z * g.NXp;
    a.pzout[o] = A * p[4] + B * d1u;
    a.zzout[o] = zn;
    corr[q] = kk[q] * (dp + zn);
  }
  // the additions land on the stencil kernel's output: wait for it here,
  // after this thread's loads and arithmetic
  grid_dep_wait();
#pragma unroll
  for (int q = 0; q < ZCH; ++q) {
    if (!FULL && zs + q >= ze) break;
    atomicAdd(a.un + so + (zs + q) * g.NXp, corr[q]);
  }
}

template <bool NC, bool OWN>
__device__ __forceinline__ void fwd_z(const AcFixArgs& a, int s, int bl) {
  const Geom& g = a.g;
  const int ch = bl / a.zbx;
  const int x = (bl - ch * a.zbx) * FT + ftid();
  if (x >= g.NX) return;
  if (OWN && x_group_col(a, x)) return;  // the x part owns those columns
  constexpr int ZCH = ZCH_F;
  const int nch = (g.P + ZCH - 1) / ZCH;  // chunks per strip
  const int strip = ch >= nch ? 1 : 0;
  const int base = strip ? g.P + g.nz : 0;
  const int zs = base + (ch - strip * nch) * ZCH;
  const int ze = min(zs + ZCH, base + g.P);
  const size_t so = (size_t)s * g.fstride + x;  // this column of this shot
  if (ze == zs + ZCH && zs >= 4 && zs + ZCH + 4 <= g.NZ)
    fwd_z_chunk<NC, true>(a, so, x, zs, ze);
  else
    fwd_z_chunk<NC, false>(a, so, x, zs, ze);
}

// Staged forward z chunk (the per-step kernel): the block's 128 columns of
// one chunk, its row windows copied into shared memory by four TMA copies
// (u and psi_z on rows zs-4 .. zs+ZCH+3, zeta_z and K on the chunk's rows;
// rows outside the grid read as zero, as in fwd_z_chunk), then the same
// arithmetic per column.  smem: kZStageF bytes + one mbarrier.
constexpr int ZW_F = ZCH_F + 8;
constexpr uint32_t kZStageF = (2 * ZW_F + 2 * ZCH_F) * FT * 4;

// Issue a z block's copies and wait for them (bounded); false: gave up
// (SWEEP_ETIMEOUT latched, copies drained).  All threads call it.
template <int NCOPY>
__device__ __forceinline__ bool z_stage(const AcFixArgs& a, uint64_t* bar, uint32_t bytes,
                                        float* const (&dst)[NCOPY],
                                        const CUtensorMap* const (&map)[NCOPY],
                                        const int (&y)[NCOPY], int x0, int s) {
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
    mbar_arrive_expect_tx(bar, bytes);
#pragma unroll
    for (int i = 0; i < NCOPY; ++i) {
      if (map[i] == &a.tzK)
        tma_load_2d(dst[i], map[i], bar, x0, y[i]);
      else
        tma_load_3d(dst[i], map[i], bar, x0, y[i], s);
    }
  }
  __syncthreads();  // the barrier is initialised before anyone waits on it
  const bool got = mbar_wait(bar, 0);
  if (__syncthreads_or(!got)) {
    if (threadIdx.x == 0) {
      latch(const_cast<int*>(a.status), SWEEP_ETIMEOUT);
      mbar_wait(bar, 0);  // drain (bounded)
    }
    __syncthreads();
    return false;
  }
  return true;
}

template <bool OWN>
__device__ __forceinline__ void fwd_z_staged(const AcFixArgs& a, int s, int bl,
                                             unsigned char* smem) {
  const Geom& g = a.g;
  const int ch = bl / a.zbx;
  const int x0 = (bl - ch * a.zbx) * FT, t = ftid(), x = x0 + t;
  constexpr int ZCH = ZCH_F, ZW = ZW_F;
  const int nch = (g.P + ZCH - 1) / ZCH;  // chunks per strip
  const int strip = ch >= nch ? 1 : 0;
  const int base = strip ? g.P + g.nz : 0;
  const int zs = base + (ch - strip * nch) * ZCH;
  const int ze = min(zs + ZCH, base + g.P);
  float* su = reinterpret_cast<float*>(smem);
  float* sp = su + ZW * FT;
  float* sz = sp + ZW * FT;
  float* sk = sz + ZCH * FT;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sk + ZCH * FT);
  float* const dst[4] = {su, sp, sz, sk};
  const CUtensorMap* const map[4] = {&a.tzu, &a.tzp, &a.tzz, &a.tzK};
  const int y[4] = {zs - 4, zs - 4, zs, zs};
  if (!z_stage<4>(a, bar, kZStageF, dst, map, y, x0, s)) return;
  if (x >= g.NX || (OWN && x_group_col(a, x))) return;  // (after the block's waits)
  const size_t so = (size_t)s * g.fstride + x;
  float corr[ZCH];
#pragma unroll
  for (int q = 0; q < ZCH; ++q) {
    const int z = zs + q;
    corr[q] = 0.f;
    if (z >= ze) break;
    const float A = __ldg(a.az + z), B = __ldg(a.bz + z);
    float w[9], p[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      w[k] = su[(q + k) * FT + t];
      p[k] = sp[(q + k) * FT + t];
    }
    const float d2u = d2(w[0], w[1], w[2], w[3], w[4], w[5], w[6], w[7], w[8]);
    const float d1u = d1(w[0], w[1], w[2], w[3], w[5], w[6], w[7], w[8]);
    const float dp = d1(p[0], p[1], p[2], p[3], p[5], p[6], p[7], p[8]);
    const float zn = A * sz[q * FT + t] + B * (d2u + dp);
    const size_t o = so + (size_t)z * g.NXp;
    a.pzout[o] = A * p[4] + B * d1u;
    a.zzout[o] = zn;
    corr[q] = sk[q * FT + t] * (dp + zn);
  }
  grid_dep_wait();  // the additions land on the stencil kernel's output
#pragma unroll
  for (int q = 0; q < ZCH; ++q) {
    if (zs + q >= ze) break;
    if (!OWN || corr[q] != 0.f) atomicAdd(a.un + so + (size_t)(zs + q) * g.NXp, corr[q]);
  }
}

template <bool NC, bool OWN>
__device__ __forceinline__ void fwd_x_group(const AcFixArgs& a, int s, int z, int x) {
  const Geom& g = a.g;
  const size_t ro = (size_t)s * g.fstride + z * g.NXp;
  float e[12], f[12], zt[4], kk[4], A[4], B[4];
  ldrow12<NC>(a.u + ro, x, g.NXp, e);
  ldrow12<NC>(a.pxin + ro, x, g.NXp, f);
  f4a(ld4(a.zxin + ro + x), zt);
  f4a(ldg4(a.K + z * g.NXp + x), kk);
  f4a(ldg4(a.ax + x), A);
  f4a(ldg4(a.bx + x), B);
  float po[4], zo[4], du[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const float* w = e + c;
    const float* p = f + c;
    const float d2u = d2(w[0], w[1], w[2], w[3], w[4], w[5], w[6], w[7], w[8]);
    const float d1u = d1(w[0], w[1], w[2], w[3], w[5], w[6], w[7], w[8]);
    const float dp = d1(p[0], p[1], p[2], p[3], p[5], p[6], p[7], p[8]);
    const float zn = A[c] * zt[c] + B[c] * (d2u + dp);
    const bool m = x_border(g, x + c) && x + c < g.NX;
    po[c] = A[c] * p[4] + B[c] * d1u;  // zero off the strip (a = b = psi = 0)
    zo[c] = zn;
    du[c] = m ? kk[c] * (dp + zn) : 0.f;
  }
  st4(a.pxout + ro + x, po);
  st4(a.zxout + ro + x, zo);
  if (OWN && z_border(g, z)) {
    // a row of the z strip: this group also owns its cells' z terms (the
    // z part's arithmetic, as sums streamed over the 9 rows, 4 columns at
    // a time)
    const float Az = __ldg(a.az + z), Bz = __ldg(a.bz + z);
    float d2u[4] = {0.f, 0.f, 0.f, 0.f}, d1u[4] = {0.f, 0.f, 0.f, 0.f};
    float dp[4] = {0.f, 0.f, 0.f, 0.f}, pc[4] = {0.f, 0.f, 0.f, 0.f};
    const size_t so = (size_t)s * g.fstride + x;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const int zz = z - 4 + k;
      if (zz < 0 || zz >= g.NZ) continue;  // zero outside the grid
      float w[4], p[4];
      f4a(ldf4<NC>(a.u + so + (size_t)zz * g.NXp), w);
      f4a(ldf4<NC>(a.pzin + so + (size_t)zz * g.NXp), p);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        d2u[c] += kD2w(k) * w[c];
        d1u[c] += kD1w(k) * w[c];
        dp[c] += kD1w(k) * p[c];
        if (k == 4) pc[c] = p[c];
      }
    }
    float zt4[4], pzo[4], zzo[4];
    f4a(ld4(a.zzin + ro + x), zt4);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float zn = Az * zt4[c] + Bz * (d2u[c] + dp[c]);
      pzo[c] = Az * pc[c] + Bz * d1u[c];
      zzo[c] = zn;
      if (x + c < g.NX) du[c] += kk[c] * (dp[c] + zn);
    }
    st4(a.pzout + ro + x, pzo);
    st4(a.zzout + ro + x, zzo);
  }
  grid_dep_wait();  // the addition lands on the stencil kernel's output
  if constexpr (OWN)
    red4_nonzero(a.un + ro + x, du);
  else
    red4(a.un + ro + x, du);
}

// (row, group) pair t of the x part: row t / ngr, group t % ngr of the two
// bands; false past the last row
__device__ __forceinline__ bool x_pair(const AcFixArgs& a, int bl, int* z, int* x) {
  const int t = bl * FT + ftid();
  const int r = t / a.xb.ngr, j = t - r * a.xb.ngr;
  *z = r;
  *x = 4 * (j < a.xb.gl ? j : a.xb.gr0 + (j - a.xb.gl));
  return r < a.g.NZ;
}

template <bool NC, bool OWN>
__device__ __forceinline__ void fwd_x(const AcFixArgs& a, int s, int bl) {
  int z, x;
  if (x_pair(a, bl, &z, &x)) fwd_x_group<NC, OWN>(a, s, z, x);
}

__device__ __forceinline__ void fwd_rec(const AcFixArgs& a, int s, int bl) {
  const Geom& g = a.g;
  const int r = bl * FT + ftid();
  if (r >= g.nrec) return;
  const long long i = (long long)s * g.nrec + r;
  const int rz = a.rec[2 * i] + g.P, rx = a.rec[2 * i + 1] + g.P;
  a.data[i * g.nt + a.n] = a.un[(size_t)s * g.fstride + (size_t)rz * g.NXp + rx];
}

// Interior coordinates (zi, xi) of ring cell ri.  The ring (w = ringw cells
// around the interior) is stored as the w rows above it and the w rows below
// it, each nx + 2w cells wide, then for every interior row its w cells on
// the left, then for every interior row its w cells on the right.
__device__ __forceinline__ void ring_cell(const Geom& g, int ri, int& zi, int& xi) {
  const int w = g.ringw, W = g.nx + 2 * w;
  if (ri < 2 * w * W) {
    const int r = ri < w * W ? ri : ri - w * W;
    zi = ri < w * W ? r / W - w : g.nz + r / W;
    xi = r % W - w;
  } else if (ri < 2 * w * W + g.nz * w) {
    const int r = ri - 2 * w * W;
    zi = r / w;
    xi = r % w - w;
  } else {
    const int r = ri - 2 * w * W - g.nz * w;
    zi = r / w;
    xi = g.nx + r % w;
  }
}

// boundary save: ring cells 4q .. 4q+3 of u^n (final: the previous step's
// kernels have completed) into the ring slot, in ring order
__device__ __forceinline__ void fwd_ring(const AcFixArgs& a, int s, int bl) {
  const Geom& g = a.g;
  const int q = bl * FT + ftid();
  if (4 * q >= g.nring) return;
  const float* u = a.u + (size_t)s * g.fstride;
  float* sv = a.save + (size_t)s * g.nring;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int ri = 4 * q + j;
    if (ri >= g.nring) break;
    int zi, xi;
    ring_cell(g, ri, zi, xi);
    sv[ri] = u[(size_t)(zi + g.P) * g.NXp + (xi + g.P)];
  }
}


// ----------------------------------------------------------------- backward
// One backward z-part chunk: rows [zs, ze) of column x, window zs-4 .. zs+ZCH+3.
// FULL: the window lies inside the grid and inside one strip and the chunk
// is whole, so no row needs a bounds or strip test.
template <bool NC, bool FULL>
__device__ __forceinline__ void bwd_z_chunk(const AcFixArgs& a, size_t so, int x, int zs,
                                            int ze) {
  const Geom& g = a.g;
  constexpr int ZCH = ZCH_B, ZW = ZCH + 8;
  float wm[ZW], wz[ZW], wp[ZW], kk[ZCH], bb[ZW];
#pragma unroll
  for (int k = 0; k < ZW; ++k) {
    const int zz = zs - 4 + k;
    const bool ok = FULL || (zz >= 0 && zz < g.NZ);
    const int o = zz * g.NXp;
    wm[k] = ok ? ldf<NC>(a.u + so + o) : 0.f;
    wz[k] = ok ? ldf<NC>(a.zzin + so + o) : 0.f;
    wp[k] = ok ? ldf<NC>(a.pzin + so + o) : 0.f;
    bb[k] = ok ? __ldg(a.bz + zz) : 0.f;
  }
#pragma unroll
  for (int q = 0; q < ZCH; ++q) {
    const bool ok = FULL || zs + q < ze;
    kk[q] = ok ? __ldg(a.K + x + (zs + q) * g.NXp) : 0.f;
  }
  float wc[ZW], wb[ZW], wg[ZW];
#pragma unroll
  for (int k = 0; k < ZW; ++k) {
    const int zz = zs - 4 + k;
    wc[k] = bb[k] * (wm[k] + wz[k]);
    wb[k] = bb[k] * wp[k];
    // m G: zero off the strip rows
    wg[k] = (FULL || (zz >= 0 && zz < g.NZ && z_border(g, zz))) ? wm[k] + wc[k] : 0.f;
  }
  float corr[ZCH];
#pragma unroll
  for (int q = 0; q < ZCH; ++q) {
    const int z = zs + q;
    corr[q] = 0.f;
    if (!FULL && z >= ze) break;
    const size_t o = so + z * g.NXp;
    const float* C = wc + q;
    const float* B = wb + q;
    const float* G = wg + q;
    corr[q] = kk[q] * (d2(C[0], C[1], C[2], C[3], C[4], C[5], C[6], C[7], C[8]) -
                       d1(B[0], B[1], B[2], B[3], B[5], B[6], B[7], B[8]));
    if (FULL || z_border(g, z)) {
      const float A = __ldg(a.az + z);
      a.pzout[o] = A * wp[q + 4] - d1(G[0], G[1], G[2], G[3], G[5], G[6], G[7], G[8]);
      a.zzout[o] = A * (wm[q + 4] + wz[q + 4]);
    }
  }
  grid_dep_wait();  // mu^n is the stencil kernel's output
#pragma unroll
  for (int q = 0; q < ZCH; ++q) {
    if (!FULL && zs + q >= ze) break;
    atomicAdd(a.un + so + (zs + q) * g.NXp, corr[q]);
  }
}

template <bool NC, bool OWN>
__device__ __forceinline__ void bwd_z(const AcFixArgs& a, int s, int bl) {
  const Geom& g = a.g;
  const int ch = bl / a.zbx;
  const int x = (bl - ch * a.zbx) * FT + ftid();
  if (x >= g.NX) return;
  if (OWN && x_group_col(a, x)) return;  // the x part owns those columns
  const int lo_end = band_lo_end(g.P, g.NZ), hi_start = band_hi_start(g.P, g.nz, g.NZ);
  constexpr int ZCH = ZCH_B;
  const int nlo = (lo_end + ZCH - 1) / ZCH;
  const int band = ch >= nlo ? 1 : 0;
  const int zs = (band ? hi_start : 0) + (ch - band * nlo) * ZCH;
  const int ze = min(zs + ZCH, band ? g.NZ : lo_end);
  if (zs >= ze) return;
  const size_t so = (size_t)s * g.fstride + x;  // this column of this shot
  const bool full = ze == zs + ZCH && zs >= 4 && zs + ZCH + 4 <= g.NZ &&
                    (zs + ZCH + 4 <= g.P || zs - 4 >= g.P + g.nz);
  if (full)
    bwd_z_chunk<NC, true>(a, so, x, zs, ze);
  else
    bwd_z_chunk<NC, false>(a, so, x, zs, ze);
}

template <bool NC, bool OWN>
__device__ __forceinline__ void bwd_x_group(const AcFixArgs& a, int s, int z, int x) {
  const Geom& g = a.g;
  const size_t ro = (size_t)s * g.fstride + z * g.NXp;
  float em[12], ez[12], ep[12], bb[12], kk[4], A[4];
  ldrow12<NC>(a.u + ro, x, g.NXp, em);
  ldrow12<NC>(a.zxin + ro, x, g.NXp, ez);
  ldrow12<NC>(a.pxin + ro, x, g.NXp, ep);
  ldrow12<true>(a.bx, x, g.NXp, bb);  // profile: constant
  f4a(ldg4(a.K + z * g.NXp + x), kk);
  f4a(ldg4(a.ax + x), A);
  float C[12], Bv[12], G[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const int xx = x - 4 + k;
    C[k] = bb[k] * (em[k] + ez[k]);
    Bv[k] = bb[k] * ep[k];
    G[k] = (xx >= 0 && xx < g.NX && x_border(g, xx)) ? em[k] + C[k] : 0.f;
  }
  float du[4], po[4], zo[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const float* Cc = C + c;
    const float* Bc = Bv + c;
    const float* Gc = G + c;
    const float corr = d2(Cc[0], Cc[1], Cc[2], Cc[3], Cc[4], Cc[5], Cc[6], Cc[7], Cc[8]) -
                       d1(Bc[0], Bc[1], Bc[2], Bc[3], Bc[5], Bc[6], Bc[7], Bc[8]);
    const bool in = x + c < g.NX;
    const bool m = in && x_border(g, x + c);
    du[c] = in ? kk[c] * corr : 0.f;
    po[c] = m ? A[c] * ep[c + 4] - d1(Gc[0], Gc[1], Gc[2], Gc[3], Gc[5], Gc[6], Gc[7], Gc[8])
              : 0.f;
    zo[c] = m ? A[c] * (em[c + 4] + ez[c + 4]) : 0.f;
  }
  st4(a.pxout + ro + x, po);
  st4(a.zxout + ro + x, zo);
  if (OWN && (z < band_lo_end(g.P, g.NZ) || z >= band_hi_start(g.P, g.nz, g.NZ))) {
    // a row of the z band: this group also owns its cells' z terms (the
    // z part's arithmetic, as sums streamed over the 9 rows, 4 columns at
    // a time)
    const bool zb = z_border(g, z);
    float sC[4] = {0.f, 0.f, 0.f, 0.f}, sB[4] = {0.f, 0.f, 0.f, 0.f};
    float sG[4] = {0.f, 0.f, 0.f, 0.f}, mz[4] = {0.f, 0.f, 0.f, 0.f};
    float p4[4] = {0.f, 0.f, 0.f, 0.f};
    const size_t so = (size_t)s * g.fstride + x;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const int zz = z - 4 + k;
      if (zz < 0 || zz >= g.NZ) continue;  // zero outside the grid
      float m[4], zv[4], pv[4];
      const size_t o = so + (size_t)zz * g.NXp;
      f4a(ldf4<NC>(a.u + o), m);
      f4a(ldf4<NC>(a.zzin + o), zv);
      f4a(ldf4<NC>(a.pzin + o), pv);
      const float b = __ldg(a.bz + zz);
      const bool gb = z_border(g, zz);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float Cv = b * (m[c] + zv[c]);
        sC[c] += kD2w(k) * Cv;
        sB[c] += kD1w(k) * (b * pv[c]);
        sG[c] += gb ? kD1w(k) * (m[c] + Cv) : 0.f;
        if (k == 4) {
          mz[c] = m[c] + zv[c];
          p4[c] = pv[c];
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c)
      if (x + c < g.NX) du[c] += kk[c] * (sC[c] - sB[c]);
    if (zb) {
      const float Az = __ldg(a.az + z);
      float pzo[4], zzo[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        pzo[c] = Az * p4[c] - sG[c];
        zzo[c] = Az * mz[c];
      }
      st4(a.pzout + ro + x, pzo);
      st4(a.zzout + ro + x, zzo);
    }
  }
  grid_dep_wait();  // mu^n is the stencil kernel's output
  if constexpr (OWN)
    red4_nonzero(a.un + ro + x, du);
  else
    red4(a.un + ro + x, du);
}

template <bool NC, bool OWN>
__device__ __forceinline__ void bwd_x(const AcFixArgs& a, int s, int bl) {
  int z, x;
  if (x_pair(a, bl, &z, &x)) bwd_x_group<NC, OWN>(a, s, z, x);
}


// residual injection mu^n(r) += K(r) res^{n-1}(r) (outside deterministic
// mode; there the stencil kernel injects it)
__device__ __forceinline__ void bwd_rec(const AcFixArgs& a, int s, int bl) {
  const Geom& g = a.g;
  const int r = bl * FT + ftid();
  if (r >= g.nrec) return;
  const long long i = (long long)s * g.nrec + r;
  const int rz = a.rec[2 * i] + g.P, rx = a.rec[2 * i + 1] + g.P;
  const size_t c = (size_t)rz * g.NXp + rx;
  atomicAdd(a.un + (size_t)s * g.fstride + c, a.K[c] * a.res[i * g.nt + (a.n - 1)]);
}

// ring restore: u^{n-1} on the ring cells 4q .. 4q+3 from the forward save
// (the stencil kernel reconstructs the interior and leaves the ring alone)
__device__ __forceinline__ void bwd_ring(const AcFixArgs& a, int s, int bl) {
  const Geom& g = a.g;
  const int q = bl * FT + ftid();
  if (4 * q >= g.nring) return;
  float* u = a.uring + (size_t)s * g.fstride;
  const float* sv = a.save + (size_t)s * g.nring;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int ri = 4 * q + j;
    if (ri >= g.nring) break;
    int zi, xi;
    ring_cell(g, ri, zi, xi);
    u[(size_t)(zi + g.P) * g.NXp + (xi + g.P)] = sv[ri];
  }
}


int cdiv(int a, int b) { return (a + b - 1) / b; }

}  // namespace
}  // namespace sweep
