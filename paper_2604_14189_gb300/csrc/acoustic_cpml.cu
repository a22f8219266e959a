// CPML correction kernels of the acoustic step.
//
// The plain-stencil kernels (acoustic_interior.cu) update every cell of the
// padded grid as if there were no absorbing layer.  The convolutional-PML
// terms are additive per axis, so each axis is corrected afterwards by a
// kernel that visits only the cells its terms reach (see
// acoustic_common.cuh for the full update):
//
// forward, axis strip cells (sigma != 0 along that axis):
//   W = D2 u^n + D1 psi^{n-1};  zeta^n = a zeta^{n-1} + b W;
//   psi^n = a psi^{n-1} + b D1 u^n;  u^{n+1} += K (D1 psi^{n-1} + zeta^n)
// backward, strip cells and the 4 cells next to them:
//   C = b (mu^{n+1} + zetabar^n),  B = b psibar^n   (zero off the strip)
//   mu^n += K (D2 C - D1 B)
//   strip cells: psibar^{n-1} = a psibar^n - D1 (m (mu^{n+1} + C)),
//                zetabar^{n-1} = a (mu^{n+1} + zetabar^n)
//
// The profiles a, b are zero off the border, and so are psi, zeta and their
// adjoints (never written there), which removes most masks.
//
// z kernels: a thread owns 2 adjacent columns (8-byte accesses, coalesced
// across the warp) and a chunk of ZCH rows; x kernels: a thread owns 4
// consecutive cells of a row (16-byte accesses) and reads its 4 + 4
// x-neighbours as two more 16-byte loads.  Every load of a thread is issued
// before its arithmetic, so the memory latency is paid once per thread.
// The forward kernels also save the ring cells of their strips after the
// final update (z kernel: ring cells outside the x strips; x kernel: ring
// cells inside them, the x kernel runs last).
#include "acoustic_common.cuh"

namespace sweep {
namespace {

constexpr int ZT = 128;  // threads per block, z kernels (256 columns)
constexpr int ZCH = 8;   // rows per thread, z kernels
constexpr int ZW = ZCH + 8;
constexpr int XT = 256;  // threads per block, x kernels

__device__ __forceinline__ float2 ld2(const float* p) {
  return *reinterpret_cast<const float2*>(p);
}
__device__ __forceinline__ float2 ldg2(const float* p) {
  return __ldg(reinterpret_cast<const float2*>(p));
}
__device__ __forceinline__ void st2(float* p, float2 v) { *reinterpret_cast<float2*>(p) = v; }
__device__ __forceinline__ float4 ld4(const float* p) {
  return *reinterpret_cast<const float4*>(p);
}
__device__ __forceinline__ float4 ldg4(const float* p) {
  return __ldg(reinterpret_cast<const float4*>(p));
}
__device__ __forceinline__ void st4(float* p, const float* v) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }

// D2 and D1 on column pairs with the packed FP32 pipe (same rounding
// sequence as the scalar forms: one multiply, then a chain of fused adds).
__device__ __forceinline__ float2 d2p(const float2* w) {
  float2 r = __fmul2_rn(f2(kC0), w[4]);
  r = __ffma2_rn(f2(kC1), __fadd2_rn(w[5], w[3]), r);
  r = __ffma2_rn(f2(kC2), __fadd2_rn(w[6], w[2]), r);
  r = __ffma2_rn(f2(kC3), __fadd2_rn(w[7], w[1]), r);
  r = __ffma2_rn(f2(kC4), __fadd2_rn(w[8], w[0]), r);
  return r;
}
__device__ __forceinline__ float2 neg2(float2 v) { return make_float2(-v.x, -v.y); }
__device__ __forceinline__ float2 d1p(const float2* w) {
  float2 r = __fmul2_rn(f2(kD1), __fadd2_rn(w[5], neg2(w[3])));
  r = __ffma2_rn(f2(kD2), __fadd2_rn(w[6], neg2(w[2])), r);
  r = __ffma2_rn(f2(kD3), __fadd2_rn(w[7], neg2(w[1])), r);
  r = __ffma2_rn(f2(kD4), __fadd2_rn(w[8], neg2(w[0])), r);
  return r;
}

// ------------------------------------------------------------- forward, z
// blockIdx.y: strip (top [0, P), bottom [P+nz, NZ)) times chunk of ZCH rows;
// blockIdx.z: shot.
__global__ void __launch_bounds__(ZT) ac_cz_fwd_kernel(const AcCorrArgs a) {
  grid_dep_wait();
  grid_dep_trigger();
  if (*a.status) return;
  const Geom& g = a.g;
  const int x = 2 * (blockIdx.x * ZT + threadIdx.x);
  if (x >= g.NX) return;
  const int nch = (g.P + ZCH - 1) / ZCH;
  const int strip = (int)blockIdx.y >= nch ? 1 : 0;
  const int base = strip ? g.P + g.nz : 0;
  const int zs = base + ((int)blockIdx.y - strip * nch) * ZCH;
  const int ze = min(zs + ZCH, base + g.P);
  const size_t so = (size_t)blockIdx.z * g.fstride + x;
  const float* u = a.u + so;
  const float* pin = a.pin + so;
  float2 wu[ZW], wp[ZW], zt[ZCH], kk[ZCH], un[ZCH];
#pragma unroll
  for (int k = 0; k < ZW; ++k) {
    const int zz = zs - 4 + k;
    const bool ok = zz >= 0 && zz < g.NZ;
    const size_t o = (size_t)zz * g.NXp;
    wu[k] = ok ? ldg2(u + o) : f2(0.f);
    wp[k] = ok ? ldg2(pin + o) : f2(0.f);
  }
#pragma unroll
  for (int q = 0; q < ZCH; ++q) {
    const bool ok = zs + q < ze;
    const size_t o = (size_t)(zs + q) * g.NXp;
    zt[q] = ok ? ld2(a.zeta + so + o) : f2(0.f);
    kk[q] = ok ? ldg2(a.K + x + o) : f2(0.f);
    un[q] = ok ? ld2(a.un + so + o) : f2(0.f);
  }
  // ring cells of these rows that lie outside the x strips
  const bool sv0 = x >= g.P && x < g.P + g.nx, sv1 = x + 1 >= g.P && x + 1 < g.P + g.nx;
#pragma unroll
  for (int q = 0; q < ZCH; ++q) {
    const int z = zs + q;
    if (z >= ze) break;
    const float2 A = f2(__ldg(a.az + z)), B = f2(__ldg(a.bz + z));
    const float2 d2u = d2p(wu + q), d1u = d1p(wu + q), dp = d1p(wp + q);
    const float2 zn = __ffma2_rn(A, zt[q], __fmul2_rn(B, __fadd2_rn(d2u, dp)));
    const float2 po = __ffma2_rn(A, wp[q + 4], __fmul2_rn(B, d1u));
    const float2 v = __ffma2_rn(kk[q], __fadd2_rn(dp, zn), un[q]);
    const size_t o = so + (size_t)z * g.NXp;
    st2(a.pout + o, po);
    st2(a.zeta + o, zn);
    st2(a.un + o, v);
    if (a.save) {
      const int r0 = sv0 ? ring_index(g, z, x) : -1;
      const int r1 = sv1 ? ring_index(g, z, x + 1) : -1;
      float* sb = a.save + (size_t)blockIdx.z * g.nring;
      if (r0 >= 0) sb[r0] = v.x;
      if (r1 >= 0) sb[r1] = v.y;
    }
  }
}

// ---------------------------------------------------------------- x groups
// The x kernels cover a left and a right band of columns in 4-cell groups:
// left groups [0, gl), right groups [gr0, ceil(NX/4)).  Thread -> (row, group)
struct XBands {
  int gl, gr0, ngr;
};
__host__ __device__ __forceinline__ XBands x_bands(int lo_end, int hi_start, int NX) {
  XBands b;
  b.gl = (lo_end + 3) / 4;
  b.gr0 = hi_start / 4;
  if (b.gr0 < b.gl) b.gr0 = b.gl;
  b.ngr = b.gl + (NX + 3) / 4 - b.gr0;
  return b;
}

// 12 cells x-4 .. x+7 of a row (zero outside [0, NXp))
__device__ __forceinline__ void ldrow12(const float* row, int x, int NXp, float* e) {
  const float4 l = x >= 4 ? ldg4(row + x - 4) : make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 c = ldg4(row + x);
  const float4 r = x + 4 < NXp ? ldg4(row + x + 4) : make_float4(0.f, 0.f, 0.f, 0.f);
  f4a(l, e);
  f4a(c, e + 4);
  f4a(r, e + 8);
}

// ------------------------------------------------------------- forward, x
// Strip columns [0, P) and [P+nx, NX), all rows.
__global__ void __launch_bounds__(XT) ac_cx_fwd_kernel(const AcCorrArgs a, const XBands xb) {
  grid_dep_wait();
  grid_dep_trigger();
  if (*a.status) return;
  const Geom& g = a.g;
  const int idx = blockIdx.x * XT + threadIdx.x;
  const int z = idx / xb.ngr;
  if (z >= g.NZ) return;
  const int j = idx - z * xb.ngr;
  const int x = 4 * (j < xb.gl ? j : xb.gr0 + (j - xb.gl));
  const size_t ro = (size_t)blockIdx.y * g.fstride + (size_t)z * g.NXp;
  float e[12], f[12], zt[4], kk[4], un[4], A[4], B[4];
  ldrow12(a.u + ro, x, g.NXp, e);
  ldrow12(a.pin + ro, x, g.NXp, f);
  f4a(ld4(a.zeta + ro + x), zt);
  f4a(ldg4(a.K + (size_t)z * g.NXp + x), kk);
  f4a(ld4(a.un + ro + x), un);
  f4a(ldg4(a.ax + x), A);
  f4a(ldg4(a.bx + x), B);
  float po[4], zo[4], uo[4];
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
    uo[c] = m ? un[c] + kk[c] * (dp + zn) : un[c];
  }
  st4(a.pout + ro + x, po);
  st4(a.zeta + ro + x, zo);
  st4(a.un + ro + x, uo);
  if (a.save) {
    float* sb = a.save + (size_t)blockIdx.y * g.nring;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if (!(x_border(g, x + c) && x + c < g.NX)) continue;
      const int ri = ring_index(g, z, x + c);
      if (ri >= 0) sb[ri] = uo[c];
    }
  }
}

// Row bands of the backward z kernel and column bands of the backward x
// kernel: everything within 4 cells of the border, without overlap.
__host__ __device__ __forceinline__ int band_lo_end(int P, int N) { return min(P + 4, N); }
__host__ __device__ __forceinline__ int band_hi_start(int P, int n, int N) {
  return max(P + n - 4, band_lo_end(P, N));
}

// ------------------------------------------------------------ backward, z
// Bands [0, P+4) and [P+nz-4, NZ) in chunks of ZCH rows; blockIdx.y: band
// times chunk.
__global__ void __launch_bounds__(ZT) ac_cz_bwd_kernel(const AcCorrArgs a) {
  grid_dep_wait();
  grid_dep_trigger();
  if (*a.status) return;
  const Geom& g = a.g;
  const int x = 2 * (blockIdx.x * ZT + threadIdx.x);
  if (x >= g.NX) return;
  const int lo_end = band_lo_end(g.P, g.NZ), hi_start = band_hi_start(g.P, g.nz, g.NZ);
  const int nlo = (lo_end + ZCH - 1) / ZCH;
  const int band = (int)blockIdx.y >= nlo ? 1 : 0;
  const int zs = (band ? hi_start : 0) + ((int)blockIdx.y - band * nlo) * ZCH;
  const int ze = min(zs + ZCH, band ? g.NZ : lo_end);
  if (zs >= ze) return;
  const size_t so = (size_t)blockIdx.z * g.fstride + x;
  const float* m1 = a.u + so;  // mu^{n+1}
  const float* zb = a.zeta + so;
  const float* pb = a.pin + so;
  float2 wm[ZW], wz[ZW], wp[ZW], mo[ZCH], kk[ZCH];
  float bb[ZW];
#pragma unroll
  for (int k = 0; k < ZW; ++k) {
    const int zz = zs - 4 + k;
    const bool ok = zz >= 0 && zz < g.NZ;
    const size_t o = (size_t)zz * g.NXp;
    wm[k] = ok ? ldg2(m1 + o) : f2(0.f);
    wz[k] = ok ? ldg2(zb + o) : f2(0.f);
    wp[k] = ok ? ldg2(pb + o) : f2(0.f);
    bb[k] = ok ? __ldg(a.bz + zz) : 0.f;
  }
#pragma unroll
  for (int q = 0; q < ZCH; ++q) {
    const bool ok = zs + q < ze;
    const size_t o = (size_t)(zs + q) * g.NXp;
    mo[q] = ok ? ld2(a.un + so + o) : f2(0.f);
    kk[q] = ok ? ldg2(a.K + x + o) : f2(0.f);
  }
  float2 wc[ZW], wb[ZW], wg[ZW];
#pragma unroll
  for (int k = 0; k < ZW; ++k) {
    const int zz = zs - 4 + k;
    const float2 b = f2(bb[k]);
    wc[k] = __fmul2_rn(b, __fadd2_rn(wm[k], wz[k]));
    wb[k] = __fmul2_rn(b, wp[k]);
    // m G: zero off the strip rows
    wg[k] = (zz >= 0 && zz < g.NZ && z_border(g, zz)) ? __fadd2_rn(wm[k], wc[k]) : f2(0.f);
  }
#pragma unroll
  for (int q = 0; q < ZCH; ++q) {
    const int z = zs + q;
    if (z >= ze) break;
    const size_t o = so + (size_t)z * g.NXp;
    const float2 corr = __fadd2_rn(d2p(wc + q), neg2(d1p(wb + q)));
    st2(a.un + o, __ffma2_rn(kk[q], corr, mo[q]));  // mu^n
    if (z_border(g, z)) {
      const float2 A = f2(__ldg(a.az + z));
      st2(a.pout + o, __fadd2_rn(__fmul2_rn(A, wp[q + 4]), neg2(d1p(wg + q))));
      st2(a.zout + o, __fmul2_rn(A, __fadd2_rn(wm[q + 4], wz[q + 4])));
    }
  }
}

// ------------------------------------------------------------ backward, x
// Bands [0, P+4) and [P+nx-4, NX), all rows.
__global__ void __launch_bounds__(XT) ac_cx_bwd_kernel(const AcCorrArgs a, const XBands xb) {
  grid_dep_wait();
  grid_dep_trigger();
  if (*a.status) return;
  const Geom& g = a.g;
  const int idx = blockIdx.x * XT + threadIdx.x;
  const int z = idx / xb.ngr;
  if (z >= g.NZ) return;
  const int j = idx - z * xb.ngr;
  const int x = 4 * (j < xb.gl ? j : xb.gr0 + (j - xb.gl));
  const size_t ro = (size_t)blockIdx.y * g.fstride + (size_t)z * g.NXp;
  float em[12], ez[12], ep[12], bb[12], kk[4], mo[4], A[4];
  ldrow12(a.u + ro, x, g.NXp, em);
  ldrow12(a.zeta + ro, x, g.NXp, ez);
  ldrow12(a.pin + ro, x, g.NXp, ep);
  ldrow12(a.bx, x, g.NXp, bb);
  f4a(ldg4(a.K + (size_t)z * g.NXp + x), kk);
  f4a(ld4(a.un + ro + x), mo);
  f4a(ldg4(a.ax + x), A);
  float C[12], Bv[12], G[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const int xx = x - 4 + k;
    C[k] = bb[k] * (em[k] + ez[k]);
    Bv[k] = bb[k] * ep[k];
    G[k] = (xx >= 0 && xx < g.NX && x_border(g, xx)) ? em[k] + C[k] : 0.f;
  }
  float uo[4], po[4], zo[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const float* Cc = C + c;
    const float* Bc = Bv + c;
    const float* Gc = G + c;
    const float corr = d2(Cc[0], Cc[1], Cc[2], Cc[3], Cc[4], Cc[5], Cc[6], Cc[7], Cc[8]) -
                       d1(Bc[0], Bc[1], Bc[2], Bc[3], Bc[5], Bc[6], Bc[7], Bc[8]);
    const bool in = x + c < g.NX;
    const bool m = in && x_border(g, x + c);
    uo[c] = in ? mo[c] + kk[c] * corr : mo[c];
    po[c] = m ? A[c] * ep[c + 4] - d1(Gc[0], Gc[1], Gc[2], Gc[3], Gc[5], Gc[6], Gc[7], Gc[8])
              : 0.f;
    zo[c] = m ? A[c] * (em[c + 4] + ez[c + 4]) : 0.f;
  }
  st4(a.un + ro + x, uo);
  st4(a.pout + ro + x, po);
  st4(a.zout + ro + x, zo);
}

}  // namespace

void launch_ac_corr_fwd(const AcCorrArgs& z, const AcCorrArgs& x, cudaStream_t st) {
  const Geom& g = z.g;
  if (g.P <= 0 || g.nshot <= 0) return;
  void* tok = profile_begin(SWEEP_K_AC_FWD_FR, st);
  const dim3 gz((g.NX + 2 * ZT - 1) / (2 * ZT), 2 * ((g.P + ZCH - 1) / ZCH), g.nshot);
  launch_dependent(ac_cz_fwd_kernel, gz, dim3(ZT), 0, st, z);
  const XBands xb = x_bands(g.P, g.P + g.nx, g.NX);
  const dim3 gx((unsigned)(((long long)g.NZ * xb.ngr + XT - 1) / XT), g.nshot, 1);
  launch_dependent(ac_cx_fwd_kernel, gx, dim3(XT), 0, st, x, xb);
  profile_end(tok, st);
  note_launches(2);
}

void launch_ac_corr_bwd(const AcCorrArgs& z, const AcCorrArgs& x, cudaStream_t st) {
  const Geom& g = z.g;
  if (g.P <= 0 || g.nshot <= 0) return;
  void* tok = profile_begin(SWEEP_K_AC_BWD_FR, st);
  const int lo_end = band_lo_end(g.P, g.NZ), hi_start = band_hi_start(g.P, g.nz, g.NZ);
  const dim3 gz((g.NX + 2 * ZT - 1) / (2 * ZT),
                (lo_end + ZCH - 1) / ZCH + (g.NZ - hi_start + ZCH - 1) / ZCH, g.nshot);
  launch_dependent(ac_cz_bwd_kernel, gz, dim3(ZT), 0, st, z);
  const XBands xb =
      x_bands(band_lo_end(g.P, g.NX), band_hi_start(g.P, g.nx, g.NX), g.NX);
  const dim3 gx((unsigned)(((long long)g.NZ * xb.ngr + XT - 1) / XT), g.nshot, 1);
  launch_dependent(ac_cx_bwd_kernel, gx, dim3(XT), 0, st, x, xb);
  profile_end(tok, st);
  note_launches(2);
}

}  // namespace sweep
