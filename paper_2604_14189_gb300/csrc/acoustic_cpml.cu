// Second kernel of the acoustic time step: CPML terms and receivers.
//
// The stencil kernels (acoustic_interior.cu) update every cell of the padded
// grid as if there were no absorbing layer.  The convolutional-PML terms are
// additive per axis, and they read only the step's inputs (u^n or mu^{n+1}
// and the memory variables), never the stencil kernel's output.  So one
// kernel adds both axes' terms, and the receiver work, to the output field
// with vector reductions (red.global.add): its z part, x part and receiver
// part run concurrently, and a cell in a corner of the border simply gets
// two additions.  See acoustic_common.cuh for the full update:
//
// forward, axis strip cells (sigma != 0 along that axis):
//   W = D2 u^n + D1 psi^{n-1};  zeta^n = a zeta^{n-1} + b W;
//   psi^n = a psi^{n-1} + b D1 u^n;  u^{n+1} += K (D1 psi^{n-1} + zeta^n)
//   receivers: d[n] = u^{n+1}(r) (interior cells: no CPML term reaches them)
//   boundary save: the ring cells of u^n into their slot (gradient mode)
// backward, strip cells and the 4 cells next to them:
//   C = b (mu^{n+1} + zetabar^n),  B = b psibar^n   (zero off the strip)
//   mu^n += K (D2 C - D1 B)
//   strip cells: psibar^{n-1} = a psibar^n - D1 (m (mu^{n+1} + C)),
//                zetabar^{n-1} = a (mu^{n+1} + zetabar^n)
//   receivers: mu^n(r) += K(r) res^{n-1}(r)
//   ring restore: u^{n-1} on the ring from the forward save (gradient mode)
//
// The profiles a, b are zero off the border, and so are psi, zeta and their
// adjoints (never written there), which removes most masks.
//
// z part: a thread owns 2 adjacent columns (8-byte accesses, coalesced across
// the warp) and a chunk of ZCH rows; x part: a thread owns 4 consecutive
// cells of a row (16-byte accesses) and reads its 4 + 4 x-neighbours as two
// more 16-byte loads.  Every load of a thread is issued before its
// arithmetic, so the memory latency is paid once per thread.
#include "acoustic_common.cuh"

namespace sweep {
namespace {

constexpr int FT = 256;  // threads per block
constexpr int ZCH = 4;   // rows per thread, z part
constexpr int ZW = ZCH + 8;

__device__ __forceinline__ float2 ldg2(const float* p) {
  return __ldg(reinterpret_cast<const float2*>(p));
}
__device__ __forceinline__ void st2(float* p, float2 v) { *reinterpret_cast<float2*>(p) = v; }
__device__ __forceinline__ float4 ldg4(const float* p) {
  return __ldg(reinterpret_cast<const float4*>(p));
}
__device__ __forceinline__ float4 ld4(const float* p) {
  return *reinterpret_cast<const float4*>(p);
}
__device__ __forceinline__ void st4(float* p, const float* v) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void red2(float* p, float2 v) {
  atomicAdd(reinterpret_cast<float2*>(p), v);
}
__device__ __forceinline__ void red4(float* p, const float* v) {
  atomicAdd(reinterpret_cast<float4*>(p), make_float4(v[0], v[1], v[2], v[3]));
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

// 12 cells x-4 .. x+7 of a row (zero outside [0, NXp))
__device__ __forceinline__ void ldrow12(const float* row, int x, int NXp, float* e) {
  const float4 l = x >= 4 ? ldg4(row + x - 4) : make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 c = ldg4(row + x);
  const float4 r = x + 4 < NXp ? ldg4(row + x + 4) : make_float4(0.f, 0.f, 0.f, 0.f);
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

// (column pair, row chunk, shot) of z-part thread t; false past the end
__device__ __forceinline__ bool z_item(const AcFixArgs& a, long long t, int& x, int& ch,
                                       int& s) {
  const int cp = (int)(t % a.ncp);
  const long long r = t / a.ncp;
  ch = (int)(r % a.nchz);
  s = (int)(r / a.nchz);
  x = 2 * cp;
  return s < a.g.nshot && x < a.g.NX;
}

// (row, column group origin, shot) of x-part thread t
__device__ __forceinline__ bool x_item(const AcFixArgs& a, long long t, int& z, int& x,
                                       int& s) {
  const int j = (int)(t % a.xb.ngr);
  const long long r = t / a.xb.ngr;
  z = (int)(r % a.g.NZ);
  s = (int)(r / a.g.NZ);
  x = 4 * (j < a.xb.gl ? j : a.xb.gr0 + (j - a.xb.gl));
  return s < a.g.nshot;
}

// ------------------------------------------------------------------ forward
__device__ __forceinline__ void fwd_z(const AcFixArgs& a, long long t) {
  const Geom& g = a.g;
  int x, ch, s;
  if (!z_item(a, t, x, ch, s)) return;
  const int nch = (g.P + ZCH - 1) / ZCH;  // chunks per strip
  const int strip = ch >= nch ? 1 : 0;
  const int base = strip ? g.P + g.nz : 0;
  const int zs = base + (ch - strip * nch) * ZCH;
  const int ze = min(zs + ZCH, base + g.P);
  const size_t so = (size_t)s * g.fstride + x;
  float2 wu[ZW], wp[ZW], zt[ZCH], kk[ZCH];
#pragma unroll
  for (int k = 0; k < ZW; ++k) {
    const int zz = zs - 4 + k;
    const bool ok = zz >= 0 && zz < g.NZ;
    const size_t o = (size_t)zz * g.NXp;
    wu[k] = ok ? ldg2(a.u + so + o) : f2(0.f);
    wp[k] = ok ? ldg2(a.pzin + so + o) : f2(0.f);
  }
#pragma unroll
  for (int q = 0; q < ZCH; ++q) {
    const bool ok = zs + q < ze;
    const size_t o = (size_t)(zs + q) * g.NXp;
    zt[q] = ok ? *reinterpret_cast<const float2*>(a.zzin + so + o) : f2(0.f);
    kk[q] = ok ? ldg2(a.K + x + o) : f2(0.f);
  }
#pragma unroll
  for (int q = 0; q < ZCH; ++q) {
    const int z = zs + q;
    if (z >= ze) break;
    const float2 A = f2(__ldg(a.az + z)), B = f2(__ldg(a.bz + z));
    const float2 d2u = d2p(wu + q), d1u = d1p(wu + q), dp = d1p(wp + q);
    const float2 zn = __ffma2_rn(A, zt[q], __fmul2_rn(B, __fadd2_rn(d2u, dp)));
    const float2 po = __ffma2_rn(A, wp[q + 4], __fmul2_rn(B, d1u));
    const size_t o = so + (size_t)z * g.NXp;
    st2(a.pzout + o, po);
    st2(a.zzout + o, zn);
    red2(a.un + o, __fmul2_rn(kk[q], __fadd2_rn(dp, zn)));
  }
}

__device__ __forceinline__ void fwd_x(const AcFixArgs& a, long long t) {
  const Geom& g = a.g;
  int z, x, s;
  if (!x_item(a, t, z, x, s)) return;
  const size_t ro = (size_t)s * g.fstride + (size_t)z * g.NXp;
  float e[12], f[12], zt[4], kk[4], A[4], B[4];
  ldrow12(a.u + ro, x, g.NXp, e);
  ldrow12(a.pxin + ro, x, g.NXp, f);
  f4a(ld4(a.zxin + ro + x), zt);
  f4a(ldg4(a.K + (size_t)z * g.NXp + x), kk);
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
  red4(a.un + ro + x, du);
}

__device__ __forceinline__ void fwd_rec(const AcFixArgs& a, long long t) {
  const Geom& g = a.g;
  const int r = (int)(t % g.nrec), s = (int)(t / g.nrec);
  if (s >= g.nshot) return;
  const long long i = (long long)s * g.nrec + r;
  const int rz = a.rec[2 * i] + g.P, rx = a.rec[2 * i + 1] + g.P;
  a.data[i * g.nt + a.n] = a.un[(size_t)s * g.fstride + (size_t)rz * g.NXp + rx];
}

// Interior coordinates (zi, xi) of ring cell ri: the inverse of ring_index
// (rows above, rows below, then the left and right side columns).
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
__device__ __forceinline__ void fwd_ring(const AcFixArgs& a, long long t) {
  const Geom& g = a.g;
  const int nq = (g.nring + 3) / 4;
  const int q = (int)(t % nq), s = (int)(t / nq);
  if (s >= g.nshot) return;
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

__global__ void __launch_bounds__(FT) ac_fix_fwd_kernel(const AcFixArgs a) {
  grid_dep_wait();
  grid_dep_trigger();
  if (*a.status) return;
  int b = blockIdx.x;
  if (b < a.nbz) {
    fwd_z(a, (long long)b * FT + threadIdx.x);
    return;
  }
  b -= a.nbz;
  if (b < a.nbx) {
    fwd_x(a, (long long)b * FT + threadIdx.x);
    return;
  }
  b -= a.nbx;
  if (b < a.nbr) {
    fwd_rec(a, (long long)b * FT + threadIdx.x);
    return;
  }
  b -= a.nbr;
  fwd_ring(a, (long long)b * FT + threadIdx.x);
}

// ----------------------------------------------------------------- backward
__device__ __forceinline__ void bwd_z(const AcFixArgs& a, long long t) {
  const Geom& g = a.g;
  int x, ch, s;
  if (!z_item(a, t, x, ch, s)) return;
  const int lo_end = band_lo_end(g.P, g.NZ), hi_start = band_hi_start(g.P, g.nz, g.NZ);
  const int nlo = (lo_end + ZCH - 1) / ZCH;
  const int band = ch >= nlo ? 1 : 0;
  const int zs = (band ? hi_start : 0) + (ch - band * nlo) * ZCH;
  const int ze = min(zs + ZCH, band ? g.NZ : lo_end);
  if (zs >= ze) return;
  const size_t so = (size_t)s * g.fstride + x;
  float2 wm[ZW], wz[ZW], wp[ZW], kk[ZCH];
  float bb[ZW];
#pragma unroll
  for (int k = 0; k < ZW; ++k) {
    const int zz = zs - 4 + k;
    const bool ok = zz >= 0 && zz < g.NZ;
    const size_t o = (size_t)zz * g.NXp;
    wm[k] = ok ? ldg2(a.u + so + o) : f2(0.f);
    wz[k] = ok ? ldg2(a.zzin + so + o) : f2(0.f);
    wp[k] = ok ? ldg2(a.pzin + so + o) : f2(0.f);
    bb[k] = ok ? __ldg(a.bz + zz) : 0.f;
  }
#pragma unroll
  for (int q = 0; q < ZCH; ++q) {
    const bool ok = zs + q < ze;
    kk[q] = ok ? ldg2(a.K + x + (size_t)(zs + q) * g.NXp) : f2(0.f);
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
    red2(a.un + o, __fmul2_rn(kk[q], corr));  // mu^n
    if (z_border(g, z)) {
      const float2 A = f2(__ldg(a.az + z));
      st2(a.pzout + o, __fadd2_rn(__fmul2_rn(A, wp[q + 4]), neg2(d1p(wg + q))));
      st2(a.zzout + o, __fmul2_rn(A, __fadd2_rn(wm[q + 4], wz[q + 4])));
    }
  }
}

__device__ __forceinline__ void bwd_x(const AcFixArgs& a, long long t) {
  const Geom& g = a.g;
  int z, x, s;
  if (!x_item(a, t, z, x, s)) return;
  const size_t ro = (size_t)s * g.fstride + (size_t)z * g.NXp;
  float em[12], ez[12], ep[12], bb[12], kk[4], A[4];
  ldrow12(a.u + ro, x, g.NXp, em);
  ldrow12(a.zxin + ro, x, g.NXp, ez);
  ldrow12(a.pxin + ro, x, g.NXp, ep);
  ldrow12(a.bx, x, g.NXp, bb);
  f4a(ldg4(a.K + (size_t)z * g.NXp + x), kk);
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
  red4(a.un + ro + x, du);
  st4(a.pxout + ro + x, po);
  st4(a.zxout + ro + x, zo);
}

__device__ __forceinline__ void bwd_rec(const AcFixArgs& a, long long t) {
  const Geom& g = a.g;
  const int r = (int)(t % g.nrec), s = (int)(t / g.nrec);
  if (s >= g.nshot) return;
  const long long i = (long long)s * g.nrec + r;
  const int rz = a.rec[2 * i] + g.P, rx = a.rec[2 * i + 1] + g.P;
  const size_t c = (size_t)rz * g.NXp + rx;
  atomicAdd(a.un + (size_t)s * g.fstride + c, a.K[c] * a.res[i * g.nt + (a.n - 1)]);
}

// ring restore: u^{n-1} on the ring cells 4q .. 4q+3 from the forward save
// (the stencil kernel reconstructs the interior and leaves the ring alone)
__device__ __forceinline__ void bwd_ring(const AcFixArgs& a, long long t) {
  const Geom& g = a.g;
  const int nq = (g.nring + 3) / 4;
  const int q = (int)(t % nq), s = (int)(t / nq);
  if (s >= g.nshot) return;
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

__global__ void __launch_bounds__(FT) ac_fix_bwd_kernel(const AcFixArgs a) {
  grid_dep_wait();
  grid_dep_trigger();
  if (*a.status) return;
  int b = blockIdx.x;
  if (b < a.nbz) {
    bwd_z(a, (long long)b * FT + threadIdx.x);
    return;
  }
  b -= a.nbz;
  if (b < a.nbx) {
    bwd_x(a, (long long)b * FT + threadIdx.x);
    return;
  }
  b -= a.nbx;
  if (b < a.nbr) {
    bwd_rec(a, (long long)b * FT + threadIdx.x);
    return;
  }
  b -= a.nbr;
  bwd_ring(a, (long long)b * FT + threadIdx.x);
}

int blocks(long long threads) { return (int)((threads + FT - 1) / FT); }

}  // namespace

void launch_ac_fix_fwd(AcFixArgs a, cudaStream_t st) {
  const Geom& g = a.g;
  if (g.nshot <= 0) return;
  a.ncp = (g.NX + 1) / 2;
  a.nchz = g.P > 0 ? 2 * ((g.P + ZCH - 1) / ZCH) : 0;
  a.xb = x_bands(g.P, g.P + g.nx, g.NX);
  a.nbz = g.P > 0 ? blocks((long long)a.ncp * a.nchz * g.nshot) : 0;
  a.nbx = g.P > 0 ? blocks((long long)g.NZ * a.xb.ngr * g.nshot) : 0;
  a.nbr = (a.data && g.nrec > 0) ? blocks((long long)g.nrec * g.nshot) : 0;
  a.nbs = (a.save && g.nring > 0) ? blocks((long long)((g.nring + 3) / 4) * g.nshot) : 0;
  const int nb = a.nbz + a.nbx + a.nbr + a.nbs;
  if (nb == 0) return;
  void* tok = profile_begin(SWEEP_K_AC_FWD_FR, st);
  launch_dependent(ac_fix_fwd_kernel, dim3(nb), dim3(FT), 0, st, a);
  profile_end(tok, st);
  note_launches(1);
}

void launch_ac_fix_bwd(AcFixArgs a, cudaStream_t st) {
  const Geom& g = a.g;
  if (g.nshot <= 0) return;
  const int lo_end = band_lo_end(g.P, g.NZ), hi_start = band_hi_start(g.P, g.nz, g.NZ);
  a.ncp = (g.NX + 1) / 2;
  a.nchz = g.P > 0 ? (lo_end + ZCH - 1) / ZCH + (g.NZ - hi_start + ZCH - 1) / ZCH : 0;
  a.xb = x_bands(band_lo_end(g.P, g.NX), band_hi_start(g.P, g.nx, g.NX), g.NX);
  a.nbz = g.P > 0 ? blocks((long long)a.ncp * a.nchz * g.nshot) : 0;
  a.nbx = g.P > 0 ? blocks((long long)g.NZ * a.xb.ngr * g.nshot) : 0;
  a.nbr = (a.res && g.nrec > 0 && a.n >= 1) ? blocks((long long)g.nrec * g.nshot) : 0;
  a.nbs = (a.save && a.uring && g.nring > 0)
              ? blocks((long long)((g.nring + 3) / 4) * g.nshot)
              : 0;
  const int nb = a.nbz + a.nbx + a.nbr + a.nbs;
  if (nb == 0) return;
  void* tok = profile_begin(SWEEP_K_AC_BWD_FR, st);
  launch_dependent(ac_fix_bwd_kernel, dim3(nb), dim3(FT), 0, st, a);
  profile_end(tok, st);
  note_launches(1);
}

}  // namespace sweep
