// CPML correction kernels of the acoustic step.
//
// The plain-stencil kernels (acoustic_interior.cu) update every cell of the
// padded grid as if there were no absorbing layer.  The convolutional-PML
// terms are additive per axis, so each axis is corrected afterwards by a
// kernel that visits only the cells its terms reach (see
// acoustic_common.cuh for the full update):
//
// forward, axis strip cells (σ ≠ 0 along that axis):
//   W = D2 u^n + D1 psi^{n-1};  zeta^n = a zeta^{n-1} + b W;
//   psi^n = a psi^{n-1} + b D1 u^n;  u^{n+1} += K (D1 psi^{n-1} + zeta^n)
// backward, strip cells and the 4 cells next to them:
//   C = b (mu^{n+1} + zetabar^n),  B = b psibar^n   (zero off the strip)
//   mu^n += K (D2 C - D1 B)
//   strip cells: psibar^{n-1} = a psibar^n - D1 (m (mu^{n+1} + C)),
//                zetabar^{n-1} = a (mu^{n+1} + zetabar^n)
// The z kernels walk down a column per thread with register windows
// (coalesced across the warp); the x kernels stage row segments of the
// strips in shared memory.  The forward kernels also save the ring cells of
// their strips after the final update (z kernel: ring cells outside the x
// strips; x kernel: ring cells inside them, the x kernel runs last).
#include "acoustic_common.cuh"

namespace sweep {
namespace {

constexpr int CZ_T = 128;   // threads (columns) per block, z kernels
constexpr int CX_TZ = 16;   // rows per block, x kernels
constexpr int CX_TX = 64;   // strip columns per block, x kernels
constexpr int CX_T = 256;
constexpr int CX_W = CX_TX + 16;  // staged width (halo + alignment)

__device__ __forceinline__ float ldz(const float* f, const Geom& g, int z, int x) {
  return (z >= 0 && z < g.NZ) ? f[(long long)z * g.NXp + x] : 0.f;
}

// ------------------------------------------------------------- forward, z
// A thread owns one column and a chunk of CH rows of one strip; every load
// of the chunk is issued before any arithmetic so that the memory latency is
// paid once per chunk.  blockIdx.y: strip (top [0, P), bottom [P+nz, NZ))
// times chunk; blockIdx.z: shot.
constexpr int CH = 8;
constexpr int CW = CH + 8;

__global__ void __launch_bounds__(CZ_T) ac_cz_fwd_kernel(const AcCorrArgs a) {
  if (*a.status) return;
  const Geom& g = a.g;
  const int x = blockIdx.x * CZ_T + threadIdx.x;
  if (x >= g.NX) return;
  const int s = blockIdx.z;
  const long long so = (long long)s * g.fstride;
  const int nch = (g.P + CH - 1) / CH;
  const int strip = blockIdx.y / nch, ch = blockIdx.y - strip * nch;
  const int base = strip == 0 ? 0 : g.P + g.nz;
  const int zs = base + ch * CH;
  const int ze = min(zs + CH, base + g.P);
  const float* u = a.u + so;
  const float* pin = a.pin + so;
  float wu[CW], wp[CW], zt[CH], kk[CH], un[CH];
#pragma unroll
  for (int k = 0; k < CW; ++k) {
    wu[k] = ldz(u, g, zs - 4 + k, x);
    wp[k] = ldz(pin, g, zs - 4 + k, x);
  }
#pragma unroll
  for (int q = 0; q < CH; ++q) {
    const int z = zs + q;
    const long long c = (long long)z * g.NXp + x;
    const bool ok = z < ze;
    zt[q] = ok ? a.zeta[so + c] : 0.f;
    kk[q] = ok ? a.K[c] : 0.f;
    un[q] = ok ? a.un[so + c] : 0.f;
  }
  const bool xin = x >= g.P && x < g.P + g.nx;
#pragma unroll
  for (int q = 0; q < CH; ++q) {
    const int z = zs + q;
    if (z >= ze) break;
    const float* w = wu + q;
    const float* p = wp + q;
    const long long c = (long long)z * g.NXp + x;
    const float A = __ldg(a.az + z), B = __ldg(a.bz + z);
    const float d2u = d2(w[0], w[1], w[2], w[3], w[4], w[5], w[6], w[7], w[8]);
    const float d1u = d1(w[0], w[1], w[2], w[3], w[5], w[6], w[7], w[8]);
    const float d1p = d1(p[0], p[1], p[2], p[3], p[5], p[6], p[7], p[8]);
    const float zn = A * zt[q] + B * (d2u + d1p);
    a.pout[so + c] = A * p[4] + B * d1u;
    a.zeta[so + c] = zn;
    const float v = un[q] + kk[q] * (d1p + zn);
    a.un[so + c] = v;
    if (a.save && xin) {
      const int ri = ring_index(g, z, x);
      if (ri >= 0) a.save[(long long)s * g.nring + ri] = v;
    }
  }
}

// ------------------------------------------------------------- forward, x
// Two column bands, left [0, lw) and right [r0, NX), tiled by CX_TZ x CX_TX.
// blockIdx.x: tile index over both bands; blockIdx.z: shot.
__host__ __device__ __forceinline__ int x_band_tiles(const Geom& g, int w) {
  return ((w + CX_TX - 1) / CX_TX) * ((g.NZ + CX_TZ - 1) / CX_TZ);
}

__device__ __forceinline__ void x_tile(const Geom& g, int t, int lw, int r0, int& z0, int& xa,
                                       int& xb) {
  const int ntz = (g.NZ + CX_TZ - 1) / CX_TZ;
  const int nl = x_band_tiles(g, lw);
  const bool right = t >= nl;
  const int w = right ? g.NX - r0 : lw;
  const int ntx = (w + CX_TX - 1) / CX_TX;
  const int r = right ? t - nl : t;
  const int tz = r / ntx, tx = r - tz * ntx;
  (void)ntz;
  z0 = tz * CX_TZ;
  xa = (right ? r0 : 0) + tx * CX_TX;
  xb = min(xa + CX_TX, right ? g.NX : lw);
}

// Row bands of the backward z kernel and column bands of the backward x
// kernel: everything within 4 cells of the border, without overlap.
__host__ __device__ __forceinline__ int band_lo_end(int P, int N) { return min(P + 4, N); }
__host__ __device__ __forceinline__ int band_hi_start(int P, int n, int N) {
  return max(P + n - 4, band_lo_end(P, N));
}

__global__ void __launch_bounds__(CX_T) ac_cx_fwd_kernel(const AcCorrArgs a) {
  __shared__ __align__(16) float su[CX_TZ * CX_W];
  __shared__ __align__(16) float sp[CX_TZ * CX_W];
  if (*a.status) return;
  const Geom& g = a.g;
  const int s = blockIdx.z;
  const long long so = (long long)s * g.fstride;
  int z0, x0, x1;
  x_tile(g, blockIdx.x, g.P, g.P + g.nx, z0, x0, x1);
  const int xs = (x0 - 4) & ~3;  // aligned staging origin (covers x0-4 .. x0+CX_TX+4)
  for (int idx = threadIdx.x; idx < CX_TZ * (CX_W / 4); idx += CX_T) {
    const int r = idx / (CX_W / 4), c4 = idx - r * (CX_W / 4);
    const int z = z0 + r, x = xs + 4 * c4;
    float4 vu = make_float4(0.f, 0.f, 0.f, 0.f), vp = vu;
    if (z < g.NZ && x >= 0 && x < g.NXp) {
      vu = *reinterpret_cast<const float4*>(a.u + so + (long long)z * g.NXp + x);
      vp = *reinterpret_cast<const float4*>(a.pin + so + (long long)z * g.NXp + x);
    }
    *reinterpret_cast<float4*>(su + r * CX_W + 4 * c4) = vu;
    *reinterpret_cast<float4*>(sp + r * CX_W + 4 * c4) = vp;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < CX_TZ * CX_TX; idx += CX_T) {
    const int r = idx / CX_TX, cc = idx - r * CX_TX;
    const int z = z0 + r, x = x0 + cc;
    if (z >= g.NZ || x >= x1) continue;
    const float* ur = su + r * CX_W + (x - xs);
    const float* pr = sp + r * CX_W + (x - xs);
    const float d2u = d2(ur[-4], ur[-3], ur[-2], ur[-1], ur[0], ur[1], ur[2], ur[3], ur[4]);
    const float d1u = d1(ur[-4], ur[-3], ur[-2], ur[-1], ur[1], ur[2], ur[3], ur[4]);
    const float d1p = d1(pr[-4], pr[-3], pr[-2], pr[-1], pr[1], pr[2], pr[3], pr[4]);
    const long long c = (long long)z * g.NXp + x;
    const float A = __ldg(a.ax + x), B = __ldg(a.bx + x);
    const float zn = A * a.zeta[so + c] + B * (d2u + d1p);
    a.pout[so + c] = A * pr[0] + B * d1u;
    a.zeta[so + c] = zn;
    const float v = a.un[so + c] + a.K[c] * (d1p + zn);
    a.un[so + c] = v;
    if (a.save) {
      const int ri = ring_index(g, z, x);
      if (ri >= 0) a.save[(long long)s * g.nring + ri] = v;
    }
  }
}

// ------------------------------------------------------------ backward, z
// Bands [0, P+4) and [P+nz-4, NZ) (without overlap), chunks of CH rows per
// thread, all loads of a chunk issued first.  blockIdx.y: band times chunk.
__global__ void __launch_bounds__(CZ_T) ac_cz_bwd_kernel(const AcCorrArgs a) {
  if (*a.status) return;
  const Geom& g = a.g;
  const int x = blockIdx.x * CZ_T + threadIdx.x;
  if (x >= g.NX) return;
  const int s = blockIdx.z;
  const long long so = (long long)s * g.fstride;
  const int lo_end = band_lo_end(g.P, g.NZ), hi_start = band_hi_start(g.P, g.nz, g.NZ);
  const int nlo = (lo_end + CH - 1) / CH;
  const int band = (int)blockIdx.y >= nlo ? 1 : 0;
  const int ch = band ? blockIdx.y - nlo : blockIdx.y;
  const int zs = (band ? hi_start : 0) + ch * CH;
  const int ze = min(zs + CH, band ? g.NZ : lo_end);
  if (zs >= ze) return;
  const float* m1 = a.u + so;  // mu^{n+1}
  const float* zb = a.zeta + so;
  const float* pb = a.pin + so;
  // rows zs-4 .. zs+CH+3: C = b (mu + zetabar), B = b psibar, m G
  float wm[CW], wz[CW], wp[CW];
#pragma unroll
  for (int k = 0; k < CW; ++k) {
    const int zz = zs - 4 + k;
    const bool inb = zz >= 0 && zz < g.NZ;
    const bool bord = inb && z_border(g, zz);
    const long long c = (long long)zz * g.NXp + x;
    wm[k] = bord ? m1[c] : 0.f;
    wz[k] = bord ? zb[c] : 0.f;
    wp[k] = bord ? pb[c] : 0.f;
  }
  float mo[CH], kk[CH];
#pragma unroll
  for (int q = 0; q < CH; ++q) {
    const int z = zs + q;
    const long long c = (long long)z * g.NXp + x;
    mo[q] = z < ze ? a.un[so + c] : 0.f;
    kk[q] = z < ze ? a.K[c] : 0.f;
  }
  float wc[CW], wb[CW], wg[CW];
#pragma unroll
  for (int k = 0; k < CW; ++k) {
    const int zz = zs - 4 + k;
    const float b = (zz >= 0 && zz < g.NZ && z_border(g, zz)) ? __ldg(a.bz + zz) : 0.f;
    wc[k] = b * (wm[k] + wz[k]);
    wb[k] = b * wp[k];
    wg[k] = wm[k] + wc[k];  // zero off the border rows (m G)
  }
#pragma unroll
  for (int q = 0; q < CH; ++q) {
    const int z = zs + q;
    if (z >= ze) break;
    const long long c = (long long)z * g.NXp + x;
    const float* C = wc + q;
    const float* B = wb + q;
    const float* G = wg + q;
    const float corr = d2(C[0], C[1], C[2], C[3], C[4], C[5], C[6], C[7], C[8]) -
                       d1(B[0], B[1], B[2], B[3], B[5], B[6], B[7], B[8]);
    a.un[so + c] = mo[q] + kk[q] * corr;  // mu^n
    if (z_border(g, z)) {
      const float A = __ldg(a.az + z);
      a.pout[so + c] = A * wp[q + 4] - d1(G[0], G[1], G[2], G[3], G[5], G[6], G[7], G[8]);
      a.zout[so + c] = A * (wm[q + 4] + wz[q + 4]);
    }
  }
}

// ------------------------------------------------------------ backward, x
// bands [0, P+4) and [P+nx-4, NX) over all rows
__global__ void __launch_bounds__(CX_T) ac_cx_bwd_kernel(const AcCorrArgs a) {
  __shared__ __align__(16) float sc[CX_TZ * CX_W];  // C
  __shared__ __align__(16) float sb[CX_TZ * CX_W];  // B
  __shared__ __align__(16) float sg[CX_TZ * CX_W];  // m G
  if (*a.status) return;
  const Geom& g = a.g;
  const int s = blockIdx.z;
  const long long so = (long long)s * g.fstride;
  int z0, x0, x1;
  x_tile(g, blockIdx.x, band_lo_end(g.P, g.NX), band_hi_start(g.P, g.nx, g.NX), z0, x0, x1);
  const int xs = (x0 - 4) & ~3;
  for (int idx = threadIdx.x; idx < CX_TZ * CX_W; idx += CX_T) {
    const int r = idx / CX_W, j = idx - r * CX_W;
    const int z = z0 + r, x = xs + j;
    float C = 0.f, Bv = 0.f, G = 0.f;
    if (z < g.NZ && x >= 0 && x < g.NX && x_border(g, x)) {
      const long long c = so + (long long)z * g.NXp + x;
      const float b = __ldg(a.bx + x);
      const float m = a.u[c];
      C = b * (m + a.zeta[c]);
      Bv = b * a.pin[c];
      G = m + C;
    }
    sc[idx] = C;
    sb[idx] = Bv;
    sg[idx] = G;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < CX_TZ * CX_TX; idx += CX_T) {
    const int r = idx / CX_TX, cc = idx - r * CX_TX;
    const int z = z0 + r, x = x0 + cc;
    if (z >= g.NZ || x >= x1) continue;
    const int o = r * CX_W + (x - xs);
    const float* C = sc + o;
    const float* Bv = sb + o;
    const float* G = sg + o;
    const float corr = d2(C[-4], C[-3], C[-2], C[-1], C[0], C[1], C[2], C[3], C[4]) -
                       d1(Bv[-4], Bv[-3], Bv[-2], Bv[-1], Bv[1], Bv[2], Bv[3], Bv[4]);
    const long long c = (long long)z * g.NXp + x;
    a.un[so + c] += a.K[c] * corr;
    if (x_border(g, x)) {
      const float A = __ldg(a.ax + x);
      const float m = a.u[so + c];
      a.pout[so + c] = A * a.pin[so + c] - d1(G[-4], G[-3], G[-2], G[-1], G[1], G[2], G[3], G[4]);
      a.zout[so + c] = A * (m + a.zeta[so + c]);
    }
  }
}

}  // namespace

void launch_ac_corr_fwd(const AcCorrArgs& z, const AcCorrArgs& x, cudaStream_t st) {
  const Geom& g = z.g;
  if (g.P <= 0 || g.nshot <= 0) return;
  void* tok = profile_begin(SWEEP_K_AC_FWD_FR, st);
  dim3 gz((g.NX + CZ_T - 1) / CZ_T, 2 * ((g.P + CH - 1) / CH), g.nshot);
  ac_cz_fwd_kernel<<<gz, CZ_T, 0, st>>>(z);
  dim3 gx(x_band_tiles(g, g.P) + x_band_tiles(g, g.NX - (g.P + g.nx)), 1, g.nshot);
  ac_cx_fwd_kernel<<<gx, CX_T, 0, st>>>(x);
  profile_end(tok, st);
  note_launches(2);
}

void launch_ac_corr_bwd(const AcCorrArgs& z, const AcCorrArgs& x, cudaStream_t st) {
  const Geom& g = z.g;
  if (g.P <= 0 || g.nshot <= 0) return;
  void* tok = profile_begin(SWEEP_K_AC_BWD_FR, st);
  const int lo_end = band_lo_end(g.P, g.NZ), hi_start = band_hi_start(g.P, g.nz, g.NZ);
  dim3 gz((g.NX + CZ_T - 1) / CZ_T, (lo_end + CH - 1) / CH + (g.NZ - hi_start + CH - 1) / CH,
          g.nshot);
  ac_cz_bwd_kernel<<<gz, CZ_T, 0, st>>>(z);
  const int lw = band_lo_end(g.P, g.NX), r0 = band_hi_start(g.P, g.nx, g.NX);
  dim3 gx(x_band_tiles(g, lw) + x_band_tiles(g, g.NX - r0), 1, g.nshot);
  ac_cx_bwd_kernel<<<gx, CX_T, 0, st>>>(x);
  profile_end(tok, st);
  note_launches(2);
}

}  // namespace sweep
