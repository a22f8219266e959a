// Acoustic step kernels for sm_103a: the fused forward step and the fused
// backward step (adjoint propagation + wavefield reconstruction + imaging).
//
// Scheme (Sec. 3.1.2, Eq. 2, in the update form of the Sec. 2.1 listing):
//   u^{n+1} = 2 u^n - u^{n-1} + K (Lx + Lz) + K f^n delta_s,  K = v^2 dt^2/dx^2
// with, per axis, L = D2 u^n away from the border and, inside the border,
//   W = D2 u^n + D1 psi^{n-1};  zeta^n = a zeta^{n-1} + b W;
//   psi^n = a psi^{n-1} + b D1 u^n;  L = W + zeta^n.
// D2, D1: 8th-order centred differences (unit spacing; 1/dx^2 is in K).
//
// Backward step n (exact transpose, written for mu = K lambda):
//   G  = (1 + b) mu^{n+1} + b zetabar^n          per axis, per cell
//   mu^n = 2 mu^{n+1} - mu^{n+2} + K sum_axes [D2 G - D1 (b psibar^n)]
//          + K R^T r^{n-1}
//   psibar^{n-1} = a psibar^n - D1 (m G)    (m = 1 inside that axis' border)
//   zetabar^{n-1} = a (mu^{n+1} + zetabar^n)
// Away from the border (and 4 cells into it) this reduces to the forward
// update itself.  Imaging (interior cells):
//   graw += mu^{n+1} (D2x u^n + D2z u^n + f^n delta_s)
// and the interior wavefield runs backwards,
//   u^{n-1} = 2 u^n - u^{n+1} + K (Lap u^n + f^n delta_s),
// with the 4-cell ring around the interior restored from the forward save.
//
// Each CTA owns a 32 x 128 tile of one shot: the tile of u^n (or mu^{n+1})
// plus a 4-cell halo is staged in shared memory; a warp covers the tile width
// (4 cells per lane, float4 accesses), and walks 8 rows keeping a 9-row
// register window for the z stencil.
#include "sweep_internal.cuh"

namespace sweep {
namespace {

constexpr float kC0 = -205.0f / 72.0f;
constexpr float kC1 = 8.0f / 5.0f;
constexpr float kC2 = -1.0f / 5.0f;
constexpr float kC3 = 8.0f / 315.0f;
constexpr float kC4 = -1.0f / 560.0f;
constexpr float kD1 = 4.0f / 5.0f;
constexpr float kD2 = -1.0f / 5.0f;
constexpr float kD3 = 4.0f / 105.0f;
constexpr float kD4 = -1.0f / 280.0f;

constexpr int SW = AC_BX + 8;      // shared row pitch (floats)
constexpr int SROWS = AC_BZ + 8;   // shared rows

__device__ __forceinline__ float4 lds4(const float* t, int r, int c) {
  return *reinterpret_cast<const float4*>(t + r * SW + c);
}

__device__ __forceinline__ void f4a(const float4 v, float* o) {
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}

// Stage rows z0-4 .. z0+BZ+3, columns x0-4 .. x0+BX+3 of field f (one shot,
// [NZ][NXp]) into shared memory; zero outside the padded grid.
__device__ __forceinline__ void load_tile(float* tile, const float* __restrict__ f,
                                          const Geom& g, int z0, int x0) {
  constexpr int C4 = SW / 4;
  for (int idx = threadIdx.x; idx < SROWS * C4; idx += AC_THREADS) {
    const int r = idx / C4, c = idx - r * C4;
    const int gz = z0 - 4 + r, gx = x0 - 4 + 4 * c;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (gz >= 0 && gz < g.NZ && gx >= 0 && gx < g.NXp)
      v = __ldg(reinterpret_cast<const float4*>(f + (long long)gz * g.NXp + gx));
    *reinterpret_cast<float4*>(tile + r * SW + 4 * c) = v;
  }
}

// 8th-order second difference at e[4] of a 9-sample window
__device__ __forceinline__ float d2(float m4, float m3, float m2, float m1, float c,
                                    float p1, float p2, float p3, float p4) {
  return kC0 * c + kC1 * (p1 + m1) + kC2 * (p2 + m2) + kC3 * (p3 + m3) + kC4 * (p4 + m4);
}
__device__ __forceinline__ float d1(float m4, float m3, float m2, float m1,
                                    float p1, float p2, float p3, float p4) {
  return kD1 * (p1 - m1) + kD2 * (p2 - m2) + kD3 * (p3 - m3) + kD4 * (p4 - m4);
}

__device__ __forceinline__ float ld0(const float* __restrict__ f, const Geom& g, int z, int x) {
  return (z >= 0 && z < g.NZ && x >= 0 && x < g.NX) ? f[(long long)z * g.NXp + x] : 0.f;
}

// Index of padded cell (z, x) in the saved ring around the interior, or -1.
__device__ __forceinline__ int ring_index(const Geom& g, int z, int x) {
  const int w = g.ringw, P = g.P;
  if (w == 0) return -1;
  const int zi = z - P, xi = x - P;  // interior coordinates
  if (zi < -w || zi >= g.nz + w || xi < -w || xi >= g.nx + w) return -1;
  const int W = g.nx + 2 * w;
  if (zi < 0) return (zi + w) * W + (xi + w);
  if (zi >= g.nz) return w * W + (zi - g.nz) * W + (xi + w);
  if (xi < 0) return 2 * w * W + zi * w + (xi + w);
  if (xi >= g.nx) return 2 * w * W + g.nz * w + zi * w + (xi - g.nx);
  return -1;  // interior
}

// ------------------------------------------------------------------ forward
__global__ void __launch_bounds__(AC_THREADS) ac_fwd_kernel(const AcFwdArgs a) {
  __shared__ __align__(16) float tile[SROWS * SW];
  if (*a.status) return;
  const Geom& g = a.g;
  const int s = blockIdx.z;
  const int x0 = blockIdx.x * AC_BX, z0 = blockIdx.y * AC_BZ;
  const long long so = (long long)s * g.fstride;
  load_tile(tile, a.u + so, g, z0, x0);
  __syncthreads();

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lx = 4 * lane, gx = x0 + lx, r0 = warp * AC_RPW;
  const int P = g.P;
  const bool pure = x0 >= P && x0 + AC_BX <= P + g.nx && z0 >= P && z0 + AC_BZ <= P + g.nz;
  const int sz = a.src[2 * s] + P, sx = a.src[2 * s + 1] + P;
  const float fn = a.wavelet[(long long)s * g.nt + a.n];

  float w[9][4];
#pragma unroll
  for (int k = 0; k < 8; ++k) f4a(lds4(tile, r0 + k, lx + 4), w[k]);
#pragma unroll
  for (int q = 0; q < AC_RPW; ++q) {
    f4a(lds4(tile, r0 + q + 8, lx + 4), w[8]);
    float e[12];
    f4a(lds4(tile, r0 + q + 4, lx), e);
    f4a(lds4(tile, r0 + q + 4, lx + 4), e + 4);
    f4a(lds4(tile, r0 + q + 4, lx + 8), e + 8);
    const int gz = z0 + r0 + q;
    if (gz < g.NZ && gx < g.NXp) {
      const long long ci = so + (long long)gz * g.NXp + gx;
      float4 upv = *reinterpret_cast<const float4*>(a.un + ci);
      float4 kv = __ldg(reinterpret_cast<const float4*>(a.K + (long long)gz * g.NXp + gx));
      float up[4], kk[4], out[4];
      f4a(upv, up);
      f4a(kv, kk);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int gxc = gx + c;
        float lxx = d2(e[c], e[c + 1], e[c + 2], e[c + 3], e[c + 4], e[c + 5], e[c + 6],
                       e[c + 7], e[c + 8]);
        float lzz = d2(w[0][c], w[1][c], w[2][c], w[3][c], w[4][c], w[5][c], w[6][c],
                       w[7][c], w[8][c]);
        if (!pure && gxc < g.NX) {
          const long long cc = ci + c;
          if (gxc < P || gxc >= P + g.nx) {
            const float* ps = a.psx_in + so;
            const float dp = d1(ld0(ps, g, gz, gxc - 4), ld0(ps, g, gz, gxc - 3),
                                ld0(ps, g, gz, gxc - 2), ld0(ps, g, gz, gxc - 1),
                                ld0(ps, g, gz, gxc + 1), ld0(ps, g, gz, gxc + 2),
                                ld0(ps, g, gz, gxc + 3), ld0(ps, g, gz, gxc + 4));
            const float du = d1(e[c], e[c + 1], e[c + 2], e[c + 3], e[c + 5], e[c + 6],
                                e[c + 7], e[c + 8]);
            const float A = __ldg(a.ax + gxc), B = __ldg(a.bx + gxc);
            const float W = lxx + dp;
            const float zn = A * a.zex[cc] + B * W;
            a.psx_out[cc] = A * a.psx_in[cc] + B * du;
            a.zex[cc] = zn;
            lxx = W + zn;
          }
          if (gz < P || gz >= P + g.nz) {
            const float* ps = a.psz_in + so;
            const float dp = d1(ld0(ps, g, gz - 4, gxc), ld0(ps, g, gz - 3, gxc),
                                ld0(ps, g, gz - 2, gxc), ld0(ps, g, gz - 1, gxc),
                                ld0(ps, g, gz + 1, gxc), ld0(ps, g, gz + 2, gxc),
                                ld0(ps, g, gz + 3, gxc), ld0(ps, g, gz + 4, gxc));
            const float du = d1(w[0][c], w[1][c], w[2][c], w[3][c], w[5][c], w[6][c],
                                w[7][c], w[8][c]);
            const float A = __ldg(a.az + gz), B = __ldg(a.bz + gz);
            const float W = lzz + dp;
            const float zn = A * a.zez[cc] + B * W;
            a.psz_out[cc] = A * a.psz_in[cc] + B * du;
            a.zez[cc] = zn;
            lzz = W + zn;
          }
        }
        float v = 2.f * w[4][c] - up[c] + kk[c] * (lxx + lzz);
        if (gz == sz && gxc == sx) v += kk[c] * fn;
        out[c] = gxc < g.NX ? v : 0.f;
        if (a.save) {
          const int ri = ring_index(g, gz, gxc);
          if (ri >= 0) a.save[(long long)s * g.nring + ri] = out[c];
        }
      }
      *reinterpret_cast<float4*>(a.un + ci) = make_float4(out[0], out[1], out[2], out[3]);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
#pragma unroll
      for (int c = 0; c < 4; ++c) w[k][c] = w[k + 1][c];
    }
  }
  if (a.data) {
    __syncthreads();  // this CTA's stores of u^{n+1} are visible below
    const float* un = a.un + so;
    for (int r = threadIdx.x; r < g.nrec; r += AC_THREADS) {
      const int32_t* q = a.rec + 2 * ((long long)s * g.nrec + r);
      const int rz = q[0] + P, rx = q[1] + P;
      if (rz >= z0 && rz < z0 + AC_BZ && rx >= x0 && rx < x0 + AC_BX)
        a.data[((long long)s * g.nrec + r) * g.nt + a.n] = un[(long long)rz * g.NXp + rx];
    }
  }
}

// ------------------------------------------------------------------ backward
// General (border-affected) adjoint update of one cell.  em: 12 mu^{n+1}
// samples of the row (centre at em[c+4]); wm: 9-row window (centre wm[4][c]).
__device__ __forceinline__ float adj_border_cell(const AcBwdArgs& a, long long so, int gz,
                                                 int gxc, const float* em,
                                                 const float (*wm)[4], int c, float m2,
                                                 float kk) {
  const Geom& g = a.g;
  const int P = g.P;
  const long long rowx = so + (long long)gz * g.NXp;
  float Gx[9], Bx[9], Gz[9], Bz[9];
  float mxG[9], mzG[9];
#pragma unroll
  for (int t = 0; t < 9; ++t) {
    const int jj = gxc - 4 + t;
    const float m = em[c + t];
    float gv = m, bv = 0.f, mg = 0.f;
    if (jj >= 0 && jj < g.NX && (jj < P || jj >= P + g.nx)) {
      const float B = __ldg(a.bx + jj);
      gv = m + B * (m + a.zbx_in[rowx + jj]);
      bv = B * a.pbx_in[rowx + jj];
      mg = gv;
    }
    Gx[t] = gv; Bx[t] = bv; mxG[t] = mg;
    const int ii = gz - 4 + t;
    const float mz = wm[t][c];
    float gzv = mz, bzv = 0.f, mgz = 0.f;
    if (ii >= 0 && ii < g.NZ && (ii < P || ii >= P + g.nz)) {
      const long long ro = so + (long long)ii * g.NXp + gxc;
      const float B = __ldg(a.bz + ii);
      gzv = mz + B * (mz + a.zbz_in[ro]);
      bzv = B * a.pbz_in[ro];
      mgz = gzv;
    }
    Gz[t] = gzv; Bz[t] = bzv; mzG[t] = mgz;
  }
  const float lam = d2(Gx[0], Gx[1], Gx[2], Gx[3], Gx[4], Gx[5], Gx[6], Gx[7], Gx[8]) +
                    d2(Gz[0], Gz[1], Gz[2], Gz[3], Gz[4], Gz[5], Gz[6], Gz[7], Gz[8]) -
                    d1(Bx[0], Bx[1], Bx[2], Bx[3], Bx[5], Bx[6], Bx[7], Bx[8]) -
                    d1(Bz[0], Bz[1], Bz[2], Bz[3], Bz[5], Bz[6], Bz[7], Bz[8]);
  const float m1 = em[c + 4];
  const long long cc = rowx + gxc;
  if (gxc < P || gxc >= P + g.nx) {
    const float A = __ldg(a.ax + gxc);
    a.pbx_out[cc] = A * a.pbx_in[cc] -
                    d1(mxG[0], mxG[1], mxG[2], mxG[3], mxG[5], mxG[6], mxG[7], mxG[8]);
    a.zbx_out[cc] = A * (m1 + a.zbx_in[cc]);
  }
  if (gz < P || gz >= P + g.nz) {
    const float A = __ldg(a.az + gz);
    a.pbz_out[cc] = A * a.pbz_in[cc] -
                    d1(mzG[0], mzG[1], mzG[2], mzG[3], mzG[5], mzG[6], mzG[7], mzG[8]);
    a.zbz_out[cc] = A * (m1 + a.zbz_in[cc]);
  }
  return 2.f * m1 - m2 + kk * lam;
}

__global__ void __launch_bounds__(AC_THREADS) ac_bwd_kernel(const AcBwdArgs a) {
  __shared__ __align__(16) float tm[SROWS * SW];  // mu^{n+1}
  __shared__ __align__(16) float tu[SROWS * SW];  // u^n
  if (*a.status) return;
  const Geom& g = a.g;
  const int s = blockIdx.z;
  const int x0 = blockIdx.x * AC_BX, z0 = blockIdx.y * AC_BZ;
  const long long so = (long long)s * g.fstride;
  const int P = g.P;
  // does the tile hold interior cells (imaging / reconstruction)?
  const bool has_int = x0 + AC_BX > P && x0 < P + g.nx && z0 + AC_BZ > P && z0 < P + g.nz;
  const bool img = a.do_img && has_int;
  load_tile(tm, a.mA + so, g, z0, x0);
  if (img) load_tile(tu, a.uA + so, g, z0, x0);
  __syncthreads();

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lx = 4 * lane, gx = x0 + lx, r0 = warp * AC_RPW;
  const bool pure = x0 - 4 >= P && x0 + AC_BX + 4 <= P + g.nx && z0 - 4 >= P &&
                    z0 + AC_BZ + 4 <= P + g.nz;
  const int sz = a.src[2 * s] + P, sx = a.src[2 * s + 1] + P;
  const float fn = a.do_img ? a.wavelet[(long long)s * g.nt + a.n] : 0.f;

  float wm[9][4], wu[9][4];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    f4a(lds4(tm, r0 + k, lx + 4), wm[k]);
    if (img) f4a(lds4(tu, r0 + k, lx + 4), wu[k]);
  }
#pragma unroll
  for (int q = 0; q < AC_RPW; ++q) {
    f4a(lds4(tm, r0 + q + 8, lx + 4), wm[8]);
    if (img) f4a(lds4(tu, r0 + q + 8, lx + 4), wu[8]);
    const int gz = z0 + r0 + q;
    if (gz < g.NZ && gx < g.NXp) {
      const long long ci = so + (long long)gz * g.NXp + gx;
      float kk[4];
      f4a(__ldg(reinterpret_cast<const float4*>(a.K + (long long)gz * g.NXp + gx)), kk);
      float em[12];
      f4a(lds4(tm, r0 + q + 4, lx), em);
      f4a(lds4(tm, r0 + q + 4, lx + 4), em + 4);
      f4a(lds4(tm, r0 + q + 4, lx + 8), em + 8);
      if (a.do_adj) {
        float m2[4], out[4];
        f4a(*reinterpret_cast<const float4*>(a.mB + ci), m2);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int gxc = gx + c;
          float v;
          if (pure) {
            const float lap =
                d2(em[c], em[c + 1], em[c + 2], em[c + 3], em[c + 4], em[c + 5], em[c + 6],
                   em[c + 7], em[c + 8]) +
                d2(wm[0][c], wm[1][c], wm[2][c], wm[3][c], wm[4][c], wm[5][c], wm[6][c],
                   wm[7][c], wm[8][c]);
            v = 2.f * em[c + 4] - m2[c] + kk[c] * lap;
          } else if (gxc < g.NX) {
            v = adj_border_cell(a, so, gz, gxc, em, wm, c, m2[c], kk[c]);
          } else {
            v = 0.f;
          }
          out[c] = gxc < g.NX ? v : 0.f;
        }
        *reinterpret_cast<float4*>(a.mB + ci) = make_float4(out[0], out[1], out[2], out[3]);
      }
      if (img && gz >= P && gz < P + g.nz) {
        float eu[12];
        f4a(lds4(tu, r0 + q + 4, lx), eu);
        f4a(lds4(tu, r0 + q + 4, lx + 4), eu + 4);
        f4a(lds4(tu, r0 + q + 4, lx + 8), eu + 8);
        float u1[4];
        if (a.do_rec) f4a(*reinterpret_cast<const float4*>(a.uB + ci), u1);
        const long long gi = ((long long)s * g.nz + (gz - P)) * g.nx - P;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int gxc = gx + c;
          if (gxc >= P && gxc < P + g.nx) {
            float lap = d2(eu[c], eu[c + 1], eu[c + 2], eu[c + 3], eu[c + 4], eu[c + 5],
                           eu[c + 6], eu[c + 7], eu[c + 8]) +
                        d2(wu[0][c], wu[1][c], wu[2][c], wu[3][c], wu[4][c], wu[5][c],
                           wu[6][c], wu[7][c], wu[8][c]);
            if (gz == sz && gxc == sx) lap += fn;
            a.graw[gi + gxc] += em[c + 4] * lap;
            if (a.illum) a.illum[gi + gxc] += wu[4][c] * wu[4][c];
            if (a.do_rec) a.uB[ci + c] = 2.f * wu[4][c] - u1[c] + kk[c] * lap;
          }
        }
      }
      if (a.do_rec && a.save) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int ri = ring_index(g, gz, gx + c);
          if (ri >= 0) a.uB[ci + c] = a.save[(long long)s * g.nring + ri];
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        wm[k][c] = wm[k + 1][c];
        wu[k][c] = wu[k + 1][c];
      }
    }
  }
  if (a.wgrad && a.n < g.nt) {
    if (threadIdx.x == 0 && sz >= z0 && sz < z0 + AC_BZ && sx >= x0 && sx < x0 + AC_BX)
      a.wgrad[(long long)s * g.nt + a.n] = tm[(sz - z0 + 4) * SW + (sx - x0 + 4)];
  }
  if (a.do_adj && a.n >= 1) {
    __syncthreads();  // this CTA's stores of mu^n precede the injections
    for (int r = threadIdx.x; r < g.nrec; r += AC_THREADS) {
      const int32_t* q = a.rec + 2 * ((long long)s * g.nrec + r);
      const int rz = q[0] + P, rx = q[1] + P;
      if (rz >= z0 && rz < z0 + AC_BZ && rx >= x0 && rx < x0 + AC_BX) {
        const float rv = a.res[((long long)s * g.nrec + r) * g.nt + (a.n - 1)];
        atomicAdd(a.mB + so + (long long)rz * g.NXp + rx,
                  __ldg(a.K + (long long)rz * g.NXp + rx) * rv);
      }
    }
  }
}

}  // namespace

void launch_ac_fwd(const AcFwdArgs& a, cudaStream_t st) {
  const Geom& g = a.g;
  dim3 grid((g.NXp + AC_BX - 1) / AC_BX, (g.NZ + AC_BZ - 1) / AC_BZ, g.nshot);
  void* tok = profile_begin(SWEEP_K_AC_FWD, st);
  ac_fwd_kernel<<<grid, AC_THREADS, 0, st>>>(a);
  profile_end(tok, st);
}

void launch_ac_bwd(const AcBwdArgs& a, cudaStream_t st) {
  const Geom& g = a.g;
  dim3 grid((g.NXp + AC_BX - 1) / AC_BX, (g.NZ + AC_BZ - 1) / AC_BZ, g.nshot);
  void* tok = profile_begin(SWEEP_K_AC_BWD, st);
  ac_bwd_kernel<<<grid, AC_THREADS, 0, st>>>(a);
  profile_end(tok, st);
}

}  // namespace sweep
