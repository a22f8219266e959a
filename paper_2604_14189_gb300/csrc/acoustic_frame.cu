// Frame acoustic step kernels: every cell outside the interior kernels'
// rectangles (the absorbing border, plus the interior cells next to it),
// with the full convolutional-PML update, ring save/restore, and source and
// receiver handling.  See acoustic_common.cuh for the equations.
//
// A CTA owns a FR_TZ x FR_TX tile of one frame rectangle for one shot.  All
// neighbour data (wavefield with halo, PML memory variables with the halo
// along their own axis, and for the backward step the per-axis adjoint
// combinations G = (1+b) mu + b zetabar) is staged in shared memory first.
#include "acoustic_common.cuh"

namespace sweep {
namespace {

constexpr int FW = FR_TX + 8;
constexpr int FH = FR_TZ + 8;

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

// Stage rows [zs, zs+h) and columns [xs, xs+w) (xs, w multiples of 4) of
// one shot's field into t (row pitch w); zero outside the padded grid.
__device__ __forceinline__ void stage(float* t, const float* __restrict__ f, const Geom& g,
                                      int zs, int h, int xs, int w) {
  const int w4 = w / 4;
  for (int idx = threadIdx.x; idx < h * w4; idx += FR_THREADS) {
    const int r = idx / w4, c = idx - r * w4;
    const int gz = zs + r, gx = xs + 4 * c;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (gz >= 0 && gz < g.NZ && gx >= 0 && gx < g.NXp)
      v = *reinterpret_cast<const float4*>(f + (long long)gz * g.NXp + gx);
    *reinterpret_cast<float4*>(t + r * w + 4 * c) = v;
  }
}

__device__ __forceinline__ bool tile_has_xborder(const Geom& g, int xa, int xb) {
  // any column of [xa, xb) inside the x border strips (and the grid)?
  return (xa < g.P && xb > 0) || (xb > g.P + g.nx && xa < g.NX);
}
__device__ __forceinline__ bool tile_has_zborder(const Geom& g, int za, int zb) {
  return (za < g.P && zb > 0) || (zb > g.P + g.nz && za < g.NZ);
}

// ------------------------------------------------------------------ forward
__global__ void __launch_bounds__(FR_THREADS) ac_fr_fwd_kernel(const AcFrFwdArgs a) {
  __shared__ __align__(16) float su[FH * FW];
  __shared__ __align__(16) float spx[FR_TZ * FW];
  __shared__ __align__(16) float spz[FH * FR_TX];
  if (*a.status) return;
  const Geom& g = a.g;
  const int s = blockIdx.y;
  int z0, x0, z1, x1;
  frame_tile(a.fr, blockIdx.x, z0, x0, z1, x1);
  const long long so = (long long)s * g.fstride;
  const bool hx = tile_has_xborder(g, x0, x0 + FR_TX);
  const bool hz = tile_has_zborder(g, z0, z0 + FR_TZ);
  stage(su, a.u + so, g, z0 - 4, FH, x0 - 4, FW);
  if (hx) stage(spx, a.psx_in + so, g, z0, FR_TZ, x0 - 4, FW);
  if (hz) stage(spz, a.psz_in + so, g, z0 - 4, FH, x0, FR_TX);
  __syncthreads();
  const int sz = a.src[2 * s] + g.P, sx = a.src[2 * s + 1] + g.P;
  const float fn = a.wavelet[(long long)s * g.nt + a.n];
  const int cg = threadIdx.x & 15, rg = threadIdx.x >> 4;
  for (int rr = 0; rr < 2; ++rr) {
    const int r = 2 * rg + rr, gz = z0 + r;
    if (gz >= z1) continue;
#pragma unroll
    for (int cc4 = 0; cc4 < 4; ++cc4) {
      const int c = 4 * cg + cc4, gx = x0 + c;
      if (gx >= x1) continue;
      const float* row = su + (r + 4) * FW + (c + 4);
      float lapx = d2(row[-4], row[-3], row[-2], row[-1], row[0], row[1], row[2], row[3], row[4]);
      float lapz = d2(row[-4 * FW], row[-3 * FW], row[-2 * FW], row[-FW], row[0], row[FW],
                      row[2 * FW], row[3 * FW], row[4 * FW]);
      const long long ci = so + (long long)gz * g.NXp + gx;
      if (x_border(g, gx)) {
        const float* pr = spx + r * FW + (c + 4);
        const float dp = d1(pr[-4], pr[-3], pr[-2], pr[-1], pr[1], pr[2], pr[3], pr[4]);
        const float du = d1(row[-4], row[-3], row[-2], row[-1], row[1], row[2], row[3], row[4]);
        const float A = a.ax[gx], B = a.bx[gx];
        const float W = lapx + dp;
        const float zn = A * a.zex[ci] + B * W;
        a.psx_out[ci] = A * pr[0] + B * du;
        a.zex[ci] = zn;
        lapx = W + zn;
      }
      if (z_border(g, gz)) {
        const float* pc = spz + (r + 4) * FR_TX + c;
        const float dp = d1(pc[-4 * FR_TX], pc[-3 * FR_TX], pc[-2 * FR_TX], pc[-FR_TX],
                            pc[FR_TX], pc[2 * FR_TX], pc[3 * FR_TX], pc[4 * FR_TX]);
        const float du = d1(row[-4 * FW], row[-3 * FW], row[-2 * FW], row[-FW], row[FW],
                            row[2 * FW], row[3 * FW], row[4 * FW]);
        const float A = a.az[gz], B = a.bz[gz];
        const float W = lapz + dp;
        const float zn = A * a.zez[ci] + B * W;
        a.psz_out[ci] = A * pc[0] + B * du;
        a.zez[ci] = zn;
        lapz = W + zn;
      }
      const float kk = a.K[(long long)gz * g.NXp + gx];
      float v = 2.f * row[0] - a.un[ci] + kk * (lapx + lapz);
      if (gz == sz && gx == sx) v += kk * fn;
      a.un[ci] = v;
      if (a.save) {
        const int ri = ring_index(g, gz, gx);
        if (ri >= 0) a.save[(long long)s * g.nring + ri] = v;
      }
    }
  }
  if (a.data && tile_meets_box(a.rbox + 4 * s, z0, FR_TZ, x0, FR_TX)) {
    __syncthreads();
    for (int r = threadIdx.x; r < g.nrec; r += FR_THREADS) {
      const int32_t* q = a.rec + 2 * ((long long)s * g.nrec + r);
      const int rz = q[0] + g.P, rx = q[1] + g.P;
      if (rz >= z0 && rz < z1 && rx >= x0 && rx < x1)
        a.data[((long long)s * g.nrec + r) * g.nt + a.n] = a.un[so + (long long)rz * g.NXp + rx];
    }
  }
}

// ----------------------------------------------------------------- backward
__global__ void __launch_bounds__(FR_THREADS) ac_fr_bwd_kernel(const AcFrBwdArgs a) {
  __shared__ __align__(16) float sm[FH * FW];       // mu^{n+1}
  __shared__ __align__(16) float su[FH * FW];       // u^n
  __shared__ __align__(16) float gxs[FR_TZ * FW];   // G_x
  __shared__ __align__(16) float pxs[FR_TZ * FW];   // psibar_x (raw)
  __shared__ __align__(16) float gzs[FH * FR_TX];   // G_z
  __shared__ __align__(16) float pzs[FH * FR_TX];   // psibar_z (raw)
  __shared__ float bxs[FW];
  __shared__ float bzs[FH];
  if (*a.status) return;
  const Geom& g = a.g;
  const int s = blockIdx.y;
  int z0, x0, z1, x1;
  frame_tile(a.fr, blockIdx.x, z0, x0, z1, x1);
  const long long so = (long long)s * g.fstride;
  const bool adj = a.do_adj != 0, rec = a.do_rec != 0;
  const bool img = a.do_img && z1 > g.P && z0 < g.P + g.nz && x1 > g.P && x0 < g.P + g.nx;
  stage(sm, a.mA + so, g, z0 - 4, FH, x0 - 4, FW);
  if (img) stage(su, a.uA + so, g, z0 - 4, FH, x0 - 4, FW);
  for (int j = threadIdx.x; j < FW; j += FR_THREADS) {
    const int x = x0 - 4 + j;
    bxs[j] = (x >= 0 && x < g.NX) ? a.bx[x] : 0.f;
  }
  for (int i = threadIdx.x; i < FH; i += FR_THREADS) {
    const int z = z0 - 4 + i;
    bzs[i] = (z >= 0 && z < g.NZ) ? a.bz[z] : 0.f;
  }
  __syncthreads();
  if (adj) {
    // G and raw psibar along x on the tile rows, with the x halo
    for (int idx = threadIdx.x; idx < FR_TZ * FW; idx += FR_THREADS) {
      const int r = idx / FW, j = idx - r * FW;
      const int z = z0 + r, x = x0 - 4 + j;
      const float m1 = sm[(r + 4) * FW + j];
      const float b = bxs[j];
      float G = m1, pb = 0.f;
      if (b != 0.f && z < g.NZ) {
        const long long ci = so + (long long)z * g.NXp + x;
        G = m1 + b * (m1 + a.zbx_in[ci]);
        pb = a.pbx_in[ci];
      }
      gxs[idx] = G;
      pxs[idx] = pb;
    }
    // G and raw psibar along z on the tile columns, with the z halo
    for (int idx = threadIdx.x; idx < FH * FR_TX; idx += FR_THREADS) {
      const int i = idx / FR_TX, c = idx - i * FR_TX;
      const int z = z0 - 4 + i, x = x0 + c;
      const float m1 = sm[i * FW + c + 4];
      const float b = bzs[i];
      float G = m1, pb = 0.f;
      if (b != 0.f && x < g.NX) {
        const long long ci = so + (long long)z * g.NXp + x;
        G = m1 + b * (m1 + a.zbz_in[ci]);
        pb = a.pbz_in[ci];
      }
      gzs[idx] = G;
      pzs[idx] = pb;
    }
    __syncthreads();
  }
  const int sz = a.src[2 * s] + g.P, sx = a.src[2 * s + 1] + g.P;
  const float fn = a.do_img ? a.wavelet[(long long)s * g.nt + a.n] : 0.f;
  const int cg = threadIdx.x & 15, rg = threadIdx.x >> 4;
  for (int rr = 0; rr < 2; ++rr) {
    const int r = 2 * rg + rr, gz = z0 + r;
    if (gz >= z1) continue;
#pragma unroll
    for (int cc4 = 0; cc4 < 4; ++cc4) {
      const int c = 4 * cg + cc4, gx = x0 + c;
      if (gx >= x1) continue;
      const long long ci = so + (long long)gz * g.NXp + gx;
      const float m1 = sm[(r + 4) * FW + c + 4];
      const float kk = a.K[(long long)gz * g.NXp + gx];
      if (adj) {
        const float* G1 = gxs + r * FW + c + 4;
        const float* P1 = pxs + r * FW + c + 4;
        const float* B1 = bxs + c + 4;
        const float* G2 = gzs + (r + 4) * FR_TX + c;
        const float* P2 = pzs + (r + 4) * FR_TX + c;
        const float* B2 = bzs + r + 4;
        const int T = FR_TX;
        const float lx = d2(G1[-4], G1[-3], G1[-2], G1[-1], G1[0], G1[1], G1[2], G1[3], G1[4]);
        const float lz = d2(G2[-4 * T], G2[-3 * T], G2[-2 * T], G2[-T], G2[0], G2[T], G2[2 * T],
                            G2[3 * T], G2[4 * T]);
        const float px = d1(B1[-4] * P1[-4], B1[-3] * P1[-3], B1[-2] * P1[-2], B1[-1] * P1[-1],
                            B1[1] * P1[1], B1[2] * P1[2], B1[3] * P1[3], B1[4] * P1[4]);
        const float pz = d1(B2[-4] * P2[-4 * T], B2[-3] * P2[-3 * T], B2[-2] * P2[-2 * T],
                            B2[-1] * P2[-T], B2[1] * P2[T], B2[2] * P2[2 * T],
                            B2[3] * P2[3 * T], B2[4] * P2[4 * T]);
        a.mB[ci] = 2.f * m1 - a.mB[ci] + kk * (lx + lz - px - pz);
        if (x_border(g, gx)) {
          float mg[9];
#pragma unroll
          for (int t = 0; t < 9; ++t) {
            const int xx = gx - 4 + t;
            mg[t] = (xx >= 0 && xx < g.NX && x_border(g, xx)) ? G1[t - 4] : 0.f;
          }
          const float A = a.ax[gx];
          a.pbx_out[ci] = A * P1[0] - d1(mg[0], mg[1], mg[2], mg[3], mg[5], mg[6], mg[7], mg[8]);
          a.zbx_out[ci] = A * (m1 + a.zbx_in[ci]);
        }
        if (z_border(g, gz)) {
          float mg[9];
#pragma unroll
          for (int t = 0; t < 9; ++t) {
            const int zz = gz - 4 + t;
            mg[t] = (zz >= 0 && zz < g.NZ && z_border(g, zz)) ? G2[(t - 4) * T] : 0.f;
          }
          const float A = a.az[gz];
          a.pbz_out[ci] = A * P2[0] - d1(mg[0], mg[1], mg[2], mg[3], mg[5], mg[6], mg[7], mg[8]);
          a.zbz_out[ci] = A * (m1 + a.zbz_in[ci]);
        }
      }
      if (img && interior(g, gz, gx)) {
        const float* row = su + (r + 4) * FW + (c + 4);
        float lap = d2(row[-4], row[-3], row[-2], row[-1], row[0], row[1], row[2], row[3],
                       row[4]) +
                    d2(row[-4 * FW], row[-3 * FW], row[-2 * FW], row[-FW], row[0], row[FW],
                       row[2 * FW], row[3 * FW], row[4 * FW]);
        if (gz == sz && gx == sx) lap += fn;
        a.graw[ci] += m1 * lap;
        if (a.illum) a.illum[ci] += row[0] * row[0];
        if (rec) a.uB[ci] = 2.f * row[0] - a.uB[ci] + kk * lap;
      }
      if (rec && a.save) {
        const int ri = ring_index(g, gz, gx);
        if (ri >= 0) a.uB[ci] = a.save[(long long)s * g.nring + ri];
      }
    }
  }
  if (a.wgrad && a.n < g.nt && threadIdx.x == 0 && sz >= z0 && sz < z1 && sx >= x0 && sx < x1)
    a.wgrad[(long long)s * g.nt + a.n] = sm[(sz - z0 + 4) * FW + (sx - x0 + 4)];
  if (adj && a.n >= 1 && tile_meets_box(a.rbox + 4 * s, z0, FR_TZ, x0, FR_TX)) {
    __syncthreads();
    for (int r = threadIdx.x; r < g.nrec; r += FR_THREADS) {
      const int32_t* q = a.rec + 2 * ((long long)s * g.nrec + r);
      const int rz = q[0] + g.P, rx = q[1] + g.P;
      if (rz >= z0 && rz < z1 && rx >= x0 && rx < x1) {
        const float rv = a.res[((long long)s * g.nrec + r) * g.nt + (a.n - 1)];
        atomicAdd(a.mB + so + (long long)rz * g.NXp + rx, a.K[(long long)rz * g.NXp + rx] * rv);
      }
    }
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
  const int tiles = a.fr.first[a.fr.n];
  if (tiles <= 0 || a.g.nshot <= 0) return;
  dim3 grid(tiles, a.g.nshot);
  ac_fr_fwd_kernel<<<grid, FR_THREADS, 0, st>>>(a);
  note_launches(1);
}

void launch_ac_fr_bwd(const AcFrBwdArgs& a, cudaStream_t st) {
  const int tiles = a.fr.first[a.fr.n];
  if (tiles <= 0 || a.g.nshot <= 0) return;
  dim3 grid(tiles, a.g.nshot);
  ac_fr_bwd_kernel<<<grid, FR_THREADS, 0, st>>>(a);
  note_launches(1);
}

}  // namespace sweep
