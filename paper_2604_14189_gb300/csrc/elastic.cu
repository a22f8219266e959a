// Elastic velocity-stress kernels (Sec. 3.5, Eq. 12) on a staggered grid.
//
// Cell (i, j) = (z, x): txx, tzz at (i, j); vx at (i, j+1/2); vz at
// (i+1/2, j); txz at (i+1/2, j+1/2).  4th-order staggered differences,
// D F = S1 (F(+1/2) - F(-1/2)) + S2 (F(+3/2) - F(-3/2)), S1 = 9/8,
// S2 = -1/24, at unit spacing; 1/dx is folded into the coefficients.
// One time step n:
//   velocity  v^{n+1/2} = v^{n-1/2} + (dt b / dx) (div tau^n)
//   stress    tau^{n+1} = tau^n + (dt / dx) C (grad v^{n+1/2})
//             txx(s), tzz(s) += dt f^n / dx^2; trace sample n = v^{n+1/2}
// Convolutional PML: each derivative d at a point with profile (a, b)
// (integer or half-cell position along its axis) becomes d + psi with
// psi = a psi + b d.  Buoyancy at a velocity point: inverse of the mean of
// the two neighbouring densities; mu at a txz point: harmonic mean of the
// four neighbours (0 if any is 0); neighbours past the grid edge are clamped.
//
// Persistent TMA-pipelined kernels (see the tile section below); the TMA
// zero-fills outside the padded grid (the Dirichlet condition).
#include <algorithm>

#include "elastic_internal.cuh"
#include "tma.cuh"

namespace sweep {
namespace {

constexpr float kS1 = 9.0f / 8.0f;
constexpr float kS2 = -1.0f / 24.0f;

// ------------------------------------------------------------- parameters
__device__ __forceinline__ float mpar(const float* model, const Geom& g, int padded, int par,
                                      int z, int x) {
  z = min(max(z, 0), g.NZ - 1);
  x = min(max(x, 0), g.NX - 1);
  if (padded) return model[((long long)par * g.NZ + z) * g.NX + x];
  const int zi = min(max(z - g.P, 0), g.nz - 1), xi = min(max(x - g.P, 0), g.nx - 1);
  return model[((long long)par * g.nz + zi) * g.nx + xi];
}

__global__ void el_params_kernel(const ElParamArgs a) {
  const Geom& g = a.g;
  const long long n = (long long)g.NZ * g.NXp;
  const double sc = (double)a.dt / a.dx;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int z = (int)(i / g.NXp), x = (int)(i - (long long)z * g.NXp);
    float bx = 0.f, bz = 0.f, l2m = 0.f, lam = 0.f, mxz = 0.f;
    if (x < g.NX) {
      const double vp = mpar(a.model, g, a.padded, 0, z, x);
      const double vs = mpar(a.model, g, a.padded, 1, z, x);
      const double rho = mpar(a.model, g, a.padded, 2, z, x);
      const double rx = mpar(a.model, g, a.padded, 2, z, x + 1);
      const double rz = mpar(a.model, g, a.padded, 2, z + 1, x);
      const double la = rho * (vp * vp - 2.0 * vs * vs), mu = rho * vs * vs;
      auto muat = [&](int zz, int xx) {
        const double v = mpar(a.model, g, a.padded, 1, zz, xx);
        return mpar(a.model, g, a.padded, 2, zz, xx) * v * v;
      };
      const double m01 = muat(z, x + 1), m10 = muat(z + 1, x), m11 = muat(z + 1, x + 1);
      const double mh = (mu == 0.0 || m01 == 0.0 || m10 == 0.0 || m11 == 0.0)
                            ? 0.0
                            : 4.0 / (1.0 / mu + 1.0 / m01 + 1.0 / m10 + 1.0 / m11);
      bx = (float)(sc * 2.0 / (rho + rx));
      bz = (float)(sc * 2.0 / (rho + rz));
      l2m = (float)(sc * (la + 2.0 * mu));
      lam = (float)(sc * la);
      mxz = (float)(sc * mh);
    }
    a.cbx[i] = bx;
    a.cbz[i] = bz;
    a.cl2m[i] = l2m;
    a.clam[i] = lam;
    a.cmu[i] = mxz;
  }
}

// ------------------------------------------------------------------ tiles
// Persistent CTAs (one per SM) take (tile, shot) units round-robin; tiles are
// TB_Z rows x TB_X cells, a warp owns E_RPW rows, a lane 4 consecutive
// cells.  Shape, threads and stages chosen by a sweep on GB300 (500x1500+40,
// 64 shots): 16 rows x 3 stages x 256 threads 72.0 Gpts/s, 16 x 4 x 256 68.1,
// 16 x 3 x 512 76.7, 24 x 3 x 256 70.6, 32 x 2 x 256 80.4, 48 x 1 x 256 83.2,
// 32 x 2 x 512 83.5 (taller tiles read fewer halo rows per output row; 48 and
// 64 rows spill at 512 threads).  The fields each kernel differentiates (and the coefficients) are
// staged by a TMA pipeline of E_STAGES stages; the fields it updates in place
// and the CPML memory variables (read only on tiles that meet a border
// strip) are read with 16-byte loads issued before the stage wait.
constexpr int TB_X = 128;
constexpr int TB_Z = 32;
constexpr int E_THREADS = 512;
constexpr int E_RPW = TB_Z / (E_THREADS / 32);  // rows per warp
constexpr int E_HW = TB_X + 8;                  // x-halo width
constexpr int E_HZ = TB_Z + 8;                  // z-halo height
constexpr int E_STAGES = 2;
constexpr int E_TABLE = 256;                    // unit descriptors per CTA

struct __align__(128) VelStage {
  float txx[TB_Z * E_HW];  // x halo
  float txz[E_HZ * E_HW];  // x and z halos
  float tzz[E_HZ * TB_X];  // z halo
  float cbx[TB_Z * TB_X];
  float cbz[TB_Z * TB_X];
};
struct __align__(128) StrStage {
  float vx[E_HZ * E_HW];
  float vz[E_HZ * E_HW];
  float l2m[TB_Z * TB_X];
  float lam[TB_Z * TB_X];
  float mu[TB_Z * TB_X];
};
static_assert(sizeof(VelStage) % 128 == 0 && sizeof(StrStage) % 128 == 0, "stage alignment");
constexpr uint32_t kVelBytes = (TB_Z * E_HW + E_HZ * E_HW + E_HZ * TB_X + 2 * TB_Z * TB_X) * 4;
constexpr uint32_t kStrBytes = (2 * E_HZ * E_HW + 3 * TB_Z * TB_X) * 4;
static_assert(kVelBytes == sizeof(VelStage) && kStrBytes == sizeof(StrStage), "stage bytes");
constexpr size_t kVelSmem = E_STAGES * sizeof(VelStage) + 8 * E_STAGES;
constexpr size_t kStrSmem = E_STAGES * sizeof(StrStage) + 8 * E_STAGES;

enum : int { EU_XS = 1, EU_ZS = 2, EU_SRC = 4 };
struct EUnit {
  int s, z0, x0, flags;
  int sz, sx;
  float amp;  // source sample of this step (dt/dx^2 f^n)
  int pad;
};

__device__ __forceinline__ EUnit e_unit(const ElStepArgs& a, int unit) {
  const Geom& g = a.g;
  const int tile = unit / g.nshot;
  EUnit u;
  u.s = unit - tile * g.nshot;
  const int tz = tile / a.ntx;
  u.z0 = tz * TB_Z;
  u.x0 = (tile - tz * a.ntx) * TB_X;
  u.sz = a.src[2 * u.s] + g.P;
  u.sx = a.src[2 * u.s + 1] + g.P;
  u.amp = a.wavelet[(size_t)u.s * g.nt + a.n] * a.src_scale;
  u.pad = 0;
  int f = 0;
  // CPML columns / rows: an integer or half-point profile is nonzero there
  if (g.P > 0 && (u.x0 < g.P || u.x0 + TB_X > g.P + g.nx - 1)) f |= EU_XS;
  if (g.P > 0 && (u.z0 < g.P || u.z0 + TB_Z > g.P + g.nz - 1)) f |= EU_ZS;
  if (u.sz >= u.z0 && u.sz < u.z0 + TB_Z && u.sx >= u.x0 && u.sx < u.x0 + TB_X) f |= EU_SRC;
  u.flags = f;
  return u;
}

__device__ __forceinline__ float4 lds4e(const float* t, int pitch, int r, int c) {
  return *reinterpret_cast<const float4*>(t + r * pitch + c);
}
__device__ __forceinline__ void f4(const float4 v, float* o) {
  o[0] = v.x;
  o[1] = v.y;
  o[2] = v.z;
  o[3] = v.w;
}
__device__ __forceinline__ float4 ldg4z(const float* p, bool ok) {
  return ok ? *reinterpret_cast<const float4*>(p) : make_float4(0.f, 0.f, 0.f, 0.f);
}
__device__ __forceinline__ void stg4(float* p, const float* v) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

// The persistent pipeline shared by both kernels: prologue (descriptor table,
// barriers, first stages) and the bounded wait of each unit.
template <typename Stage, typename Issue, typename Body>
__device__ __forceinline__ void e_pipeline(const ElStepArgs& a, unsigned char* smem_raw,
                                           EUnit* tab, EUnit* ring, Issue issue, Body body) {
  constexpr int D = E_STAGES;
  Stage* stg = reinterpret_cast<Stage*>(smem_raw);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + D * sizeof(Stage));
  const int G = gridDim.x;
  const int count = (a.units - (int)blockIdx.x + G - 1) / G;
  if (count <= 0) return;
  for (int i = threadIdx.x; i < count && i < E_TABLE; i += E_THREADS)
    tab[i] = e_unit(a, blockIdx.x + i * G);
  if (threadIdx.x == 0) {
    for (int i = 0; i < D; ++i) mbar_init(&bar[i], 1);
    fence_barrier_init();
  }
  __syncthreads();
  auto desc = [&](int k) {
    if (k < E_TABLE) return tab[k];
    const EUnit u = e_unit(a, blockIdx.x + k * G);
    ring[k % D] = u;
    return u;
  };
  if (threadIdx.x == 0)
    for (int k = 0; k < D && k < count; ++k) issue(stg[k], &bar[k], desc(k));
  __syncthreads();  // descriptors of the first units visible to all threads
  int k = 0;
  for (; k < count; ++k) {
    if (k == count - 1) grid_dep_trigger();  // the next kernel may start
    const EUnit u = k < E_TABLE ? tab[k] : ring[k % D];
    const bool ok = body(u, stg[k % D], [&]() {
      const bool got = mbar_wait(&bar[k % D], (k / D) & 1);
      return !__syncthreads_or(!got);
    });
    if (!ok) break;   // uniform: a transfer never landed
    __syncthreads();  // stage released
    if (threadIdx.x == 0 && k + D < count) {
      fence_proxy_async_smem();
      issue(stg[k % D], &bar[k % D], desc(k + D));
    }
  }
  if (k < count && threadIdx.x == 0) {
    // report, and drain the transfers still in flight (bounded waits)
    latch(a.status, SWEEP_ETIMEOUT);
    for (int j = k; j < count && j < k + D; ++j) mbar_wait(&bar[j % D], (j / D) & 1);
  }
}

// ------------------------------------------------------------- velocity
__global__ void __launch_bounds__(E_THREADS, 1) el_vel_kernel(const __grid_constant__ ElStepArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ EUnit tab[E_TABLE];
  __shared__ EUnit ring[E_STAGES];
  grid_dep_wait();
  if (*a.status) return;
  const Geom& g = a.g;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lx = 4 * lane, r0 = warp * E_RPW;
  auto issue = [&](VelStage& sg, uint64_t* b, const EUnit& u) {
    mbar_arrive_expect_tx(b, kVelBytes);
    tma_load_3d(sg.txx, &a.m_txx, b, u.x0 - 4, u.z0, u.s);
    tma_load_3d(sg.txz, &a.m_txz, b, u.x0 - 4, u.z0 - 4, u.s);
    tma_load_3d(sg.tzz, &a.m_tzz, b, u.x0, u.z0 - 4, u.s);
    tma_load_2d(sg.cbx, &a.m_cbx, b, u.x0, u.z0);
    tma_load_2d(sg.cbz, &a.m_cbz, b, u.x0, u.z0);
  };
  auto body = [&](const EUnit& u, const VelStage& sg, auto wait) {
    const int gx = u.x0 + lx;
    const bool colok = gx < g.NXp;
    const size_t so = (size_t)u.s * g.fstride;
    // fields updated in place (and memory variables on strip tiles)
    float vx[E_RPW][4], vz[E_RPW][4], p1[E_RPW][4], p2[E_RPW][4], p3[E_RPW][4], p4[E_RPW][4];
    const bool xs = u.flags & EU_XS, zs = u.flags & EU_ZS;
#pragma unroll
    for (int q = 0; q < E_RPW; ++q) {
      const int z = u.z0 + r0 + q;
      const bool ok = colok && z < g.NZ;
      const size_t c = so + (size_t)z * g.NXp + gx;
      f4(ldg4z(a.vx + c, ok), vx[q]);
      f4(ldg4z(a.vz + c, ok), vz[q]);
      f4(ldg4z(a.p1 + c, ok && xs), p1[q]);
      f4(ldg4z(a.p3 + c, ok && xs), p3[q]);
      f4(ldg4z(a.p2 + c, ok && zs), p2[q]);
      f4(ldg4z(a.p4 + c, ok && zs), p4[q]);
    }
    float axh[4], bxh[4], ax[4], bx[4];
    if (xs && colok) {
      f4(*reinterpret_cast<const float4*>(a.axh + gx), axh);
      f4(*reinterpret_cast<const float4*>(a.bxh + gx), bxh);
      f4(*reinterpret_cast<const float4*>(a.ax + gx), ax);
      f4(*reinterpret_cast<const float4*>(a.bx + gx), bx);
    }
    if (!wait()) return false;
#pragma unroll
    for (int q = 0; q < E_RPW; ++q) {
      const int r = r0 + q, z = u.z0 + r;
      if (z >= g.NZ || !colok) continue;
      float e[12], f[12], t0[4], t1[4], t2[4], t3[4], bxv[4], bzv[4];
      // vx at (z, x+1/2): Dpx txx (half point), Dmz txz (integer point)
      f4(lds4e(sg.txx, E_HW, r, lx), e);
      f4(lds4e(sg.txx, E_HW, r, lx + 4), e + 4);
      f4(lds4e(sg.txx, E_HW, r, lx + 8), e + 8);
      f4(lds4e(sg.txz, E_HW, r + 2, lx + 4), t0);
      f4(lds4e(sg.txz, E_HW, r + 3, lx + 4), t1);
      f4(lds4e(sg.txz, E_HW, r + 4, lx + 4), t2);
      f4(lds4e(sg.txz, E_HW, r + 5, lx + 4), t3);
      f4(lds4e(sg.cbx, TB_X, r, lx), bxv);
      float outx[4], outz[4];
      const float azr = zs ? __ldg(a.az + z) : 0.f, bzr = zs ? __ldg(a.bz + z) : 0.f;
      const float azh = zs ? __ldg(a.azh + z) : 0.f, bzh = zs ? __ldg(a.bzh + z) : 0.f;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float dxt = kS1 * (e[c + 5] - e[c + 4]) + kS2 * (e[c + 6] - e[c + 3]);
        float dzt = kS1 * (t2[c] - t1[c]) + kS2 * (t3[c] - t0[c]);
        if (xs) {
          p1[q][c] = axh[c] * p1[q][c] + bxh[c] * dxt;
          dxt += p1[q][c];
        }
        if (zs) {
          p2[q][c] = azr * p2[q][c] + bzr * dzt;
          dzt += p2[q][c];
        }
        outx[c] = vx[q][c] + bxv[c] * (dxt + dzt);
      }
      // vz at (z+1/2, x): Dmx txz (integer point), Dpz tzz (half point)
      f4(lds4e(sg.txz, E_HW, r + 4, lx), f);
      f4(lds4e(sg.txz, E_HW, r + 4, lx + 4), f + 4);
      f4(lds4e(sg.txz, E_HW, r + 4, lx + 8), f + 8);
      f4(lds4e(sg.tzz, TB_X, r + 3, lx), t0);
      f4(lds4e(sg.tzz, TB_X, r + 4, lx), t1);
      f4(lds4e(sg.tzz, TB_X, r + 5, lx), t2);
      f4(lds4e(sg.tzz, TB_X, r + 6, lx), t3);
      f4(lds4e(sg.cbz, TB_X, r, lx), bzv);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float dxt = kS1 * (f[c + 4] - f[c + 3]) + kS2 * (f[c + 5] - f[c + 2]);
        float dzt = kS1 * (t2[c] - t1[c]) + kS2 * (t3[c] - t0[c]);
        if (xs) {
          p3[q][c] = ax[c] * p3[q][c] + bx[c] * dxt;
          dxt += p3[q][c];
        }
        if (zs) {
          p4[q][c] = azh * p4[q][c] + bzh * dzt;
          dzt += p4[q][c];
        }
        outz[c] = vz[q][c] + bzv[c] * (dxt + dzt);
      }
      const size_t ci = so + (size_t)z * g.NXp + gx;
      stg4(a.vx_o + ci, outx);
      stg4(a.vz_o + ci, outz);
      if (xs) {
        stg4(a.p1_o + ci, p1[q]);
        stg4(a.p3_o + ci, p3[q]);
      }
      if (zs) {
        stg4(a.p2_o + ci, p2[q]);
        stg4(a.p4_o + ci, p4[q]);
      }
    }
    return true;
  };
  e_pipeline<VelStage>(a, smem_raw, tab, ring, issue, body);
}

// ---------------------------------------------------------------- stress
__global__ void __launch_bounds__(E_THREADS, 1) el_str_kernel(const __grid_constant__ ElStepArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ EUnit tab[E_TABLE];
  __shared__ EUnit ring[E_STAGES];
  grid_dep_wait();
  if (*a.status) return;
  const Geom& g = a.g;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lx = 4 * lane, r0 = warp * E_RPW;
  auto issue = [&](StrStage& sg, uint64_t* b, const EUnit& u) {
    mbar_arrive_expect_tx(b, kStrBytes);
    tma_load_3d(sg.vx, &a.m_vx, b, u.x0 - 4, u.z0 - 4, u.s);
    tma_load_3d(sg.vz, &a.m_vz, b, u.x0 - 4, u.z0 - 4, u.s);
    tma_load_2d(sg.l2m, &a.m_l2m, b, u.x0, u.z0);
    tma_load_2d(sg.lam, &a.m_lam, b, u.x0, u.z0);
    tma_load_2d(sg.mu, &a.m_mu, b, u.x0, u.z0);
  };
  auto body = [&](const EUnit& u, const StrStage& sg, auto wait) {
    const int gx = u.x0 + lx;
    const bool colok = gx < g.NXp;
    const size_t so = (size_t)u.s * g.fstride;
    float txx[E_RPW][4], tzz[E_RPW][4], txz[E_RPW][4];
    float p5[E_RPW][4], p6[E_RPW][4], p7[E_RPW][4], p8[E_RPW][4];
    const bool xs = u.flags & EU_XS, zs = u.flags & EU_ZS;
#pragma unroll
    for (int q = 0; q < E_RPW; ++q) {
      const int z = u.z0 + r0 + q;
      const bool ok = colok && z < g.NZ;
      const size_t c = so + (size_t)z * g.NXp + gx;
      f4(ldg4z(a.txx + c, ok), txx[q]);
      f4(ldg4z(a.tzz + c, ok), tzz[q]);
      f4(ldg4z(a.txz + c, ok), txz[q]);
      f4(ldg4z(a.p5 + c, ok && xs), p5[q]);
      f4(ldg4z(a.p8 + c, ok && xs), p8[q]);
      f4(ldg4z(a.p6 + c, ok && zs), p6[q]);
      f4(ldg4z(a.p7 + c, ok && zs), p7[q]);
    }
    float axh[4], bxh[4], ax[4], bx[4];
    if (xs && colok) {
      f4(*reinterpret_cast<const float4*>(a.axh + gx), axh);
      f4(*reinterpret_cast<const float4*>(a.bxh + gx), bxh);
      f4(*reinterpret_cast<const float4*>(a.ax + gx), ax);
      f4(*reinterpret_cast<const float4*>(a.bx + gx), bx);
    }
    if (!wait()) return false;
#pragma unroll
    for (int q = 0; q < E_RPW; ++q) {
      const int r = r0 + q, z = u.z0 + r;
      if (z >= g.NZ || !colok) continue;
      float e[12], f[12], v0[4], v1[4], v2[4], v3[4], w0[4], w1[4], w2[4], w3[4];
      float l2m[4], lam[4], mu[4];
      f4(lds4e(sg.vx, E_HW, r + 4, lx), e);
      f4(lds4e(sg.vx, E_HW, r + 4, lx + 4), e + 4);
      f4(lds4e(sg.vx, E_HW, r + 4, lx + 8), e + 8);
      f4(lds4e(sg.vz, E_HW, r + 4, lx), f);
      f4(lds4e(sg.vz, E_HW, r + 4, lx + 4), f + 4);
      f4(lds4e(sg.vz, E_HW, r + 4, lx + 8), f + 8);
      f4(lds4e(sg.vx, E_HW, r + 3, lx + 4), v0);
      f4(lds4e(sg.vx, E_HW, r + 5, lx + 4), v2);
      f4(lds4e(sg.vx, E_HW, r + 6, lx + 4), v3);
      f4(lds4e(sg.vz, E_HW, r + 2, lx + 4), w0);
      f4(lds4e(sg.vz, E_HW, r + 3, lx + 4), w1);
      f4(lds4e(sg.vz, E_HW, r + 5, lx + 4), w3);
      f4(lds4e(sg.l2m, TB_X, r, lx), l2m);
      f4(lds4e(sg.lam, TB_X, r, lx), lam);
      f4(lds4e(sg.mu, TB_X, r, lx), mu);
      const float azr = zs ? __ldg(a.az + z) : 0.f, bzr = zs ? __ldg(a.bz + z) : 0.f;
      const float azh = zs ? __ldg(a.azh + z) : 0.f, bzh = zs ? __ldg(a.bzh + z) : 0.f;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        v1[c] = e[c + 4];  // vx(z, x)
        w2[c] = f[c + 4];  // vz(z, x)
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        // normal stresses at (z, x): Dmx vx, Dmz vz
        float exx = kS1 * (e[c + 4] - e[c + 3]) + kS2 * (e[c + 5] - e[c + 2]);
        float ezz = kS1 * (w2[c] - w1[c]) + kS2 * (w3[c] - w0[c]);
        if (xs) {
          p5[q][c] = ax[c] * p5[q][c] + bx[c] * exx;
          exx += p5[q][c];
        }
        if (zs) {
          p6[q][c] = azr * p6[q][c] + bzr * ezz;
          ezz += p6[q][c];
        }
        txx[q][c] += l2m[c] * exx + lam[c] * ezz;
        tzz[q][c] += lam[c] * exx + l2m[c] * ezz;
        // shear stress at (z+1/2, x+1/2): Dpz vx, Dpx vz
        float ezx = kS1 * (v2[c] - v1[c]) + kS2 * (v3[c] - v0[c]);
        float exz = kS1 * (f[c + 5] - f[c + 4]) + kS2 * (f[c + 6] - f[c + 3]);
        if (zs) {
          p7[q][c] = azh * p7[q][c] + bzh * ezx;
          ezx += p7[q][c];
        }
        if (xs) {
          p8[q][c] = axh[c] * p8[q][c] + bxh[c] * exz;
          exz += p8[q][c];
        }
        txz[q][c] += mu[c] * (ezx + exz);
      }
      if ((u.flags & EU_SRC) && z == u.sz) {
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (gx + c == u.sx) {
            txx[q][c] += u.amp;
            tzz[q][c] += u.amp;
          }
      }
      const size_t ci = so + (size_t)z * g.NXp + gx;
      stg4(a.txx_o + ci, txx[q]);
      stg4(a.tzz_o + ci, tzz[q]);
      stg4(a.txz_o + ci, txz[q]);
      if (xs) {
        stg4(a.p5_o + ci, p5[q]);
        stg4(a.p8_o + ci, p8[q]);
      }
      if (zs) {
        stg4(a.p6_o + ci, p6[q]);
        stg4(a.p7_o + ci, p7[q]);
      }
    }
    return true;
  };
  e_pipeline<StrStage>(a, smem_raw, tab, ring, issue, body);
}

// -------------------------------------------------------------- receivers
// trace sample n = v^{n+1/2} at the receiver cells (after the velocity kernel)
__global__ void el_rec_kernel(const ElStepArgs a) {
  grid_dep_wait();
  grid_dep_trigger();
  if (*a.status) return;
  const Geom& g = a.g;
  const int r = blockIdx.x * blockDim.x + threadIdx.x, s = blockIdx.y;
  if (r >= g.nrec) return;
  const int32_t* q = a.rec + 2 * ((size_t)s * g.nrec + r);
  const size_t c = (size_t)s * g.fstride + (size_t)(q[0] + g.P) * g.NXp + (q[1] + g.P);
  a.data[(((size_t)s * 2 + 0) * g.nrec + r) * g.nt + a.n] = a.vx_o[c];
  a.data[(((size_t)s * 2 + 1) * g.nrec + r) * g.nt + a.n] = a.vz_o[c];
}

}  // namespace

void launch_el_params(const ElParamArgs& a, cudaStream_t st) {
  const long long n = (long long)a.g.NZ * a.g.NXp;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  el_params_kernel<<<blocks, 256, 0, st>>>(a);
  note_launches(1);
}

bool el_step_maps(ElStepArgs& a) {
  const Geom& g = a.g;
  const uint64_t S = (uint64_t)(g.nshot > 0 ? g.nshot : 1);
  auto f3 = [&](CUtensorMap* m, const float* base, uint32_t bx, uint32_t bz) {
    return make_tensor_map(m, base, 3, g.NX, g.NZ, S, g.NXp, (uint64_t)g.fstride, bx, bz, 1);
  };
  auto f2 = [&](CUtensorMap* m, const float* base) {
    return make_tensor_map(m, base, 2, g.NX, g.NZ, 1, g.NXp, (uint64_t)g.fstride, TB_X, TB_Z, 1);
  };
  bool ok = f3(&a.m_txx, a.txx, E_HW, TB_Z) && f3(&a.m_txz, a.txz, E_HW, E_HZ) &&
            f3(&a.m_tzz, a.tzz, TB_X, E_HZ) && f3(&a.m_vx, a.vx_o, E_HW, E_HZ) &&
            f3(&a.m_vz, a.vz_o, E_HW, E_HZ) && f2(&a.m_cbx, a.cbx) && f2(&a.m_cbz, a.cbz) &&
            f2(&a.m_l2m, a.cl2m) && f2(&a.m_lam, a.clam) && f2(&a.m_mu, a.cmu);
  a.ntx = (g.NXp + TB_X - 1) / TB_X;
  a.units = a.ntx * ((g.NZ + TB_Z - 1) / TB_Z) * g.nshot;
  return ok;
}

void launch_el_step(const ElStepArgs& a, cudaStream_t st) {
  const Geom& g = a.g;
  if (a.units <= 0) return;
  static const bool attr = [] {  // thread-safe one-time initialisation
    cudaFuncSetAttribute(el_vel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kVelSmem);
    cudaFuncSetAttribute(el_str_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kStrSmem);
    return true;
  }();
  (void)attr;
  const int grid = std::min(device_sms(), a.units);
  void* t1 = profile_begin(SWEEP_K_EL_VEL, st);
  launch_dependent(el_vel_kernel, dim3(grid), dim3(E_THREADS), kVelSmem, st, a);
  profile_end(t1, st);
  int k = 2;
  if (a.data && g.nrec > 0) {
    launch_dependent(el_rec_kernel, dim3((g.nrec + 127) / 128, g.nshot), dim3(128), 0, st, a);
    ++k;
  }
  void* t2 = profile_begin(SWEEP_K_EL_STR, st);
  launch_dependent(el_str_kernel, dim3(grid), dim3(E_THREADS), kStrSmem, st, a);
  profile_end(t2, st);
  note_launches(k);
}

}  // namespace sweep
