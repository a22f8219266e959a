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
// A CTA owns a 32 x 64 tile of one shot; the fields whose neighbours it
// needs are staged in shared memory (zero outside the padded grid), each
// thread owns one column of 8 rows.
#include "sweep_internal.cuh"

namespace sweep {
namespace {

constexpr float kS1 = 9.0f / 8.0f;
constexpr float kS2 = -1.0f / 24.0f;

constexpr int ET = 256;          // threads
constexpr int EX = 64;           // tile columns
constexpr int EZ = 32;           // tile rows
constexpr int ER = EZ * EX / ET; // rows per thread
constexpr int EW = EX + 8;       // staged width with x halo (4 each side)
constexpr int EH = EZ + 8;       // staged height with z halo

__device__ __forceinline__ void stage(float* t, const float* __restrict__ f, const Geom& g,
                                      int zs, int h, int xs, int w) {
  const int w4 = w / 4;
  for (int idx = threadIdx.x; idx < h * w4; idx += ET) {
    const int r = idx / w4, c = idx - r * w4;
    const int gz = zs + r, gx = xs + 4 * c;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (gz >= 0 && gz < g.NZ && gx >= 0 && gx < g.NXp)
      v = *reinterpret_cast<const float4*>(f + (long long)gz * g.NXp + gx);
    *reinterpret_cast<float4*>(t + r * w + 4 * c) = v;
  }
}

// centred staggered difference from the samples at -3/2, -1/2, +1/2, +3/2
__device__ __forceinline__ float sdiff(float m32, float m12, float p12, float p32) {
  return kS1 * (p12 - m12) + kS2 * (p32 - m32);
}

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

// ------------------------------------------------------------- velocity
__global__ void __launch_bounds__(ET) el_vel_kernel(const ElStepArgs a) {
  __shared__ __align__(16) float sxx[EZ * EW];  // txx, x halo
  __shared__ __align__(16) float szz[EH * EX];  // tzz, z halo
  __shared__ __align__(16) float sxz[EH * EW];  // txz, both halos
  if (*a.status) return;
  const Geom& g = a.g;
  const int s = blockIdx.z;
  const int x0 = blockIdx.x * EX, z0 = blockIdx.y * EZ;
  const long long so = (long long)s * g.fstride;
  stage(sxx, a.txx + so, g, z0, EZ, x0 - 4, EW);
  stage(szz, a.tzz + so, g, z0 - 4, EH, x0, EX);
  stage(sxz, a.txz + so, g, z0 - 4, EH, x0 - 4, EW);
  __syncthreads();
  const int c = threadIdx.x % EX, r0 = (threadIdx.x / EX) * ER;
  const int x = x0 + c;
  if (x >= g.NX) return;
  const float axh = a.axh[x], bxh = a.bxh[x], ax = a.ax[x], bxp = a.bx[x];
#pragma unroll
  for (int q = 0; q < ER; ++q) {
    const int r = r0 + q, z = z0 + r;
    if (z >= g.NZ) break;
    const long long ci = so + (long long)z * g.NXp + x;
    const long long pc = (long long)z * g.NXp + x;
    const float* xx = sxx + r * EW + c + 4;
    const float* xz = sxz + (r + 4) * EW + c + 4;
    const float* zz = szz + (r + 4) * EX + c;
    // vx at (z, x+1/2): d/dx txx (half point), d/dz txz (integer point)
    float dxt = sdiff(xx[-1], xx[0], xx[1], xx[2]);
    float dzt = sdiff(xz[-2 * EW], xz[-EW], xz[0], xz[EW]);
    if (bxh != 0.f) {
      const float p = axh * a.p1[ci] + bxh * dxt;
      a.p1[ci] = p;
      dxt += p;
    }
    const float azr = a.az[z], bzr = a.bz[z];
    if (bzr != 0.f) {
      const float p = azr * a.p2[ci] + bzr * dzt;
      a.p2[ci] = p;
      dzt += p;
    }
    a.vx[ci] += a.cbx[pc] * (dxt + dzt);
    // vz at (z+1/2, x): d/dx txz (integer point), d/dz tzz (half point)
    float dxt2 = sdiff(xz[-2], xz[-1], xz[0], xz[1]);
    float dzt2 = sdiff(zz[-EX], zz[0], zz[EX], zz[2 * EX]);
    if (bxp != 0.f) {
      const float p = ax * a.p3[ci] + bxp * dxt2;
      a.p3[ci] = p;
      dxt2 += p;
    }
    const float azh = a.azh[z], bzh = a.bzh[z];
    if (bzh != 0.f) {
      const float p = azh * a.p4[ci] + bzh * dzt2;
      a.p4[ci] = p;
      dzt2 += p;
    }
    a.vz[ci] += a.cbz[pc] * (dxt2 + dzt2);
  }
}

// ---------------------------------------------------------------- stress
__global__ void __launch_bounds__(ET) el_str_kernel(const ElStepArgs a) {
  __shared__ __align__(16) float svx[EH * EW];  // vx^{n+1/2}, both halos
  __shared__ __align__(16) float svz[EH * EW];  // vz^{n+1/2}, both halos
  if (*a.status) return;
  const Geom& g = a.g;
  const int s = blockIdx.z;
  const int x0 = blockIdx.x * EX, z0 = blockIdx.y * EZ;
  const long long so = (long long)s * g.fstride;
  stage(svx, a.vx + so, g, z0 - 4, EH, x0 - 4, EW);
  stage(svz, a.vz + so, g, z0 - 4, EH, x0 - 4, EW);
  __syncthreads();
  const int c = threadIdx.x % EX, r0 = (threadIdx.x / EX) * ER;
  const int x = x0 + c;
  const int sz = a.src[2 * s] + g.P, sx = a.src[2 * s + 1] + g.P;
  const float amp = a.wavelet[(long long)s * g.nt + a.n] * a.src_scale;
  if (x < g.NX) {
    const float axh = a.axh[x], bxh = a.bxh[x], ax = a.ax[x], bxp = a.bx[x];
#pragma unroll
    for (int q = 0; q < ER; ++q) {
      const int r = r0 + q, z = z0 + r;
      if (z >= g.NZ) break;
      const long long ci = so + (long long)z * g.NXp + x;
      const long long pc = (long long)z * g.NXp + x;
      const float* vx = svx + (r + 4) * EW + c + 4;
      const float* vz = svz + (r + 4) * EW + c + 4;
      // normal stresses at (z, x)
      float exx = sdiff(vx[-2], vx[-1], vx[0], vx[1]);
      float ezz = sdiff(vz[-2 * EW], vz[-EW], vz[0], vz[EW]);
      if (bxp != 0.f) {
        const float p = ax * a.p5[ci] + bxp * exx;
        a.p5[ci] = p;
        exx += p;
      }
      const float azr = a.az[z], bzr = a.bz[z];
      if (bzr != 0.f) {
        const float p = azr * a.p6[ci] + bzr * ezz;
        a.p6[ci] = p;
        ezz += p;
      }
      const float l2m = a.cl2m[pc], lam = a.clam[pc];
      float txx = a.txx[ci] + l2m * exx + lam * ezz;
      float tzz = a.tzz[ci] + lam * exx + l2m * ezz;
      if (z == sz && x == sx) {
        txx += amp;
        tzz += amp;
      }
      a.txx[ci] = txx;
      a.tzz[ci] = tzz;
      // shear stress at (z+1/2, x+1/2)
      float ezx = sdiff(vx[-EW], vx[0], vx[EW], vx[2 * EW]);
      float exz = sdiff(vz[-1], vz[0], vz[1], vz[2]);
      const float azh = a.azh[z], bzh = a.bzh[z];
      if (bzh != 0.f) {
        const float p = azh * a.p7[ci] + bzh * ezx;
        a.p7[ci] = p;
        ezx += p;
      }
      if (bxh != 0.f) {
        const float p = axh * a.p8[ci] + bxh * exz;
        a.p8[ci] = p;
        exz += p;
      }
      a.txz[ci] += a.cmu[pc] * (ezx + exz);
    }
  }
  // record v^{n+1/2} at the receivers of this shot inside this tile
  if (a.data) {
    const int32_t* box = a.rbox + 4 * s;
    if (box[0] < z0 + EZ && box[1] >= z0 && box[2] < x0 + EX && box[3] >= x0) {
      for (int rr = threadIdx.x; rr < g.nrec; rr += ET) {
        const int32_t* q = a.rec + 2 * ((long long)s * g.nrec + rr);
        const int rz = q[0] + g.P, rx = q[1] + g.P;
        if (rz >= z0 && rz < z0 + EZ && rx >= x0 && rx < x0 + EX) {
          const int o = (rz - z0 + 4) * EW + (rx - x0 + 4);
          a.data[(((long long)s * 2 + 0) * g.nrec + rr) * g.nt + a.n] = svx[o];
          a.data[(((long long)s * 2 + 1) * g.nrec + rr) * g.nt + a.n] = svz[o];
        }
      }
    }
  }
}

}  // namespace

void launch_el_params(const ElParamArgs& a, cudaStream_t st) {
  const long long n = (long long)a.g.NZ * a.g.NXp;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  el_params_kernel<<<blocks, 256, 0, st>>>(a);
  note_launches(1);
}

void launch_el_step(const ElStepArgs& a, cudaStream_t st) {
  const Geom& g = a.g;
  dim3 grid((g.NXp + EX - 1) / EX, (g.NZ + EZ - 1) / EZ, g.nshot);
  void* t1 = profile_begin(SWEEP_K_EL_VEL, st);
  el_vel_kernel<<<grid, ET, 0, st>>>(a);
  profile_end(t1, st);
  void* t2 = profile_begin(SWEEP_K_EL_STR, st);
  el_str_kernel<<<grid, ET, 0, st>>>(a);
  profile_end(t2, st);
  note_launches(2);
}

}  // namespace sweep
