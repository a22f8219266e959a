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
//   coefficients (summed over shots and steps in FP64):
//            d J / d cl2m += txx-bar Ex + tzz-bar Ez, d J / d clam +=
//            txx-bar Ez + tzz-bar Ex, d J / d cmu += txz-bar (shear bracket),
//            d J / d cbx += vx-bar (vx bracket), d J / d cbz likewise.
// Each half is a pointwise kernel (the adjoint derivative terms into four
// scratch fields, memory variables, coefficient adjoints) and a gather
// kernel (the transposed differences of those terms).
//
// A memory variable and its adjoint stay zero wherever its profile pair
// (a, b) is zero, i.e. off its border strip (both start at zero and are
// only ever replaced by a x (...)); the pointwise kernels neither read nor
// write them there, which is most of the grid.
#include "elastic_internal.cuh"

namespace sweep {
namespace {

constexpr float kS1 = 9.0f / 8.0f;
constexpr float kS2 = -1.0f / 24.0f;
constexpr int AT = 128;  // threads per block (a row segment of one shot)

struct Fld {
  const float* f;
  int NZ, NX, NXp;
  __device__ __forceinline__ float operator()(int z, int x) const {
    return (z >= 0 && z < NZ && x >= 0 && x < NX) ? f[z * NXp + x] : 0.f;
  }
};
__device__ __forceinline__ Fld fld(const float* f, const Geom& g, int s) {
  return Fld{f + (size_t)s * g.fstride, g.NZ, g.NX, g.NXp};
}
// staggered differences, as in the forward kernels
__device__ __forceinline__ float dpx(const Fld& f, int z, int x) {
  return kS1 * (f(z, x + 1) - f(z, x)) + kS2 * (f(z, x + 2) - f(z, x - 1));
}
__device__ __forceinline__ float dmx(const Fld& f, int z, int x) {
  return kS1 * (f(z, x) - f(z, x - 1)) + kS2 * (f(z, x + 1) - f(z, x - 2));
}
__device__ __forceinline__ float dpz(const Fld& f, int z, int x) {
  return kS1 * (f(z + 1, x) - f(z, x)) + kS2 * (f(z + 2, x) - f(z - 1, x));
}
__device__ __forceinline__ float dmz(const Fld& f, int z, int x) {
  return kS1 * (f(z, x) - f(z - 1, x)) + kS2 * (f(z + 1, x) - f(z - 2, x));
}

enum { G_L2M = 0, G_LAM = 1, G_MU = 2, G_BX = 3, G_BZ = 4 };

// ------------------------------------------------------------- wavelet
__global__ void el_adj_src_kernel(const ElAdjArgs a) {
  if (*a.status) return;
  const Geom& g = a.g;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.nshot) return;
  const size_t c = (size_t)s * g.fstride + (size_t)(a.src[2 * s] + g.P) * g.NXp +
                   (a.src[2 * s + 1] + g.P);
  a.wgrad[(size_t)s * g.nt + a.n] = a.src_scale * (a.atxx[c] + a.atzz[c]);
}

// ------------------------------------------------------- stress, pointwise
// One thread per cell for all shots: the coefficient adjoints are summed
// over the shots in FP64 registers and added once per step to the FP64
// accumulators [5][NZ][NXp] (shot sum and time sum in FP64).
__global__ void __launch_bounds__(AT) el_adj_str_pt_kernel(const ElAdjArgs a) {
  if (*a.status) return;
  const Geom& g = a.g;
  const int x = blockIdx.x * AT + threadIdx.x, z = blockIdx.y;
  if (x >= g.NXp) return;
  const size_t pc = (size_t)z * g.NXp + x;
  if (x >= g.NX) {  // zero terms beyond the grid for the gather kernel
    for (int s = 0; s < g.nshot; ++s) {
      const size_t c = (size_t)s * g.fstride + pc;
      a.e0[c] = a.e1[c] = a.e2[c] = a.e3[c] = 0.f;
    }
    return;
  }
  const float l2m = a.cl2m[pc], lam = a.clam[pc], mu = a.cmu[pc];
  // profile pairs of p5 (x), p6 (z), p7 (z, half points), p8 (x, half points)
  const float A5 = a.ax[x], B5 = a.bx[x], A6 = a.az[z], B6 = a.bz[z];
  const float A7 = a.azh[z], B7 = a.bzh[z], A8 = a.axh[x], B8 = a.bxh[x];
  const bool o5 = A5 != 0.f || B5 != 0.f, o6 = A6 != 0.f || B6 != 0.f;
  const bool o7 = A7 != 0.f || B7 != 0.f, o8 = A8 != 0.f || B8 != 0.f;
  double sl2m = 0.0, slam = 0.0, smu = 0.0;
  for (int s = 0; s < g.nshot; ++s) {
    const size_t c = (size_t)s * g.fstride + pc;
    const float txx = a.atxx[c], tzz = a.atzz[c], txz = a.atxz[c];
    if (a.gacc) {
      const Fld vx = fld(a.fvx, g, s), vz = fld(a.fvz, g, s);
      const float ex = dmx(vx, z, x) + (o5 ? a.fp[4][c] : 0.f);
      const float ez = dmz(vz, z, x) + (o6 ? a.fp[5][c] : 0.f);
      const float sxz = dpz(vx, z, x) + (o7 ? a.fp[6][c] : 0.f) + dpx(vz, z, x) +
                        (o8 ? a.fp[7][c] : 0.f);
      sl2m += (double)(txx * ex + tzz * ez);
      slam += (double)(txx * ez + tzz * ex);
      smu += (double)(txz * sxz);
    }
    // txz += cmu (ezx + p7' + exz + p8')
    const float T = mu * txz;
    const float P7 = (o7 ? a.ap[6][c] : 0.f) + T, P8 = (o8 ? a.ap[7][c] : 0.f) + T;
    a.e2[c] = T + B7 * P7;  // ezx-bar
    a.e3[c] = T + B8 * P8;  // exz-bar
    if (o7) a.ap[6][c] = A7 * P7;
    if (o8) a.ap[7][c] = A8 * P8;
    // txx += cl2m Ex + clam Ez, tzz += clam Ex + cl2m Ez
    const float Ex = l2m * txx + lam * tzz, Ez = lam * txx + l2m * tzz;
    const float P5 = (o5 ? a.ap[4][c] : 0.f) + Ex, P6 = (o6 ? a.ap[5][c] : 0.f) + Ez;
    a.e0[c] = Ex + B5 * P5;  // exx-bar
    a.e1[c] = Ez + B6 * P6;  // ezz-bar
    if (o5) a.ap[4][c] = A5 * P5;
    if (o6) a.ap[5][c] = A6 * P6;
  }
  if (a.gacc) {
    double* ga = a.gacc + pc;
    ga[G_L2M * g.fstride] += sl2m;
    ga[G_LAM * g.fstride] += slam;
    ga[G_MU * g.fstride] += smu;
  }
}

// ----------------------------------------------------------- stress, gather
__global__ void __launch_bounds__(AT) el_adj_str_sc_kernel(const ElAdjArgs a) {
  if (*a.status) return;
  const Geom& g = a.g;
  const int x = blockIdx.x * AT + threadIdx.x, z = blockIdx.y, s = blockIdx.z;
  if (x >= g.NX) return;
  const size_t c = (size_t)s * g.fstride + (size_t)z * g.NXp + x;
  const Fld exx = fld(a.e0, g, s), ezz = fld(a.e1, g, s), ezx = fld(a.e2, g, s),
            exz = fld(a.e3, g, s);
  a.avx[c] -= dpx(exx, z, x) + dmz(ezx, z, x);
  a.avz[c] -= dpz(ezz, z, x) + dmx(exz, z, x);
}

// ---------------------------------------------------------------- receivers
__global__ void el_adj_rec_kernel(const ElAdjArgs a) {
  if (*a.status) return;
  const Geom& g = a.g;
  const int r = blockIdx.x * blockDim.x + threadIdx.x, s = blockIdx.y;
  if (r >= g.nrec) return;
  const int32_t* q = a.rec + 2 * ((size_t)s * g.nrec + r);
  const size_t c = (size_t)s * g.fstride + (size_t)(q[0] + g.P) * g.NXp + (q[1] + g.P);
  a.avx[c] += a.res[(((size_t)s * 2 + 0) * g.nrec + r) * g.nt + a.n];
  a.avz[c] += a.res[(((size_t)s * 2 + 1) * g.nrec + r) * g.nt + a.n];
}

// ----------------------------------------------------- velocity, pointwise
__global__ void __launch_bounds__(AT) el_adj_vel_pt_kernel(const ElAdjArgs a) {
  if (*a.status) return;
  const Geom& g = a.g;
  const int x = blockIdx.x * AT + threadIdx.x, z = blockIdx.y;
  if (x >= g.NXp) return;
  const size_t pc = (size_t)z * g.NXp + x;
  if (x >= g.NX) {
    for (int s = 0; s < g.nshot; ++s) {
      const size_t c = (size_t)s * g.fstride + pc;
      a.e0[c] = a.e1[c] = a.e2[c] = a.e3[c] = 0.f;
    }
    return;
  }
  const float cbx = a.cbx[pc], cbz = a.cbz[pc];
  // profile pairs of p1 (x, half points), p2 (z), p3 (x), p4 (z, half points)
  const float A1 = a.axh[x], B1 = a.bxh[x], A2 = a.az[z], B2 = a.bz[z];
  const float A3 = a.ax[x], B3 = a.bx[x], A4 = a.azh[z], B4 = a.bzh[z];
  const bool o1 = A1 != 0.f || B1 != 0.f, o2 = A2 != 0.f || B2 != 0.f;
  const bool o3 = A3 != 0.f || B3 != 0.f, o4 = A4 != 0.f || B4 != 0.f;
  double sbx = 0.0, sbz = 0.0;
  for (int s = 0; s < g.nshot; ++s) {
    const size_t c = (size_t)s * g.fstride + pc;
    const float vx = a.avx[c], vz = a.avz[c];
    if (a.gacc) {
      const Fld txx = fld(a.ftxx, g, s), tzz = fld(a.ftzz, g, s), txz = fld(a.ftxz, g, s);
      const float sx = dpx(txx, z, x) + (o1 ? a.fp[0][c] : 0.f) + dmz(txz, z, x) +
                       (o2 ? a.fp[1][c] : 0.f);
      const float sz = dmx(txz, z, x) + (o3 ? a.fp[2][c] : 0.f) + dpz(tzz, z, x) +
                       (o4 ? a.fp[3][c] : 0.f);
      sbx += (double)(vx * sx);
      sbz += (double)(vz * sz);
    }
    // vx += cbx (dxt + p1' + dzt + p2')
    const float Q = cbx * vx;
    const float P1 = (o1 ? a.ap[0][c] : 0.f) + Q, P2 = (o2 ? a.ap[1][c] : 0.f) + Q;
    a.e0[c] = Q + B1 * P1;  // dxt-bar (Dpx txx)
    a.e1[c] = Q + B2 * P2;  // dzt-bar (Dmz txz)
    if (o1) a.ap[0][c] = A1 * P1;
    if (o2) a.ap[1][c] = A2 * P2;
    // vz += cbz (dxt + p3' + dzt + p4')
    const float Qz = cbz * vz;
    const float P3 = (o3 ? a.ap[2][c] : 0.f) + Qz, P4 = (o4 ? a.ap[3][c] : 0.f) + Qz;
    a.e2[c] = Qz + B3 * P3;  // dxt-bar (Dmx txz)
    a.e3[c] = Qz + B4 * P4;  // dzt-bar (Dpz tzz)
    if (o3) a.ap[2][c] = A3 * P3;
    if (o4) a.ap[3][c] = A4 * P4;
  }
  if (a.gacc) {
    double* ga = a.gacc + pc;
    ga[G_BX * g.fstride] += sbx;
    ga[G_BZ * g.fstride] += sbz;
  }
}

// --------------------------------------------------------- velocity, gather
__global__ void __launch_bounds__(AT) el_adj_vel_sc_kernel(const ElAdjArgs a) {
  if (*a.status) return;
  const Geom& g = a.g;
  const int x = blockIdx.x * AT + threadIdx.x, z = blockIdx.y, s = blockIdx.z;
  if (x >= g.NX) return;
  const size_t c = (size_t)s * g.fstride + (size_t)z * g.NXp + x;
  const Fld d0 = fld(a.e0, g, s), d1 = fld(a.e1, g, s), d2 = fld(a.e2, g, s),
            d3 = fld(a.e3, g, s);
  a.atxx[c] -= dmx(d0, z, x);
  a.atxz[c] -= dpz(d1, z, x) + dpx(d2, z, x);
  a.atzz[c] -= dmz(d3, z, x);
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
// coefficient adjoint k at padded point (z, x), summed over shots and steps
__device__ __forceinline__ double gsum(const double* gacc, const Geom& g, int k, int z, int x) {
  return gacc[(size_t)k * g.fstride + (size_t)z * g.NXp + x];
}

__global__ void el_grad_kernel(const Geom g, const double* gacc, const float* model, int padded,
                               double sc, float* grad, const int* status) {
  if (*status) return;
  const int i = blockIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= g.nx) return;
  const int Z = i + g.P, X = j + g.P;
  const double vp = mval(model, g, padded, 0, Z, X), vs = mval(model, g, padded, 1, Z, X);
  const double rho = mval(model, g, padded, 2, Z, X), mu = rho * vs * vs;
  // lam = rho (vp^2 - 2 vs^2): cl2m = sc (lam + 2 mu), clam = sc lam
  const double gl2m = gsum(gacc, g, G_L2M, Z, X);
  const double glam = sc * (gl2m + gsum(gacc, g, G_LAM, Z, X));
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
      gmu += mult * sc * gsum(gacc, g, G_MU, pz, px) * mxz * mxz / (4.0 * mu * mu);
    }
  // cbx at (Z, px) = sc 2 / (rho(Z, px) + rho(Z, px+1)), cbz likewise in z
  for (int dx = -1; dx <= 0; ++dx) {
    const int px = X + dx;
    if (px < 0) continue;
    const int px1 = min(px + 1, g.NX - 1);
    const int mult = (px == X) + (px1 == X);
    if (!mult) continue;
    const double r2 = mval(model, g, padded, 2, Z, px) + mval(model, g, padded, 2, Z, px1);
    grho += mult * sc * gsum(gacc, g, G_BX, Z, px) * (-2.0 / (r2 * r2));
  }
  for (int dz = -1; dz <= 0; ++dz) {
    const int pz = Z + dz;
    if (pz < 0) continue;
    const int pz1 = min(pz + 1, g.NZ - 1);
    const int mult = (pz == Z) + (pz1 == Z);
    if (!mult) continue;
    const double r2 = mval(model, g, padded, 2, pz, X) + mval(model, g, padded, 2, pz1, X);
    grho += mult * sc * gsum(gacc, g, G_BZ, pz, X) * (-2.0 / (r2 * r2));
  }
  const size_t M = (size_t)g.nz * g.nx, o = (size_t)i * g.nx + j;
  grad[o] = (float)(glam * 2.0 * rho * vp);
  grad[M + o] = (float)(glam * (-4.0 * rho * vs) + gmu * 2.0 * rho * vs);
  grad[2 * M + o] = (float)(grho + glam * (vp * vp - 2.0 * vs * vs) + gmu * vs * vs);
}

}  // namespace

namespace {

// profile pair of memory variable k (p1..p8): x axis?, half points?
__device__ __forceinline__ bool snap_on(const ElSnapArgs& a, int k, int z, int x) {
  const Geom& g = a.g;
  const bool xaxis = k == 0 || k == 2 || k == 4 || k == 7;
  const bool half = k == 0 || k == 3 || k == 6 || k == 7;
  if (!xaxis) {
    const float A = half ? a.azh[z] : a.az[z], B = half ? a.bzh[z] : a.bz[z];
    return A != 0.f || B != 0.f;
  }
  bool on = false;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (x + i < g.NX) {
      const float A = half ? a.axh[x + i] : a.ax[x + i];
      const float B = half ? a.bxh[x + i] : a.bx[x + i];
      on = on || A != 0.f || B != 0.f;
    }
  }
  return on;
}

// one thread per 4-cell group of a row of one shot
__global__ void __launch_bounds__(128) el_snapshot_kernel(const ElSnapArgs a) {
  const Geom& g = a.g;
  const int x = 4 * (blockIdx.x * 128 + threadIdx.x), z = blockIdx.y, s = blockIdx.z;
  if (x >= g.NXp) return;
  const size_t c = (size_t)s * g.fstride + (size_t)z * g.NXp + x;
#pragma unroll
  for (int f = 0; f < 5; ++f)
    *reinterpret_cast<float4*>(a.dst[f] + c) = *reinterpret_cast<const float4*>(a.src[f] + c);
  if (x >= g.NX) return;
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if (snap_on(a, k, z, x))
      *reinterpret_cast<float4*>(a.dst[5 + k] + c) =
          *reinterpret_cast<const float4*>(a.src[5 + k] + c);
}

}  // namespace

void launch_el_snapshot(const ElSnapArgs& a, cudaStream_t st) {
  const Geom& g = a.g;
  if (g.nshot <= 0) return;
  const dim3 grid((g.NXp / 4 + 127) / 128, g.NZ, g.nshot);
  el_snapshot_kernel<<<grid, 128, 0, st>>>(a);
  note_launches(1);
}

void launch_el_adj_step(const ElAdjArgs& a, cudaStream_t st) {
  const Geom& g = a.g;
  const dim3 grid((g.NXp + AT - 1) / AT, g.NZ, g.nshot);
  const dim3 cells((g.NXp + AT - 1) / AT, g.NZ);  // pointwise kernels: all shots per thread
  int k = 0;
  if (a.wgrad) {
    el_adj_src_kernel<<<(g.nshot + 127) / 128, 128, 0, st>>>(a);
    ++k;
  }
  el_adj_str_pt_kernel<<<cells, AT, 0, st>>>(a);
  el_adj_str_sc_kernel<<<grid, AT, 0, st>>>(a);
  k += 2;
  if (a.res && g.nrec > 0) {
    el_adj_rec_kernel<<<dim3((g.nrec + 127) / 128, g.nshot), 128, 0, st>>>(a);
    ++k;
  }
  el_adj_vel_pt_kernel<<<cells, AT, 0, st>>>(a);
  el_adj_vel_sc_kernel<<<grid, AT, 0, st>>>(a);
  note_launches(k + 2);
}

void launch_el_grad(const Geom& g, const double* gacc, const float* model, int padded, float dx,
                    float dt, float* grad, const int* status, cudaStream_t st) {
  const double sc = (double)dt / (double)dx;
  el_grad_kernel<<<dim3((g.nx + 127) / 128, g.nz), 128, 0, st>>>(g, gacc, model, padded, sc,
                                                                 grad, status);
  note_launches(1);
}

}  // namespace sweep
