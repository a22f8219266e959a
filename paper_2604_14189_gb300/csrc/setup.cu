// Per-call setup on the device: edge-replicated padding of the model into
// K = v^2 dt^2 / dx^2 on the padded grid, the CPML profiles, and the checks
// that need device data (positions, model values, CFL).  Errors are latched
// in the workspace status word; later kernels of the call see it and skip.
//
// CPML profile (the paper names no absorbing boundary; this is the library's
// reading): depth d cells into the border measured at the sample's own
// position, rho = d / pml, sigma = 3 vref ln(1000) / (2 pml dx) rho^2,
// alpha = pi f_ref (1 - rho), a = exp(-(sigma + alpha) dt),
// b = sigma / (sigma + alpha) (a - 1), a = b = 0 outside the border.
#include <math.h>

#include "sweep_internal.cuh"

namespace sweep {
namespace {

__device__ __forceinline__ float model_at(const SetupArgs& a, int par, int z, int x) {
  const Geom& g = a.g;
  if (a.padded) return a.model[((long long)par * g.NZ + z) * g.NX + x];
  int zi = min(max(z - g.P, 0), g.nz - 1);
  int xi = min(max(x - g.P, 0), g.nx - 1);
  return a.model[((long long)par * g.nz + zi) * g.nx + xi];
}

__global__ void setup_model_kernel(const SetupArgs a) {
  const Geom& g = a.g;
  const long long n = (long long)g.NZ * g.NXp;
  const double c = (double)a.dt * a.dt / ((double)a.dx * a.dx);
  float vmax = 0.f;
  int bad = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int z = (int)(i / g.NXp), x = (int)(i - (long long)z * g.NXp);
    float k = 0.f;
    if (x < g.NX) {
      const float v = model_at(a, 0, z, x);
      if (!isfinite(v)) bad = SWEEP_ENONFINITE;
      else if (!(v > 0.f)) bad = bad ? bad : SWEEP_EMODEL;
      else vmax = fmaxf(vmax, v);
      k = (float)((double)v * v * c);
      if (a.physics == SWEEP_ELASTIC) {
        const float vs = model_at(a, 1, z, x), rho = model_at(a, 2, z, x);
        if (!isfinite(vs) || !isfinite(rho)) bad = SWEEP_ENONFINITE;
        else if (!(vs >= 0.f) || !(rho > 0.f) || 2.f * vs * vs > v * v)
          bad = bad ? bad : SWEEP_EMODEL;
      }
    }
    if (a.K) a.K[i] = k;
  }
  if (bad) latch(a.status, bad);
  // positive floats order like their bit patterns
  for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
  if ((threadIdx.x & 31) == 0) atomicMax(a.vmax_bits, __float_as_uint(vmax));
}

__device__ void profile(int n_int, int pml, double dx, double dt, double vref,
                        double f_ref, int half, int j, float* a, float* b) {
  const double x = half ? j + 0.5 : (double)j;
  double d = 0.0;
  if (x < pml) d = pml - x;
  else if (x > pml + n_int - 1) d = x - (pml + n_int - 1);
  if (d <= 0.0 || pml == 0) {
    a[j] = 0.f;
    b[j] = 0.f;
    return;
  }
  const double rho = fmin(d / pml, 1.0);
  const double smax = 3.0 * vref * log(1000.0) / (2.0 * pml * dx);
  const double sigma = smax * rho * rho;
  const double alpha = M_PI * f_ref * (1.0 - rho);
  const double av = exp(-(sigma + alpha) * dt);
  a[j] = (float)av;
  b[j] = (float)(sigma / (sigma + alpha) * (av - 1.0));
}

__global__ void setup_geometry_kernel(const SetupArgs a) {
  const Geom& g = a.g;
  const float vmax = __uint_as_float(*a.vmax_bits);
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    if ((double)vmax * a.dt / a.dx > (double)a.cfl_limit) latch(a.status, SWEEP_ECFL);
  }
  const double vref = a.v_pml > 0.f ? (double)a.v_pml : (double)vmax;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  for (int j = tid; j < g.NXp; j += nth) {
    if (j < g.NX) {
      profile(g.nx, g.P, a.dx, a.dt, vref, a.f_ref, 0, j, a.ax, a.bx);
      if (a.axh) profile(g.nx, g.P, a.dx, a.dt, vref, a.f_ref, 1, j, a.axh, a.bxh);
    } else {
      a.ax[j] = 0.f; a.bx[j] = 0.f;
      if (a.axh) { a.axh[j] = 0.f; a.bxh[j] = 0.f; }
    }
  }
  for (int i = tid; i < g.NZ; i += nth) {
    profile(g.nz, g.P, a.dx, a.dt, vref, a.f_ref, 0, i, a.az, a.bz);
    if (a.azh) profile(g.nz, g.P, a.dx, a.dt, vref, a.f_ref, 1, i, a.azh, a.bzh);
  }
  for (int s = tid; s < g.nshot; s += nth) {
    const int z = a.src[2 * s], x = a.src[2 * s + 1];
    if (z < 0 || z >= g.nz || x < 0 || x >= g.nx) latch(a.status, SWEEP_EBOUNDS);
  }
  const long long nr = (long long)g.nshot * g.nrec;
  for (long long r = tid; r < nr; r += nth) {
    const int z = a.rec[2 * r], x = a.rec[2 * r + 1];
    if (z < 0 || z >= g.nz || x < 0 || x >= g.nx) {
      latch(a.status, SWEEP_EBOUNDS);
    }
  }
}

}  // namespace

void launch_setup(const SetupArgs& a, cudaStream_t st) {
  cudaMemsetAsync(a.vmax_bits, 0, sizeof(unsigned int), st);
  const long long n = (long long)a.g.NZ * a.g.NXp;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 1216) blocks = 1216;
  setup_model_kernel<<<blocks, 256, 0, st>>>(a);
  setup_geometry_kernel<<<8, 256, 0, st>>>(a);
  note_launches(2);
}

}  // namespace sweep
