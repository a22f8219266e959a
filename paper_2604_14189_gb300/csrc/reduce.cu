// FP64 reductions: the L2 misfit with its residual, the shot sum of the
// per-shot imaging terms into the velocity gradient, and a dot product.
// Partial sums are written per block and summed in a fixed order, so results
// do not depend on scheduling.
#include "sweep_internal.cuh"

namespace sweep {
namespace {

constexpr int RT = 256;

__device__ double block_sum(double v) {
  __shared__ double sh[RT / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < RT / 32; ++i) t += sh[i];
  return t;  // valid in thread 0
}

// r = d - d_obs (or r = d_obs when residual_in), partial[b] = sum 1/2 r^2
// res may alias d (the residual overwrites the recorded data in place)
__global__ void __launch_bounds__(RT) residual_kernel(const float* d, const float* d_obs,
                                                     float* res, long long n,
                                                     int residual_in, double* partial,
                                                     const int* status) {
  if (*status) return;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n;
       i += (long long)gridDim.x * RT) {
    const float r = residual_in ? d_obs[i] : d[i] - d_obs[i];
    res[i] = r;
    acc += 0.5 * (double)r * (double)r;
  }
  const double t = block_sum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

__global__ void __launch_bounds__(RT) finish_kernel(const double* partial, int nblocks,
                                                    double* out, int* status,
                                                    int check_finite) {
  if (status && *status) return;
  double acc = 0.0;
  // fixed assignment of partials to threads, then a fixed-order tree
  for (int i = threadIdx.x; i < nblocks; i += RT) acc += partial[i];
  const double t = block_sum(acc);
  if (threadIdx.x == 0) {
    if (out) *out = t;
    if (check_finite && status && !isfinite(t)) latch(status, SWEEP_ENONFINITE);
  }
}

__global__ void __launch_bounds__(RT) dot_kernel(const float* __restrict__ a,
                                                 const float* __restrict__ b, long long n,
                                                 double* partial) {
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n;
       i += (long long)gridDim.x * RT)
    acc += (double)a[i] * (double)b[i];
  const double t = block_sum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// grad[c] = 2 / v(c) * sum_s graw[s][c];  illum[c] = sum_s illum_raw[s][c]
__global__ void __launch_bounds__(RT) grad_reduce_kernel(const Geom g,
                                                         const float* __restrict__ graw,
                                                         const float* __restrict__ iraw,
                                                         const float* __restrict__ model,
                                                         int padded, float* grad,
                                                         float* illum, const int* status) {
  if (*status) return;
  // graw / iraw: per shot on the padded grid [S][NZ][NXp]
  const long long nint = (long long)g.nz * g.nx;
  for (long long c = blockIdx.x * (long long)RT + threadIdx.x; c < nint;
       c += (long long)gridDim.x * RT) {
    const int z = (int)(c / g.nx), x = (int)(c - (long long)z * g.nx);
    const long long pc = (long long)(z + g.P) * g.NXp + (x + g.P);
    double acc = 0.0, ill = 0.0;
    for (int s = 0; s < g.nshot; ++s) {
      acc += (double)graw[(long long)s * g.fstride + pc];
      if (iraw) ill += (double)iraw[(long long)s * g.fstride + pc];
    }
    const float v = padded ? model[(long long)(z + g.P) * g.NX + (x + g.P)] : model[c];
    grad[c] = (float)(2.0 * acc / (double)v);
    if (illum) illum[c] = (float)ill;
  }
}

}  // namespace

void launch_residual_misfit(const float* d, const float* d_obs, float* res, long long n,
                            int residual_in, double* partial, int nblocks, double* misfit,
                            int* status, cudaStream_t st) {
  residual_kernel<<<nblocks, RT, 0, st>>>(d, d_obs, res, n, residual_in, partial, status);
  finish_kernel<<<1, RT, 0, st>>>(partial, nblocks, misfit, status, 1);
}

void launch_grad_reduce(const Geom& g, const float* graw, const float* illum_raw,
                        const float* model, int padded, float* grad, float* illum,
                        const int* status, cudaStream_t st) {
  long long nint = (long long)g.nz * g.nx;
  int blocks = (int)((nint + RT - 1) / RT);
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  grad_reduce_kernel<<<blocks, RT, 0, st>>>(g, graw, illum_raw, model, padded, grad, illum,
                                            status);
}

void launch_dot(const float* a, const float* b, long long n, double* partial, int nblocks,
                double* out, cudaStream_t st) {
  dot_kernel<<<nblocks, RT, 0, st>>>(a, b, n, partial);
  finish_kernel<<<1, RT, 0, st>>>(partial, nblocks, out, nullptr, 0);
}

}  // namespace sweep
