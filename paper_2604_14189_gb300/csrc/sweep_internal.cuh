// Internal declarations of the GB300 solver library (CUDA side only).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sweep.h"

namespace sweep {

// ---------------------------------------------------------------------------
// Geometry of one acoustic problem on the padded grid.
// Fields are stored per shot as [NZ][NXp] floats, NXp = NX rounded up to a
// multiple of 32 (128-byte rows); columns NX..NXp-1 hold zeros at all times.
// ---------------------------------------------------------------------------
struct Geom {
  int nz, nx, P;      // interior size, border width
  int NZ, NX, NXp;    // padded size, row pitch (floats)
  int nshot, nrec, nt;
  int ringw;          // width of the saved ring, min(P, 4)
  int nring;          // cells in the ring
  long long fstride;  // floats per shot per field = NZ * NXp
};

// Tile shape of the acoustic step kernels: BX cells along x (one warp, 4
// cells per lane), BZ rows; RPW rows per warp.
constexpr int AC_BX = 128;
constexpr int AC_BZ = 32;
constexpr int AC_RPW = 8;
constexpr int AC_THREADS = 32 * (AC_BZ / AC_RPW);

struct AcFwdArgs {
  Geom g;
  const float* u;     // u^n            [S][NZ][NXp]
  float* un;          // in u^{n-1}, out u^{n+1}
  const float* K;     // [NZ][NXp]  v^2 dt^2 / dx^2
  const float* psx_in;
  float* psx_out;     // psi_x^{n-1} -> psi_x^n   [S][NZ][NXp]
  const float* psz_in;
  float* psz_out;
  float* zex;         // zeta_x, updated in place  [S][NZ][NXp]
  float* zez;
  const float* ax;    // profiles [NXp] / [NZ]
  const float* bx;
  const float* az;
  const float* bz;
  const float* wavelet;  // [S][nt]
  const int32_t* src;    // [S][2]
  const int32_t* rec;    // [S][R][2]
  float* data;           // [S][R][nt] or null
  float* save;           // ring slot of u^{n+1}: [S][nring] or null
  const int* status;
  int n;
};

struct AcBwdArgs {
  Geom g;
  const float* uA;    // u^n (interior + ring valid)
  float* uB;          // in u^{n+1}, out u^{n-1} (interior + ring)
  const float* mA;    // mu^{n+1}
  float* mB;          // in mu^{n+2}, out mu^n
  const float* pbx_in;
  float* pbx_out;     // adjoint psi_x: ^n -> ^{n-1}
  const float* pbz_in;
  float* pbz_out;
  const float* zbx_in;
  float* zbx_out;     // adjoint zeta_x: ^n -> ^{n-1}
  const float* zbz_in;
  float* zbz_out;
  const float* K;
  const float* ax;
  const float* bx;
  const float* az;
  const float* bz;
  const float* wavelet;  // [S][nt]
  const int32_t* src;
  const int32_t* rec;
  const float* res;      // residual [S][R][nt] (injected at sample n-1)
  const float* save;     // ring slot of u^{n-1}: [S][nring] (or null)
  float* graw;           // [S][nz][nx] sum mu^{n+1} (Lap u^n + f delta)
  float* illum;          // [S][nz][nx] sum (u^n)^2, or null
  float* wgrad;          // [S][nt] adjoint source gather, or null
  const int* status;
  int n;
  int do_adj;            // compute mu^n (and inject r^{n-1})
  int do_img;            // imaging with mu^{n+1}, u^n
  int do_rec;            // reconstruct u^{n-1} (+ ring restore)
};

// Kernel launchers (acoustic.cu)
void launch_ac_fwd(const AcFwdArgs& a, cudaStream_t st);
void launch_ac_bwd(const AcBwdArgs& a, cudaStream_t st);

// Setup (setup.cu)
struct SetupArgs {
  Geom g;
  int physics;
  const float* model;  // interior or padded
  int padded;
  float dx, dt, f_ref, v_pml;
  float cfl_limit;
  const int32_t* src;
  const int32_t* rec;
  float* K;            // out [NZ][NXp] (acoustic)
  float* ax;           // out profiles
  float* bx;
  float* az;
  float* bz;
  float* axh;          // half-point profiles (elastic)
  float* bxh;
  float* azh;
  float* bzh;
  unsigned int* vmax_bits;  // scratch: max vp as float bits
  int* status;
};
void launch_setup(const SetupArgs& a, cudaStream_t st);

// Reductions (reduce.cu)
void launch_residual_misfit(const float* d, const float* d_obs, float* res,
                            long long n, int residual_in, double* partial,
                            int nblocks, double* misfit, int* status,
                            cudaStream_t st);
void launch_grad_reduce(const Geom& g, const float* graw, const float* illum_raw,
                        const float* model, int padded, float* grad,
                        float* illum, const int* status, cudaStream_t st);
void launch_dot(const float* a, const float* b, long long n, double* partial,
                int nblocks, double* out, cudaStream_t st);

constexpr int RED_BLOCKS = 1024;  // partial sums of the FP64 reductions

// Launch accounting and optional per-launch event timing (profile.cu,
// sweep_api.cu).
void note_launches(int k);
void* profile_begin(int kernel, cudaStream_t st);
void profile_end(void* token, cudaStream_t st);

__device__ __forceinline__ void latch(int* status, int code) {
  atomicCAS(status, 0, code);
}

}  // namespace sweep
