// Internal declarations of the elastic engine (elastic.cu,
// elastic_adjoint.cu), used by the entry points in sweep_api.cu.
#pragma once

#include "sweep_internal.cuh"

namespace sweep {

// ------------------------------------------------------------------- elastic
// Coefficients on the padded grid [NZ][NXp], pre-scaled by dt / dx:
// cbx, cbz = buoyancy at vx / vz points; cl2m = lambda + 2 mu, clam = lambda
// at normal-stress points; cmu = mu at txz points.
struct ElParamArgs {
  Geom g;
  const float* model;  // [3][nz][nx] (vp, vs, rho) or padded
  int padded;
  float dx, dt;
  float* cbx;
  float* cbz;
  float* cl2m;
  float* clam;
  float* cmu;
};

struct ElStepArgs {
  Geom g;
  // state before the step: fields [S][NZ][NXp] and CPML memory variables
  float *vx, *vz, *txx, *tzz, *txz;
  float *p1, *p2, *p3, *p4;                // velocity CPML memory variables
  float *p5, *p6, *p7, *p8;                // stress CPML memory variables
  // state after the step (the same buffers for an in-place step; the
  // gradient's replay writes each step's state into its own slot).  A
  // memory variable is written on the tiles that meet its strip only.
  float *vx_o, *vz_o, *txx_o, *tzz_o, *txz_o;
  float *p1_o, *p2_o, *p3_o, *p4_o, *p5_o, *p6_o, *p7_o, *p8_o;
  const float *cbx, *cbz, *cl2m, *clam, *cmu;
  const float *ax, *bx, *axh, *bxh;        // x profiles (integer, half points)
  const float *az, *bz, *azh, *bzh;        // z profiles
  const float* wavelet;
  const int32_t* src;
  const int32_t* rec;
  float* data;                             // [S][2][R][nt] or null
  float src_scale;                         // dt / dx^2
  int* status;
  int n;
  // TMA descriptors (built by el_step_maps): stress fields before the step
  // with the halos the velocity kernel needs, velocities after it (read by
  // the stress kernel) with both halos, coefficients
  CUtensorMap m_txx, m_txz, m_tzz, m_vx, m_vz;
  CUtensorMap m_cbx, m_cbz, m_l2m, m_lam, m_mu;
  int units, ntx;  // (tile, shot) units of the persistent kernels
};
void launch_el_params(const ElParamArgs& a, cudaStream_t st);
// Fills the descriptors and the unit count of `a` (false on a driver error).
bool el_step_maps(ElStepArgs& a);
void launch_el_step(const ElStepArgs& a, cudaStream_t st);

// Elastic adjoint step (elastic_adjoint.cu): the transpose of one
// ElStepArgs step, run backwards in time.  Adjoint state (vx, vz, txx, tzz,
// txz) in av*, at*; adjoint memory variables p1..p8 read from ap_in and
// written to ap_out (two buffers, swapped by the caller every step).  With
// gacc non-null the step also adds d J / d (cl2m, clam, cmu, cbx, cbz) to
// the accumulators gacc [ngrp][5][2][NZ][NXp]: compensated FP32 sums (hi,
// lo planes; shot group q's shots, in shot order, into block q), from the
// forward state: fvx, fvz = v^{n+1/2} and fp = p1..p8 after step n, ft* =
// tau^n (before the step).
struct ElAdjArgs {
  Geom g;
  float *avx, *avz, *atxx, *atzz, *atxz;
  const float* ap_in[8];
  float* ap_out[8];
  const float *fvx, *fvz, *ftxx, *ftzz, *ftxz;
  const float* fp[8];
  float* gacc;
  const float *cbx, *cbz, *cl2m, *clam, *cmu;
  const float *ax, *bx, *axh, *bxh, *az, *bz, *azh, *bzh;
  const float* res;     // [S][2][R][nt] injected at the receivers, or null
  const int32_t* src;
  const int32_t* rec;
  float* wgrad;         // [S][nt] wavelet adjoint, or null
  float src_scale;      // dt / dx^2
  const int* status;
  int n;
  // TMA descriptors (el_adj_maps; the forward state's by el_adj_forward_maps
  // whenever fvx .. ftxz change): boxes of a tile +- 2 rows and +- 4 columns
  CUtensorMap m_atxx, m_atzz, m_atxz, m_avx, m_avz;
  CUtensorMap m_fvx, m_fvz, m_ftxx, m_ftzz, m_ftxz;
  CUtensorMap m_l2m, m_lam, m_mu, m_cbx, m_cbz;
  int sg, ngrp;       // shots per group, groups
  int units, ntx;     // (tile, group) units of the persistent kernels
};
// Shots per group of the adjoint kernels for this geometry (the workspace
// holds ceil(nshot / group) accumulator blocks).
int el_adj_shot_group(const Geom& g);
// Fill the descriptors of the adjoint state and coefficients and the unit
// counts (false on a driver error); el_adj_forward_maps: those of the
// forward state fvx, fvz, ftxx, ftzz, ftxz.
bool el_adj_maps(ElAdjArgs& a);
bool el_adj_forward_maps(ElAdjArgs& a);
void launch_el_adj_step(const ElAdjArgs& a, cudaStream_t st);
// d J / d (vp, vs, rho) on interior cells, [3][nz][nx], from the
// coefficient adjoints (summed over the groups in FP64); padding held fixed.
void launch_el_grad(const Geom& g, const float* gacc, int ngrp, const float* model, int padded,
                    float dx, float dt, float* grad, const int* status, cudaStream_t st);

}  // namespace sweep
