// Second kernel of the acoustic time step: CPML terms and receivers.
//
// The stencil kernels (acoustic_interior.cu) update every cell of the padded
// grid as if there were no absorbing layer.  The convolutional-PML terms are
// additive per axis, and they read only the step's inputs (u^n or mu^{n+1}
// and the memory variables), never the stencil kernel's output.  So one
// kernel adds both axes' terms, and the receiver work, to the output field
// with vector reductions (red.global.add): its z part, x part and receiver
// part run concurrently, and a cell in a corner of the border simply gets
// two additions.  See acoustic_common.cuh for the full update:
//
// forward, axis strip cells (sigma != 0 along that axis):
//   W = D2 u^n + D1 psi^{n-1};  zeta^n = a zeta^{n-1} + b W;
//   psi^n = a psi^{n-1} + b D1 u^n;  u^{n+1} += K (D1 psi^{n-1} + zeta^n)
//   receivers: d[n] = u^{n+1}(r) (interior cells: no CPML term reaches them)
//   boundary save: the ring cells of u^n into their slot (gradient mode)
// backward, strip cells and the 4 cells next to them:
//   C = b (mu^{n+1} + zetabar^n),  B = b psibar^n   (zero off the strip)
//   mu^n += K (D2 C - D1 B)
//   strip cells: psibar^{n-1} = a psibar^n - D1 (m (mu^{n+1} + C)),
//                zetabar^{n-1} = a (mu^{n+1} + zetabar^n)
//   receivers: mu^n(r) += K(r) res^{n-1}(r)
//   ring restore: u^{n-1} on the ring from the forward save (gradient mode)
//
// The profiles a, b are zero off the border, and so are psi, zeta and their
// adjoints (never written there), which removes most masks.
//
// z part: a thread owns a column (coalesced across the warp) and a chunk of
// ZCH_F / ZCH_B rows; x part: a thread owns 4 consecutive
// cells of a row (16-byte accesses) and reads its 4 + 4 x-neighbours as two
// more 16-byte loads.  Every load of a thread is issued before its
// arithmetic, so the memory latency is paid once per thread.
#include <algorithm>

#include "acoustic_cpml.cuh"

namespace sweep {
namespace {

template <int NP, bool OWN>
__global__ void __launch_bounds__(FT, 8)
    ac_fix_fwd_kernel(const __grid_constant__ StepBatch<AcFixArgs, NP> m) {
  extern __shared__ __align__(128) unsigned char smem_raw[];  // z blocks' windows
  int blk, nblk;  // this block's index and the block count of its problem
  const AcFixArgs& a = m.p[step_problem(m, &blk, &nblk)];
  grid_dep_trigger();
  const int bps = a.nbz + a.nbx + a.nbr + a.nbs;
  const int s = blk / bps;
  int b = blk - s * bps;
  // The z and x parts read only the step's inputs (the previous step's
  // fields, complete before the stencil kernel of this step started) and
  // write memory variables nothing else touches during the step; they wait
  // for the stencil kernel only before adding into its output.
  if (b < a.nbz + a.nbx) {
    if (b < a.nbz) {  // (the status test is made uniform: the block syncs inside)
      if (!__syncthreads_or(threadIdx.x == 0 && *a.status != 0))
        fwd_z_staged<OWN>(a, s, b, smem_raw);
    } else if (!*a.status) {
      fwd_x<true, OWN>(a, s, b - a.nbz);
    }
    // One thread always waits, so that this kernel never completes before
    // the stencil kernel does (the next step's kernels rely on that order).
    if (blockIdx.x == 0 && threadIdx.x == 0) grid_dep_wait();
    return;
  }
  grid_dep_wait();
  if (*a.status) return;
  b -= a.nbz + a.nbx;
  if (b < a.nbr) {
    fwd_rec(a, s, b);
    return;
  }
  fwd_ring(a, s, b - a.nbr);
}

template <int NP, bool OWN>
__global__ void __launch_bounds__(FT, 7)
    ac_fix_bwd_kernel(const __grid_constant__ StepBatch<AcFixArgs, NP> m) {
  int blk, nblk;  // this block's index and the block count of its problem
  const AcFixArgs& a = m.p[step_problem(m, &blk, &nblk)];
  grid_dep_trigger();
  const int bps = a.nbz + a.nbx + a.nbr + a.nbs;
  const int s = blk / bps;
  int b = blk - s * bps;
  // The z and x parts read only the step's inputs (the previous step's
  // fields, complete before the stencil kernel of this step started) and
  // write memory variables nothing else touches during the step; they wait
  // for the stencil kernel only before adding into its output.
  if (b < a.nbz + a.nbx) {
    if (!*a.status) {
      if (b < a.nbz)
        bwd_z<true, OWN>(a, s, b);
      else
        bwd_x<true, OWN>(a, s, b - a.nbz);
    }
    // One thread always waits, so that this kernel never completes before
    // the stencil kernel does (the next step's kernels rely on that order).
    if (blockIdx.x == 0 && threadIdx.x == 0) grid_dep_wait();
    return;
  }
  grid_dep_wait();
  if (*a.status) return;
  b -= a.nbz + a.nbx;
  if (b < a.nbr) {  // (no receiver part in deterministic mode)
    bwd_rec(a, s, b);
    return;
  }
  bwd_ring(a, s, b - a.nbr);
}

}  // namespace

// Work split of one problem's step (blocks per shot of each part); returns
// the blocks per shot, 0 when the step has no CPML, receiver or ring work.
int fix_fwd_split(AcFixArgs& a) {
  const Geom& g = a.g;
  if (g.nshot <= 0) return 0;
  a.zbx = cdiv(g.NX, FT);
  a.nchz = g.P > 0 ? 2 * cdiv(g.P, ZCH_F) : 0;
  a.xb = x_bands(g.P, g.P + g.nx, g.NX);
  a.nbz = a.zbx * a.nchz;
  a.nbx = (g.P > 0 && a.xb.ngr > 0) ? cdiv(g.NZ * a.xb.ngr, FT) : 0;
  a.nbr = (a.data && g.nrec > 0) ? cdiv(g.nrec, FT) : 0;
  a.nbs = (a.save && g.nring > 0) ? cdiv(cdiv(g.nring, 4), FT) : 0;
  return a.nbz + a.nbx + a.nbr + a.nbs;
}

int fix_bwd_split(AcFixArgs& a) {
  const Geom& g = a.g;
  if (g.nshot <= 0) return 0;
  const int lo_end = band_lo_end(g.P, g.NZ), hi_start = band_hi_start(g.P, g.nz, g.NZ);
  a.zbx = cdiv(g.NX, FT);
  a.nchz = g.P > 0 ? cdiv(lo_end, ZCH_B) + cdiv(g.NZ - hi_start, ZCH_B) : 0;
  a.xb = x_bands(band_lo_end(g.P, g.NX), band_hi_start(g.P, g.nx, g.NX), g.NX);
  a.nbz = a.zbx * a.nchz;
  a.nbx = (g.P > 0 && a.xb.ngr > 0) ? cdiv(g.NZ * a.xb.ngr, FT) : 0;
  // deterministic mode: the stencil kernel injects the residual
  a.nbr = (!a.own && a.res && g.nrec > 0 && a.n >= 1) ? cdiv(g.nrec, FT) : 0;
  a.nbs = (a.save && a.uring && g.nring > 0) ? cdiv(cdiv(g.nring, 4), FT) : 0;
  return a.nbz + a.nbx + a.nbr + a.nbs;
}

void launch_ac_fix_fwd(AcFixArgs a, cudaStream_t st) {
  const int bps = fix_fwd_split(a);
  if (bps == 0) return;
  StepBatch<AcFixArgs, 1> m;
  m.p[0] = a;
  void* tok = profile_begin(SWEEP_K_AC_FWD_FR, st);
  launch_dependent(a.own ? ac_fix_fwd_kernel<1, true> : ac_fix_fwd_kernel<1, false>,
                   dim3(bps * a.g.nshot), dim3(FT), kZStageF + 16, st, m);
  profile_end(tok, st);
  note_launches(1);
}

void launch_ac_fix_bwd(AcFixArgs a, cudaStream_t st) {
  const int bps = fix_bwd_split(a);
  if (bps == 0) return;
  StepBatch<AcFixArgs, 1> m;
  m.p[0] = a;
  void* tok = profile_begin(SWEEP_K_AC_BWD_FR, st);
  launch_dependent(a.own ? ac_fix_bwd_kernel<1, true> : ac_fix_bwd_kernel<1, false>,
                   dim3(bps * a.g.nshot), dim3(FT), 0, st, m);
  profile_end(tok, st);
  note_launches(1);
}

template <int (*SPLIT)(AcFixArgs&), typename K>
void launch_fix_batch(K kernel, const AcFixArgs* a, int np, size_t smem, cudaStream_t st) {
  if (np <= 0 || np > kStepBatch) return;
  StepBatch<AcFixArgs, kStepBatch> m;
  m.start[0] = 0;
  for (int i = 0; i < kStepBatch; ++i) {
    int c = 0;
    if (i < np) {
      m.p[i] = a[i];
      c = SPLIT(m.p[i]) * m.p[i].g.nshot;  // consecutive blocks of problem i
    }
    m.start[i + 1] = m.start[i] + c;
  }
  if (m.start[kStepBatch] == 0) return;
  launch_dependent(kernel, dim3(m.start[kStepBatch]), dim3(FT), smem, st, m);
  note_launches(1);
}

// (the problems of one launch share the mode: the batched entry points
// require it)
void launch_ac_fix_fwd_batch(const AcFixArgs* a, int np, cudaStream_t st) {
  if (np <= 0) return;
  launch_fix_batch<fix_fwd_split>(a[0].own ? ac_fix_fwd_kernel<kStepBatch, true>
                                           : ac_fix_fwd_kernel<kStepBatch, false>,
                                  a, np, kZStageF + 16, st);
}

void launch_ac_fix_bwd_batch(const AcFixArgs* a, int np, cudaStream_t st) {
  if (np <= 0) return;
  launch_fix_batch<fix_bwd_split>(a[0].own ? ac_fix_bwd_kernel<kStepBatch, true>
                                           : ac_fix_bwd_kernel<kStepBatch, false>,
                                  a, np, 0, st);
}

}  // namespace sweep
