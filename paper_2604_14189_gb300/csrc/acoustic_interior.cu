// Stencil kernels of the acoustic step: the plain 8th-order update of every
// cell of the padded grid (forward), and the fused adjoint + reconstruction
// + imaging update (backward).  The CPML terms of both axes, the receivers
// and the boundary ring are handled afterwards by the step's second kernel
// (acoustic_cpml.cu).  See acoustic_common.cuh for the equations.
//
// Work is a list of (tile, shot) units taken round-robin by persistent CTAs
// (one per SM; a launch that carries several problems shares its one wave
// of CTAs out among them in proportion to their units, each CTA serving one
// problem).  Each CTA runs a multi-stage TMA pipeline: while it computes
// unit k from shared memory, the tiles of the next units are in flight
// (cp.async.bulk.tensor, completion on one mbarrier per stage).  Halo tiles
// carry 4 extra cells per side; the TMA zero-fills outside the padded grid,
// which is the Dirichlet condition.  A warp covers the 128-cell tile width
// (4 cells per lane, 16-byte shared-memory reads), walks its rows with a
// register window for the z stencil, and stores results with 16-byte global
// stores.
#include <algorithm>

#include "acoustic_stencil.cuh"

namespace sweep {
namespace {

template <int NP>
__global__ void __launch_bounds__(FWD_THREADS, 1)
    ac_in_fwd_kernel(const __grid_constant__ StepBatch<AcInFwdArgs, NP> m) {
  int bx, G;  // this CTA's index and the CTA count of its problem
  const AcInFwdArgs& a = m.p[step_problem(m, &bx, &G)];
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ ShotTable T;
  __shared__ UnitDesc desc[kMaxStages];
  __shared__ UnitDesc utab[kUnitTable];
  const StepCtl c{a.n, 0, 0, 0};
  if (a.bz == IN_BZ_SMALL)  // uniform over the CTA: one problem per CTA
    fwd_body<IN_BZ_SMALL, true>(a, c, bx, G, T, desc, utab, smem_raw);
  else
    fwd_body<IN_BZ, true>(a, c, bx, G, T, desc, utab, smem_raw);
}

template <int NP, bool INJ>
__global__ void __launch_bounds__(BWD_THREADS, 1)
    ac_in_bwd_kernel(const __grid_constant__ StepBatch<AcInBwdArgs, NP> m) {
  int bx, G;  // this CTA's index and the CTA count of its problem
  const AcInBwdArgs& a = m.p[step_problem(m, &bx, &G)];
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ ShotTable T;
  __shared__ UnitDesc desc[kMaxStages];
  __shared__ UnitDesc utab[kUnitTable];
  const StepCtl c{a.n, a.do_adj, a.do_img, a.do_rec};
  if (a.bz == IN_BZ_SMALL)  // uniform over the CTA: one problem per CTA
    bwd_body<IN_BZ_SMALL, true, INJ>(a, c, bx, G, T, desc, utab, smem_raw);
  else
    bwd_body<IN_BZ, true, INJ>(a, c, bx, G, T, desc, utab, smem_raw);
}

// Receiver lists of the backward units, one block per shot: for each tile
// (in chunks of the block's threads) the count of the shot's receivers in it,
// an exclusive scan over the tiles, then each tile's receivers in receiver
// order.  Every receiver lies in exactly one tile, so shot s's entries fill
// rlist[s nrec, (s + 1) nrec).
constexpr int kRecThreads = 256;
__global__ void __launch_bounds__(kRecThreads) rec_tiles_kernel(const Geom g,
                                                                const int32_t* rec, int bz,
                                                                int ntx, int2* rtile,
                                                                int4* rlist) {
  __shared__ int scan[kRecThreads];
  const int s = blockIdx.x, S = g.nshot;
  const int ntz = (g.NZ + bz - 1) / bz, T = ntz * ntx;
  const int32_t* r = rec + 2 * (size_t)s * g.nrec;
  int carry = 0;
  for (int t0 = 0; t0 < T; t0 += kRecThreads) {
    const int t = t0 + threadIdx.x;
    const int z0 = (t / ntx) * bz, x0 = (t % ntx) * IN_BX;
    int cnt = 0;
    if (t < T)
      for (int i = 0; i < g.nrec; ++i) {
        const int rz = r[2 * i] + g.P, rx = r[2 * i + 1] + g.P;
        cnt += rz >= z0 && rz < z0 + bz && rx >= x0 && rx < x0 + IN_BX;
      }
    scan[threadIdx.x] = cnt;
    __syncthreads();
    for (int d = 1; d < kRecThreads; d <<= 1) {  // inclusive scan
      const int v = threadIdx.x >= d ? scan[threadIdx.x - d] : 0;
      __syncthreads();
      scan[threadIdx.x] += v;
      __syncthreads();
    }
    const int off = s * g.nrec + carry + scan[threadIdx.x] - cnt;
    if (t < T) {
      rtile[(size_t)t * S + s] = make_int2(off, cnt);
      int k = 0;
      for (int i = 0; i < g.nrec && k < cnt; ++i) {
        const int rz = r[2 * i] + g.P, rx = r[2 * i + 1] + g.P;
        if (rz >= z0 && rz < z0 + bz && rx >= x0 && rx < x0 + IN_BX)
          rlist[off + k++] = make_int4(i, rz, rx, 0);
      }
    }
    carry += scan[kRecThreads - 1];
    __syncthreads();  // scan[] reused by the next chunk
  }
}

}  // namespace

void launch_rec_tiles(const Geom& g, const int32_t* rec, int bz, int ntx, int2* rtile,
                      int4* rlist, cudaStream_t st) {
  if (g.nshot <= 0 || g.nrec <= 0) return;
  rec_tiles_kernel<<<g.nshot, kRecThreads, 0, st>>>(g, rec, bz, ntx, rtile, rlist);
}

int device_sms() {
  static const int n = [] {  // thread-safe one-time initialisation
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
  }();
  return n;
}

template <int NP>
void set_fwd_attr() {
  static const bool attr = [] {  // thread-safe one-time initialisation
    cudaFuncSetAttribute(ac_in_fwd_kernel<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kFwdSmem);
    return true;
  }();
  (void)attr;
}
template <int NP, bool INJ>
void set_bwd_attr() {
  static const bool attr = [] {  // thread-safe one-time initialisation
    cudaFuncSetAttribute(ac_in_bwd_kernel<NP, INJ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kBwdSmem);
    return true;
  }();
  (void)attr;
}

void launch_ac_in_fwd(const AcInFwdArgs& a, cudaStream_t st) {
  if (a.units <= 0) return;
  set_fwd_attr<1>();
  int grid = device_sms();
  if (grid > a.units) grid = a.units;
  StepBatch<AcInFwdArgs, 1> m;
  m.p[0] = a;
  void* tok = profile_begin(SWEEP_K_AC_FWD_IN, st);
  launch_dependent(ac_in_fwd_kernel<1>, dim3(grid), dim3(FWD_THREADS), kFwdSmem, st, m);
  profile_end(tok, st);
  note_launches(1);
}

void launch_ac_in_bwd(const AcInBwdArgs& a, cudaStream_t st) {
  if (a.units <= 0) return;
  const bool inj = a.rtile != nullptr;
  if (inj)
    set_bwd_attr<1, true>();
  else
    set_bwd_attr<1, false>();
  int grid = device_sms();
  if (grid > a.units) grid = a.units;
  StepBatch<AcInBwdArgs, 1> m;
  m.p[0] = a;
  void* tok = profile_begin(SWEEP_K_AC_BWD_IN, st);
  launch_dependent(inj ? ac_in_bwd_kernel<1, true> : ac_in_bwd_kernel<1, false>, dim3(grid),
                   dim3(BWD_THREADS), kBwdSmem, st, m);
  profile_end(tok, st);
  note_launches(1);
}

// Several problems in one launch: the persistent CTAs (one wave, one per
// SM) are shared out in proportion to the problems' cells (units x tile
// rows: a 16-row unit is half the work of a 32-row one), at least one per
// problem with work and never more than its units.
int split_ctas(int units, long long cells, long long total) {
  if (units <= 0) return 0;
  const long long c = (long long)device_sms() * cells / total;
  return (int)std::max(1LL, std::min<long long>(c, units));
}

template <typename Args, typename K>
void launch_in_batch(K kernel, const Args* a, int np, int threads, size_t smem,
                     cudaStream_t st) {
  StepBatch<Args, kStepBatch> m;
  long long total = 0;
  for (int i = 0; i < np; ++i) total += (long long)std::max(a[i].units, 0) * a[i].bz;
  if (total <= 0) return;
  m.start[0] = 0;
  for (int i = 0; i < kStepBatch; ++i) {
    int c = 0;
    if (i < np) {
      m.p[i] = a[i];
      c = split_ctas(a[i].units, (long long)std::max(a[i].units, 0) * a[i].bz, total);
    }
    m.start[i + 1] = m.start[i] + c;
  }
  launch_dependent(kernel, dim3(m.start[kStepBatch]), dim3(threads), smem, st, m);
  note_launches(1);
}

void launch_ac_in_fwd_batch(const AcInFwdArgs* a, int np, cudaStream_t st) {
  if (np <= 0) return;
  if (np > kStepBatch) return;  // the caller splits larger groups
  set_fwd_attr<kStepBatch>();
  launch_in_batch(ac_in_fwd_kernel<kStepBatch>, a, np, FWD_THREADS, kFwdSmem, st);
}

void launch_ac_in_bwd_batch(const AcInBwdArgs* a, int np, cudaStream_t st) {
  if (np <= 0) return;
  if (np > kStepBatch) return;
  bool inj = false;  // deterministic mode: the stencil kernel injects the residual
  for (int i = 0; i < np; ++i) inj = inj || a[i].rtile != nullptr;
  if (inj) {
    set_bwd_attr<kStepBatch, true>();
    launch_in_batch(ac_in_bwd_kernel<kStepBatch, true>, a, np, BWD_THREADS, kBwdSmem, st);
  } else {
    set_bwd_attr<kStepBatch, false>();
    launch_in_batch(ac_in_bwd_kernel<kStepBatch, false>, a, np, BWD_THREADS, kBwdSmem, st);
  }
}

}  // namespace sweep
