// Time-loop kernels of the acoustic engine: every step of a direction
// (forward, or backward) of up to kStepBatch problems in one launch.
//
// The per-step path launches two kernels per step (acoustic_interior.cu,
// acoustic_cpml.cu).  Here one cooperative launch with one CTA per SM runs
// the same work, per step:
//
//   stencil phase   the CTAs are shared out among the problems that have
//                   the step, in proportion to their cells (one CTA at
//                   least each); a CTA runs the stencil body of its problem
//                   over its units (TMA pipeline, as in the per-step kernel)
//   grid barrier
//   CPML phase      the CPML, receiver and ring work of every problem, as
//                   FT-thread slices of the CTAs over the per-step kernel's
//                   blocks (coherent loads: the fields change within the
//                   launch)
//   grid barrier
//
// The barrier is a counter and a generation word in global memory: a CTA's
// thread 0 fences, reads the generation, adds one arrival; the last arrival
// resets the counter and publishes the next generation (release), the
// others spin on it (acquire).  Every spin is bounded by the global timer:
// a CTA that gives up (or whose stencil body lost a transfer) sets the
// abort word, latches SWEEP_ETIMEOUT in every problem's status and leaves,
// and the other CTAs leave at their next barrier.  All CTAs are resident at
// once (cooperative launch, after an occupancy check), so a barrier is only
// left by timeout if something else is broken.
#include <algorithm>

#include "acoustic_cpml.cuh"
#include "acoustic_stencil.cuh"

namespace sweep {
namespace {

// 2 s: a phase of a time step takes microseconds; a barrier that has not
// opened by then never will.
constexpr uint64_t kBarrierLimitNs = 2000ull * 1000ull * 1000ull;

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Latches SWEEP_ETIMEOUT in every problem of the launch and sets the abort
// word (thread 0 of a CTA that leaves early).
__device__ void abort_loop(const LoopArgs& L) {
  for (int i = 0; i < L.np; ++i) latch(L.p[i]->fin[0].status, SWEEP_ETIMEOUT);
  atomicExch(L.bar + 2, 1u);
}

// Grid-wide barrier over the words bar[0..2] (arrivals, generation, abort);
// false when it gave up or a CTA aborted.  *flag: a shared-memory word.
__device__ bool grid_sync_words(unsigned* bar, int* flag) {
  __syncthreads();  // this CTA's work of the phase is done
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned gen = ld_acquire(bar + 1);
    __threadfence();  // this CTA's writes before its arrival
    const unsigned prev = atomicAdd(bar, 1u);
    if (prev == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      st_release(bar + 1, gen + 1);
    } else {
      const uint64_t t0 = global_timer_ns();
      while (ld_acquire(bar + 1) == gen) {
        if (ld_acquire(bar + 2) != 0 || global_timer_ns() - t0 > kBarrierLimitNs) {
          ok = 0;
          break;
        }
      }
    }
    if (!ok) atomicExch(bar + 2, 1u);
    __threadfence();  // the other CTAs' writes before this CTA's reads
    *flag = ok;
  }
  __syncthreads();
  return *flag != 0;
}

// The loop's barrier: on failure every problem's status gets SWEEP_ETIMEOUT.
__device__ bool grid_sync(const LoopArgs& L, int* flag) {
  if (grid_sync_words(L.bar, flag)) return true;
  if (threadIdx.x == 0) abort_loop(L);
  return false;
}

// The tensor maps of the loop's problems were written to global memory by
// an earlier kernel: make them visible to this thread's TMA (tensormap
// proxy) before its first copy.
__device__ void acquire_maps(const LoopArgs& L, bool fwd) {
  for (int i = 0; i < L.np; ++i)
    for (int k = 0; k < 2; ++k) {
      if (fwd) {
        const AcInFwdArgs& a = L.p[i]->fin[k];
        fence_tensormap_acquire(&a.tu);
        fence_tensormap_acquire(&a.tup);
        fence_tensormap_acquire(&a.tK);
      } else {
        const AcInBwdArgs& a = L.p[i]->bin[k];
        fence_tensormap_acquire(&a.tuA);
        fence_tensormap_acquire(&a.tmA);
        fence_tensormap_acquire(&a.tuB);
        fence_tensormap_acquire(&a.tmB);
        fence_tensormap_acquire(&a.tK);
        fence_tensormap_acquire(&a.tG);
      }
    }
}

// Stencil phase of a step: the CTA range [cs[i], cs[i + 1]) of each problem
// (thread 0 computes it, identically in every CTA).  Units and tile rows of
// problem i are u[i], bz[i]; live[i] says whether it has this step.
__device__ void split_ctas_dev(int np, const int* u, const int* bz, const bool* live, int G,
                               int* cs) {
  long long W = 0;
  int nl = 0;
  for (int i = 0; i < np; ++i)
    if (live[i] && u[i] > 0) {
      W += (long long)u[i] * bz[i];
      ++nl;
    }
  int acc = 0;
  for (int i = 0; i < np; ++i) {
    cs[i] = acc;
    if (live[i] && u[i] > 0) {
      int c = 1 + (int)((long long)(G - nl) * u[i] * bz[i] / W);
      acc += c < u[i] ? c : u[i];
    }
  }
  cs[np] = acc;  // <= G: one each plus at most (G - nl) in proportion
}

// This CTA's problem in the stencil phase (-1: none) and its index and CTA
// count within the problem.
__device__ __forceinline__ int my_problem(int np, const int* cs, int* b, int* G) {
  for (int i = 0; i < np; ++i)
    if ((int)blockIdx.x >= cs[i] && (int)blockIdx.x < cs[i + 1]) {
      *b = blockIdx.x - cs[i];
      *G = cs[i + 1] - cs[i];
      return i;
    }
  return -1;
}

// Copies np CPML argument blocks into shared memory (all threads).
__device__ void copy_fix(AcFixArgs* dst, const AcFixArgs* const* src, const bool* live, int np) {
  static_assert(sizeof(AcFixArgs) % 4 == 0, "word copy");
  constexpr int W = sizeof(AcFixArgs) / 4;
  for (int t = threadIdx.x; t < np * W; t += blockDim.x) {
    const int i = t / W, w = t - i * W;
    if (live[i])
      reinterpret_cast<unsigned*>(dst + i)[w] = reinterpret_cast<const unsigned*>(src[i])[w];
  }
}

struct LoopShared {
  ShotTable T;
  UnitDesc desc[kMaxStages];
  UnitDesc utab[kUnitTable];
  int cs[kStepBatch + 1];   // stencil CTA ranges
  int vs[kStepBatch + 1];   // CPML slice ranges (blocks of the per-step kernel)
  int u[kStepBatch], bz[kStepBatch];
  bool live[kStepBatch];
  int flag;
};

// ----------------------------------------------------------------- forward
__global__ void __launch_bounds__(FWD_THREADS, 1)
    ac_loop_fwd_kernel(const __grid_constant__ LoopArgs L) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ LoopShared S;
  constexpr int NSUB = FWD_THREADS / FT;  // FT-thread slices per CTA
  const int sub = threadIdx.x / FT;
  if (threadIdx.x < L.np) {
    S.u[threadIdx.x] = L.p[threadIdx.x]->fin[0].units;
    S.bz[threadIdx.x] = L.p[threadIdx.x]->fin[0].bz;
  }
  if (threadIdx.x == 0) acquire_maps(L, true);  // thread 0 issues every copy
  __syncthreads();
  for (int n = 0; n < L.nsteps; ++n) {
    // ---- stencil phase
    if (threadIdx.x == 0) {
      for (int i = 0; i < L.np; ++i) S.live[i] = n < L.p[i]->nt;
      split_ctas_dev(L.np, S.u, S.bz, S.live, gridDim.x, S.cs);
    }
    __syncthreads();
    int b = 0, G = 1;
    const int i = my_problem(L.np, S.cs, &b, &G);
    if (i >= 0) {
      const AcInFwdArgs& a = L.p[i]->fin[n & 1];
      const StepCtl c{n, 0, 0, 0};
      const bool ok = S.bz[i] == IN_BZ_SMALL
                          ? fwd_body<IN_BZ_SMALL, false>(a, c, b, G, S.T, S.desc, S.utab, smem_raw)
                          : fwd_body<IN_BZ, false>(a, c, b, G, S.T, S.desc, S.utab, smem_raw);
      if (!ok) {  // a transfer never landed (uniform over the CTA)
        if (threadIdx.x == 0) abort_loop(L);
        return;
      }
    }
    if (!grid_sync(L, &S.flag)) return;
    // ---- CPML phase: arguments of this step in the (free) stage memory
    AcFixArgs* fx = reinterpret_cast<AcFixArgs*>(smem_raw);
    const AcFixArgs* src[kStepBatch];
    for (int k = 0; k < L.np; ++k) src[k] = &L.p[k]->ffix[n & 1];
    copy_fix(fx, src, S.live, L.np);
    __syncthreads();
    if (threadIdx.x == 0) {
      int acc = 0;
      for (int k = 0; k < L.np; ++k) {
        S.vs[k] = acc;
        if (!S.live[k]) continue;
        fx[k].n = n;
        fx[k].save = L.p[k]->fsave ? L.p[k]->fsave + n * L.p[k]->slot : nullptr;
        acc += (fx[k].nbz + fx[k].nbx + fx[k].nbr + fx[k].nbs) * fx[k].g.nshot;
      }
      S.vs[L.np] = acc;
    }
    __syncthreads();
    for (int vb = blockIdx.x * NSUB + sub; sub < NSUB && vb < S.vs[L.np];
         vb += gridDim.x * NSUB) {
      int k = 0;
      while (vb >= S.vs[k + 1]) ++k;
      const AcFixArgs& a = fx[k];
      if (*a.status) continue;
      const int bps = a.nbz + a.nbx + a.nbr + a.nbs;
      const int blk = vb - S.vs[k];
      const int s = blk / bps;
      const int p = blk - s * bps;
      if (p < a.nbz)
        fwd_z<false, false>(a, s, p);
      else if (p < a.nbz + a.nbx)
        fwd_x<false, false>(a, s, p - a.nbz);
      else if (p < a.nbz + a.nbx + a.nbr)
        fwd_rec(a, s, p - a.nbz - a.nbx);
      else
        fwd_ring(a, s, p - a.nbz - a.nbx - a.nbr);
    }
    if (!grid_sync(L, &S.flag)) return;
  }
}

// ---------------------------------------------------------------- backward
// Step t runs step n = nt - t of each problem (t = 0 .. max nt).
__global__ void __launch_bounds__(BWD_THREADS, 1)
    ac_loop_bwd_kernel(const __grid_constant__ LoopArgs L) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ LoopShared S;
  __shared__ int fixlive_any;
  constexpr int NSUB = (BWD_THREADS / FT);  // the last, partial slice sits out
  const int sub = threadIdx.x / FT;
  if (threadIdx.x < L.np) {
    S.u[threadIdx.x] = L.p[threadIdx.x]->bin[0].units;
    S.bz[threadIdx.x] = L.p[threadIdx.x]->bin[0].bz;
  }
  if (threadIdx.x == 0) acquire_maps(L, false);
  __syncthreads();
  for (int t = 0; t < L.nsteps; ++t) {
    // ---- stencil phase: adjoint, reconstruction, imaging
    if (threadIdx.x == 0) {
      for (int i = 0; i < L.np; ++i) S.live[i] = L.p[i]->nt - t >= 0;
      split_ctas_dev(L.np, S.u, S.bz, S.live, gridDim.x, S.cs);
    }
    __syncthreads();
    int b = 0, G = 1;
    const int i = my_problem(L.np, S.cs, &b, &G);
    if (i >= 0) {
      const int nt = L.p[i]->nt, n = nt - t;
      const AcInBwdArgs& a = L.p[i]->bin[n & 1];
      const StepCtl c{n, n >= 1, n <= nt - 1, n >= 1 && n <= nt - 1};
      const bool ok = S.bz[i] == IN_BZ_SMALL
                          ? bwd_body<IN_BZ_SMALL, false, false>(a, c, b, G, S.T, S.desc,
                                                                 S.utab, smem_raw)
                          : bwd_body<IN_BZ, false, false>(a, c, b, G, S.T, S.desc, S.utab,
                                                           smem_raw);
      if (!ok) {
        if (threadIdx.x == 0) abort_loop(L);
        return;
      }
    }
    if (!grid_sync(L, &S.flag)) return;
    // ---- CPML phase (steps n >= 1): CPML terms of mu^n, residual
    // injection, ring restore of u^{n-1}
    if (threadIdx.x == 0) {
      int any = 0;
      for (int k = 0; k < L.np; ++k) {
        S.live[k] = L.p[k]->nt - t >= 1;
        any |= S.live[k];
      }
      fixlive_any = any;
    }
    __syncthreads();
    if (!fixlive_any) continue;  // the last step (n = 0 everywhere): no CPML phase
    AcFixArgs* fx = reinterpret_cast<AcFixArgs*>(smem_raw);
    const AcFixArgs* src[kStepBatch];
    for (int k = 0; k < L.np; ++k) src[k] = &L.p[k]->bfix[(L.p[k]->nt - t) & 1];
    copy_fix(fx, src, S.live, L.np);
    __syncthreads();
    if (threadIdx.x == 0) {
      int acc = 0;
      for (int k = 0; k < L.np; ++k) {
        S.vs[k] = acc;
        if (!S.live[k]) continue;
        const int nt = L.p[k]->nt, n = nt - t;
        fx[k].n = n;
        if (n <= nt - 1 && fx[k].save) {  // reconstruction: restore the ring of u^{n-1}
          fx[k].save = fx[k].save + (n - 1) * L.p[k]->slot;
        } else {
          fx[k].save = nullptr;
          fx[k].uring = nullptr;
          fx[k].nbs = 0;
        }
        acc += (fx[k].nbz + fx[k].nbx + fx[k].nbr + fx[k].nbs) * fx[k].g.nshot;
      }
      S.vs[L.np] = acc;
    }
    __syncthreads();
    for (int vb = blockIdx.x * NSUB + sub; sub < NSUB && vb < S.vs[L.np];
         vb += gridDim.x * NSUB) {
      int k = 0;
      while (vb >= S.vs[k + 1]) ++k;
      const AcFixArgs& a = fx[k];
      if (*a.status) continue;
      const int bps = a.nbz + a.nbx + a.nbr + a.nbs;
      const int blk = vb - S.vs[k];
      const int s = blk / bps;
      const int p = blk - s * bps;
      if (p < a.nbz)
        bwd_z<false, false>(a, s, p);
      else if (p < a.nbz + a.nbx)
        bwd_x<false, false>(a, s, p - a.nbz);
      else if (p < a.nbz + a.nbx + a.nbr)
        bwd_rec(a, s, p - a.nbz - a.nbx);
      else
        bwd_ring(a, s, p - a.nbz - a.nbx - a.nbr);
    }
    if (!grid_sync(L, &S.flag)) return;
  }
}

// Diagnostic: CTA 1 leaves without arriving (a barrier nobody completes),
// so CTA 0's barrier runs out after kBarrierLimitNs and latches
// SWEEP_ETIMEOUT.  Nothing else is touched.
__global__ void barrier_timeout_kernel(unsigned* bar, int* status) {
  __shared__ int flag;
  if (blockIdx.x != 0) return;
  if (!grid_sync_words(bar, &flag) && threadIdx.x == 0) latch(status, SWEEP_ETIMEOUT);
}

// One LoopProblem copied from the launch parameters into device memory.
__global__ void loop_install_kernel(const __grid_constant__ LoopProblem h, LoopProblem* d) {
  static_assert(sizeof(LoopProblem) % 4 == 0, "word copy");
  const unsigned* s = reinterpret_cast<const unsigned*>(&h);
  unsigned* o = reinterpret_cast<unsigned*>(d);
  for (int w = threadIdx.x; w < (int)(sizeof(LoopProblem) / 4); w += blockDim.x) o[w] = s[w];
}

// `attr`: the kernel's own one-time shared-memory attribute result (both
// kernels have the same type, so it cannot be a static of this function).
int launch_loop(void (*kernel)(LoopArgs), bool attr, const LoopArgs& a, int threads,
                size_t smem, cudaStream_t st) {
  if (!attr) return SWEEP_ECUDA;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) !=
      cudaSuccess)
    return SWEEP_ECUDA;
  const int grid = device_sms();
  if (per_sm < 1 || grid < a.np) return SWEEP_EUNSUPPORTED;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);  // one CTA per SM: all resident
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, kernel, a) != cudaSuccess) return SWEEP_ECUDA;
  note_launches(1);
  return SWEEP_OK;
}

}  // namespace

void launch_loop_install(const LoopProblem& h, LoopProblem* d, cudaStream_t st) {
  loop_install_kernel<<<1, 256, 0, st>>>(h, d);
  note_launches(1);
}

int launch_ac_loop_fwd(const LoopArgs& a, cudaStream_t st) {
  static_assert(kStepBatch * sizeof(AcFixArgs) <= FwdTile<IN_BZ>::SMEM, "CPML arguments");
  static const bool attr =  // thread-safe one-time initialisation
      cudaFuncSetAttribute(ac_loop_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kFwdSmem) == cudaSuccess;
  return launch_loop(ac_loop_fwd_kernel, attr, a, FWD_THREADS, kFwdSmem, st);
}

int launch_barrier_timeout_check(unsigned* bar, int* status, cudaStream_t st) {
  if (cudaMemsetAsync(bar, 0, sizeof(unsigned) * 4, st) != cudaSuccess) return SWEEP_ECUDA;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2);  // both resident (cooperative)
  cfg.blockDim = dim3(32);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, barrier_timeout_kernel, bar, status) != cudaSuccess)
    return SWEEP_ECUDA;
  note_launches(1);
  return SWEEP_OK;
}

int launch_ac_loop_bwd(const LoopArgs& a, cudaStream_t st) {
  static_assert(kStepBatch * sizeof(AcFixArgs) <= BwdTile<IN_BZ>::SMEM, "CPML arguments");
  static const bool attr =
      cudaFuncSetAttribute(ac_loop_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kBwdSmem) == cudaSuccess;
  return launch_loop(ac_loop_bwd_kernel, attr, a, BWD_THREADS, kBwdSmem, st);
}

}  // namespace sweep
