// Internal declarations of the GB300 solver library (CUDA side only).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "sweep.h"

namespace sweep {

// Rectangle [z0, z1) x [x0, x1) of the padded grid (empty if z1 <= z0 or
// x1 <= x0).
struct Region {
  int z0, z1, x0, x1;
};

// ---------------------------------------------------------------------------
// Geometry of one problem on the padded grid.
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
  // Cells covered by the plain-stencil kernels (forward, backward): the
  // whole padded grid; the CPML correction kernels then add the border terms.
  Region fin, bin;
};

// ------------------------------------------------------------------ interior
// Tiles of bz rows x IN_BX cells, bz = IN_BZ (the default) or IN_BZ_SMALL
// (chosen per problem: more units for small grids, see SWEEP_F_ROWS16);
// each warp owns a band of rows, each lane 4 consecutive cells of a row.
// Halo tiles are IN_HW wide and 8 rows taller.
constexpr int IN_BX = 128;
constexpr int IN_BZ = 32;
constexpr int IN_BZ_SMALL = 16;
constexpr int IN_HW = IN_BX + 8;  // halo tile width

struct AcInFwdArgs {
  Geom g;
  CUtensorMap tu;    // u^n, halo box     [S][NZ][NX]
  CUtensorMap tup;   // u^{n-1}, centre box
  CUtensorMap tK;    // K [NZ][NX], centre box
  float* un;         // out u^{n+1} (the u^{n-1} buffer)
  const float* wavelet;
  const int32_t* src;
  int* status;
  int n;
  int units, ntx;       // (tile, shot) units; tiles along x
  int bz;               // tile rows: IN_BZ or IN_BZ_SMALL
};

struct AcInBwdArgs {
  Geom g;
  CUtensorMap tuA;   // u^n, halo box
  CUtensorMap tmA;   // mu^{n+1}, halo box
  CUtensorMap tuB;   // u^{n+1}, centre box
  CUtensorMap tmB;   // mu^{n+2}, centre box
  CUtensorMap tK;
  CUtensorMap tG;    // imaging accumulator graw, centre box
  float* uB;         // out u^{n-1}
  float* mB;         // out mu^n
  float* graw;       // [S][NZ][NXp]
  float* illum;      // [S][NZ][NXp] or null
  const float* wavelet;
  const int32_t* src;
  float* wgrad;      // [S][nt] or null
  // receiver injection mu^n(r) += K(r) res^{n-1}(r), done by the stencil
  // kernel while it forms mu^n (so that each cell has one writer per
  // phase): per (tile, shot) unit its receivers' (offset, count) in rlist,
  // entries (receiver index, z, x) in padded coordinates, receiver order.
  // Null when there is no residual.
  const float* res;  // [S][nrec][nt]
  const int2* rtile; // [units]
  const int4* rlist; // [S * nrec]
  int* status;
  int n;
  int do_adj, do_img, do_rec;
  int units, ntx;
  int bz;            // tile rows: IN_BZ or IN_BZ_SMALL
};

// Second kernel of an acoustic time step (acoustic_cpml.cu): the CPML terms
// of both axes and the receiver work, all added to the step's output field
// with vector reductions (red.global.add), so the parts run concurrently.
// Forward: u = u^n, un = u^{n+1}, p*in/p*out = psi^{n-1}/psi^n, zeta updated
// in place (z*out == z*in), data = recorded traces (d[n] = u^{n+1}(r)),
// save = ring slot that receives the ring cells of u^n (gradient mode).
// Backward: u = mu^{n+1}, un = mu^n, p*in/p*out = psibar^n/^{n-1},
// z*in/z*out = zetabar^n/^{n-1}, res = residual injected at the receivers
// (mu^n(r) += K(r) res[n-1]; in deterministic mode the backward stencil
// kernel injects it instead), save/uring = ring restore of u^{n-1}.
// own: deterministic mode (one owner per border cell).
// Rows per z-part chunk of the CPML kernels (forward, backward): chosen by
// a sweep on GB300; the forward z part's staged copies are 4 rows taller
// each way.
constexpr int ZCH_FWD = 8;
constexpr int ZCH_BWD = 4;

struct XBands {  // 4-cell column groups: left [0, gl), right [gr0, ceil(NX/4))
  int gl, gr0, ngr;
};
struct AcFixArgs {
  // forward z part of the per-step kernel: each block copies its chunk's
  // row windows into shared memory (TMA, zero outside the grid): u^n and
  // psi_z with 4 rows above and below the chunk, zeta_z and K on the chunk's
  // rows; boxes of 128 columns
  CUtensorMap tzu, tzp, tzz, tzK;
  Geom g;
  const float* u;
  float* un;
  const float* K;
  const float* pzin;
  float* pzout;
  float* zzin;
  float* zzout;
  const float* pxin;
  float* pxout;
  float* zxin;
  float* zxout;
  const float* ax;
  const float* bx;
  const float* az;
  const float* bz;
  const int32_t* rec;
  float* data;
  const float* res;  // backward: residual injected here (null: the stencil
                     // kernel injects it, deterministic mode)
  float* save;       // forward: ring slot of u^n; backward: ring slot of u^{n-1}
  float* uring;      // backward: the u^{n-1} field whose ring is restored
  const int* status;
  int n;
  // work split, set by the launcher: blocks per shot of the z, x, receiver
  // and ring parts; z part: blocks per row chunk, row chunks
  int nbz, nbx, nbr, nbs;
  int zbx, nchz;
  XBands xb;
  int own;
};
void launch_ac_fix_fwd(AcFixArgs a, cudaStream_t st);
void launch_ac_fix_bwd(AcFixArgs a, cudaStream_t st);
// np <= kStepBatch problems in one launch (consecutive block ranges)
void launch_ac_fix_fwd_batch(const AcFixArgs* a, int np, cudaStream_t st);
void launch_ac_fix_bwd_batch(const AcFixArgs* a, int np, cudaStream_t st);

// Work split of one problem's CPML step (acoustic_cpml.cu): fills the part
// counts of `a` and returns the blocks per shot (0: no work).
int fix_fwd_split(AcFixArgs& a);
int fix_bwd_split(AcFixArgs& a);

// The arguments of up to NP problems for one launch of a step kernel: the
// launch's 1-D grid is split into consecutive block ranges, problem i owning
// blocks [start[i], start[i + 1]) (start[np..NP] = the grid size, unused
// entries of p are never read).
constexpr int kStepBatch = 16;
template <typename Args, int NP>
struct StepBatch {
  Args p[NP];
  int start[NP + 1];
};
// This block's problem and its block index and block count within it.
template <typename Args, int NP>
__device__ __forceinline__ int step_problem(const StepBatch<Args, NP>& m, int* b, int* nb) {
  if (NP == 1) {
    *b = blockIdx.x;
    *nb = gridDim.x;
    return 0;
  }
  int i = 0;
  while (i + 1 < NP && (int)blockIdx.x >= m.start[i + 1]) ++i;
  *b = blockIdx.x - m.start[i];
  *nb = m.start[i + 1] - m.start[i];
  return i;
}

// Kernel launchers (acoustic_interior.cu); the _batch forms launch the step
// of np <= kStepBatch problems at once, the persistent CTAs shared out in
// proportion to the problems' units
void launch_ac_in_fwd(const AcInFwdArgs& a, cudaStream_t st);
void launch_ac_in_bwd(const AcInBwdArgs& a, cudaStream_t st);
void launch_ac_in_fwd_batch(const AcInFwdArgs* a, int np, cudaStream_t st);
void launch_ac_in_bwd_batch(const AcInBwdArgs* a, int np, cudaStream_t st);
int device_sms();
// Receiver lists of the backward stencil launch's units (acoustic_interior.cu):
// for tiles of bz rows x IN_BX cells (ntx along x), unit u = tile * S + s.
void launch_rec_tiles(const Geom& g, const int32_t* rec, int bz, int ntx, int2* rtile,
                      int4* rlist, cudaStream_t st);

// Time-loop kernels (acoustic_loop.cu): one cooperative launch runs every
// forward (or backward) step of up to kStepBatch problems, each step as a
// stencil phase and a CPML phase separated by grid-wide barriers.
// LoopProblem holds one problem's arguments for the steps of either parity
// (n % 2 selects the buffers); the kernel sets the per-step scalars (n, the
// ring slot, the backward step's flags) itself.  It lives in the problem's
// workspace, written by launch_loop_install.
struct LoopProblem {
  AcInFwdArgs fin[2];   // forward stencil arguments of steps with n % 2 == k
  AcFixArgs ffix[2];    // forward CPML arguments (work split set)
  AcInBwdArgs bin[2];   // backward stencil arguments
  AcFixArgs bfix[2];    // backward CPML arguments, split for a step that
                        // restores the ring (save = slot of u^0, uring set)
  float* fsave;         // forward: ring slot of u^0 (null: no save)
  long long slot;       // floats per ring slot (nshot * nring)
  int nt;
  int pad;
};
struct LoopArgs {
  LoopProblem* p[kStepBatch];  // device copies
  int np;
  int nsteps;                  // forward: max nt; backward: max nt + 1
  unsigned* bar;               // barrier words (arrivals, generation, abort),
                               // arrivals and abort zero at launch
};
void launch_loop_install(const LoopProblem& h, LoopProblem* d, cudaStream_t st);
// SWEEP_OK, or SWEEP_EUNSUPPORTED when the grid cannot be co-resident
int launch_ac_loop_fwd(const LoopArgs& a, cudaStream_t st);
int launch_ac_loop_bwd(const LoopArgs& a, cudaStream_t st);
// Diagnostic: a grid barrier that one CTA never reaches runs out (~2 s) and
// latches SWEEP_ETIMEOUT in *status; bar: 4 words of scratch.
int launch_barrier_timeout_check(unsigned* bar, int* status, cudaStream_t st);

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
// sweep_api.cu).  While this thread records a graph (graph.cu) neither
// counts nor times anything.
extern thread_local bool t_capturing;
void note_launches(int k);
void* profile_begin(int kernel, cudaStream_t st);
void profile_end(void* token, cudaStream_t st);

__device__ __forceinline__ void latch(int* status, int code) {
  atomicCAS(status, 0, code);
}

// Programmatic dependent launch.  A kernel started by launch_dependent may be
// scheduled while the kernel before it in the stream is still draining; it
// must call grid_dep_wait() before its first access to memory that an
// earlier kernel writes (every such kernel here calls it first thing, so the
// stream order stays transitive).  grid_dep_trigger() lets the next kernel
// be scheduled once every CTA of this one has called it or exited.
__device__ __forceinline__ void grid_dep_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void grid_dep_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline void launch_dependent(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                             cudaStream_t st, const Args&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace sweep
