/*
 * sweep.h -- C ABI of the GB300 (sm_103a) finite-difference wave solvers.
 *
 * The library implements the time-stepping hot path of SWEEP (Wang &
 * Alkhalifah, "SWEEP: A Unified Solver Framework for Differentiable Wave
 * Physics"): the Propagator / Source / Receiver modules of Sec. 2.1 for
 *   - the constant-density acoustic equation, 2nd order in time (Sec. 3.1.2,
 *     Eq. 2, stepped in the form of the Sec. 2.1 listing), 8th order in
 *     space, with a convolutional PML;
 *   - the isotropic elastic velocity-stress equations (Sec. 3.5, Eq. 12) on a
 *     staggered grid, 4th order in space, with a convolutional PML;
 * together with the exact discrete adjoint of the acoustic recurrence and the
 * FWI velocity gradient of the L2 seismogram misfit (the adjoint-state use
 * and dot-product test motivated in Sec. 1).  Batches of shots run in one
 * launch per time step (Sec. 2.2).
 *
 * Conventions (the paper fixes none of them; these are the library's):
 *   Grid      cell (z, x), row-major, x fastest, dz == dx.  The interior model
 *             [nz][nx] is edge-replicated into a border of `pml` cells per
 *             side, giving the padded grid NZ = nz + 2 pml, NX = nx + 2 pml.
 *             Fields are zero outside the padded grid.
 *   Acoustic  u^{n+1} = 2u^n - u^{n-1} + K (Lap_x + Lap_z), K = v^2 dt^2/dx^2,
 *             where inside the border each axis term is
 *             D2 u + D1 psi^{n-1} + zeta^n with
 *             psi^n = a psi^{n-1} + b D1 u^n,
 *             zeta^n = a zeta^{n-1} + b (D2 u + D1 psi^{n-1}).
 *             Source: u^{n+1}(s) += K(s) f^n.  Trace sample n = u^{n+1}(r).
 *   Elastic   vx at (z, x+1/2), vz at (z+1/2, x), txz at (z+1/2, x+1/2);
 *             explosive source txx(s), tzz(s) += dt f^n / dx^2 after the
 *             stress update of step n; trace sample n = (vx, vz)^{n+1/2}.
 *   CPML      depth d (cells) into the border, rho = d / pml,
 *             sigma = 3 vref ln(1000) / (2 pml dx) rho^2,
 *             alpha = pi f_ref (1 - rho), a = exp(-(sigma + alpha) dt),
 *             b = sigma / (sigma + alpha) (a - 1); vref = v_pml if > 0, else
 *             the largest vp of the padded model.
 *   Gradient  d misfit / d v on interior cells, padding and CPML profile held
 *             fixed.  misfit = 1/2 sum (d - d_obs)^2, reduced in FP64.
 *
 * Memory: every array argument is a DEVICE pointer; only `prob` is a host
 * pointer.  The caller owns all memory, including the workspace; the library
 * never allocates device memory.  Calls are asynchronous on `stream` (a
 * cudaStream_t, NULL = legacy default stream).
 *
 * Errors: a call returns SWEEP_OK or a negative code.  Errors visible on the
 * host (sizes, NULL pointers, workspace too small, CFL with a given v_pml) are
 * returned before any launch.  Errors that depend on device data (positions
 * out of range, non-positive or non-finite model values, the CFL limit of the
 * model's own maximum velocity, a non-finite misfit) are latched in the
 * workspace status word by the kernels, which then skip all further work of
 * that call; sweep_status() returns it.  Each call clears the status word of
 * its workspace when it starts.  One workspace must not be used by two calls
 * at once; different workspaces may be used concurrently.
 */
#ifndef SWEEP_H
#define SWEEP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { SWEEP_ACOUSTIC = 0, SWEEP_ELASTIC = 1 } sweep_physics;

typedef enum {
  SWEEP_MODE_FORWARD = 0,
  SWEEP_MODE_ADJOINT = 1,
  SWEEP_MODE_GRADIENT = 2
} sweep_mode;

/* model is passed on the padded grid [npar][NZ][NX] instead of [npar][nz][nx] */
#define SWEEP_F_PADDED_MODEL 0x1
/* sweep_gradient: d_obs holds the data residual r itself; the gradient is
 * (dd/dv)^T r and misfit = 1/2 sum r^2 */
#define SWEEP_F_RESIDUAL_IN 0x2
/* acoustic: stencil tiles of 16 rows instead of 32 (twice the work units;
 * faster for small grids that leave SMs idle with 32-row tiles).  A tuning
 * choice only: the results are identical.  Ignored for elastic physics. */
#define SWEEP_F_ROWS16 0x4
/* acoustic sweep_forward, sweep_gradient (without illumination) and the
 * batched calls: each direction's whole time loop runs as one cooperative
 * launch (one CTA per SM, grid-wide barriers between each step's stencil
 * and CPML phases, every wait bounded) instead of two launches per step.
 * The results equal the per-step path's up to the order of the CPML corner
 * additions.  A batched call's problems must all set it or all clear it
 * (else SWEEP_EINVAL); sweep_adjoint and illumination requests return
 * SWEEP_EUNSUPPORTED with it; SWEEP_EUNSUPPORTED also when the device
 * cannot hold one CTA per SM.  Ignored for elastic physics. */
#define SWEEP_F_ONE_LAUNCH 0x8
/* acoustic: bitwise reproducible results.  Every cell of the CPML border
 * gets one writer per step (the corners' two axis terms added by one
 * thread) and the backward stencil kernel injects the residual at the
 * receivers, in receiver order, so that no two additions to a cell race.
 * Costs time (about 16 % on a 301x901 + 40 gradient).  Without it, a corner
 * cell of the border and a receiver cell inside the backward band take two
 * additions in either order, and runs agree to FP32 rounding only.  Not with
 * SWEEP_F_ONE_LAUNCH (SWEEP_EUNSUPPORTED); a batched call's problems must
 * all set it or all clear it (else SWEEP_EINVAL).  Ignored for elastic
 * physics (its kernels have one writer per cell already). */
#define SWEEP_F_DETERMINISTIC 0x10

enum {
  SWEEP_OK = 0,
  SWEEP_EINVAL = -1,      /* bad size, NULL pointer, unknown physics/mode  */
  SWEEP_ECFL = -2,        /* v dt / dx above the scheme's stability limit  */
  SWEEP_EBOUNDS = -3,     /* source or receiver outside the interior grid  */
  SWEEP_EWORKSPACE = -4,  /* workspace NULL, misaligned or too small       */
  SWEEP_ECUDA = -5,       /* a CUDA runtime call failed                    */
  SWEEP_ETIMEOUT = -6,    /* a bounded device-side wait gave up            */
  SWEEP_ENONFINITE = -7,  /* non-finite model value or misfit              */
  SWEEP_EMODEL = -8,      /* non-positive velocity or density              */
  SWEEP_EUNSUPPORTED = -9, /* combination not implemented                  */
  SWEEP_ETOOBIG = -10     /* size above a fixed internal capacity          */
};

typedef struct {
  int32_t physics; /* sweep_physics                                          */
  int32_t nz, nx;  /* interior grid, cells (>= 1)                            */
  int32_t pml;     /* border width per side, cells (>= 0)                    */
  float dx;        /* grid spacing, m (> 0); dz == dx                        */
  float dt;        /* time step, s (> 0)                                     */
  int32_t nt;      /* time steps == samples per trace (>= 1)                 */
  int32_t nshot;   /* shots in the batch (>= 0)                              */
  int32_t nrec;    /* receivers per shot (>= 0)                              */
  float f_ref;     /* CPML alpha reference frequency, Hz (>= 0)              */
  float v_pml;     /* CPML reference velocity, m/s; <= 0: max vp of model    */
  int32_t flags;   /* SWEEP_F_*; any other bit: SWEEP_EINVAL                 */
} sweep_problem;

/* Bytes of device workspace a call of `mode` needs for `prob` (0 on invalid
 * input).  The workspace must be 256-byte aligned. */
size_t sweep_workspace_bytes(const sweep_problem* prob, int mode);

/* Forward modelling (Sec. 2.1 Propagator + Source + Receiver; Eq. 2 or 12).
 *   model    acoustic [nz][nx] vp (m/s); elastic [3][nz][nx] = (vp, vs, rho)
 *            (m/s, m/s, kg/m^3); padded grid with SWEEP_F_PADDED_MODEL
 *   wavelet  [nshot][nt] source time function samples f^n
 *   src      [nshot][2] int32 (z, x) interior cell of each shot's source
 *   rec      [nshot][nrec][2] int32 (z, x) interior receiver cells
 *   data     out [nshot][ncomp][nrec][nt]; ncomp = 1 (u) or 2 (vx, vz)   */
int sweep_forward(const sweep_problem* prob, const float* model,
                  const float* wavelet, const int32_t* src, const int32_t* rec,
                  float* data, void* ws, size_t ws_bytes, void* stream);

/* Adjoint of the linear map wavelet -> data at fixed model:
 * wavelet_grad[s][n] = sum_{c,r,m} adj_data[s][c][r][m] d data[s][c][r][m]/d f_s^n
 * (adj_data in the layout of data).  The exact transpose of the discrete
 * recurrence, run backwards in time; the dot-product test
 * <F f, d> = <f, F^T d> holds to rounding.                                 */
int sweep_adjoint(const sweep_problem* prob, const float* model,
                  const float* adj_data, const int32_t* src,
                  const int32_t* rec, float* wavelet_grad, void* ws,
                  size_t ws_bytes, void* stream);

/* FWI gradient of the L2 misfit J = 1/2 sum r^2, r = data - d_obs, with the
 * padding and the CPML profiles held fixed (set v_pml to fix the profiles).
 * Acoustic: forward with boundary saving, adjoint propagation with wavefield
 * reconstruction and the imaging condition
 * g = (2/v) sum_n mu^{n+1} (Lap u^n + f^n delta_s), mu = K lambda.
 * Elastic: forward with sqrt(nt) checkpoints, the transposed steps with each
 * checkpoint segment replayed, d J / d (vp, vs, rho) through Hooke's
 * parameters, the buoyancy averages and the harmonic shear average.
 *   d_obs    [nshot][ncomp][nrec][nt] observed data (or residual, see flags)
 *   grad     out [npar][nz][nx], summed over shots (FP64 sum, FP32 result)
 *   misfit   out device double, J (may be NULL)
 *   illum    out [nz][nx] sum over shots and steps of u^2 (may be NULL;
 *            acoustic only, SWEEP_EUNSUPPORTED for elastic)               */
int sweep_gradient(const sweep_problem* prob, const float* model,
                   const float* wavelet, const int32_t* src, const int32_t* rec,
                   const float* d_obs, float* grad, double* misfit, float* illum,
                   void* ws, size_t ws_bytes, void* stream);

/* Gradients of several acoustic problems in one call (heterogeneous batch:
 * the shot / model dimension of Sec. 2.2 with each model of its own size,
 * border, record length and shot count).  Problem i takes the arguments of
 * sweep_gradient: probs[i], models[i], wavelets[i], srcs[i], recs[i],
 * d_obs[i], grads[i], misfits[i] (device double, required) and its own
 * workspace ws[i] of ws_bytes[i] >= sweep_workspace_bytes(&probs[i],
 * SWEEP_MODE_GRADIENT) bytes (no two problems share one); no illumination.
 * The problems run in groups of up to 16 in lockstep: every time-step kernel
 * launch carries the step of each problem of the group (a problem past its
 * record length drops out), so the launches' fixed cost is shared.  Results
 * equal separate sweep_gradient calls to rounding.  Every problem is checked
 * on the host before any launch (first error returned; acoustic only, else
 * SWEEP_EUNSUPPORTED); device errors are latched in each problem's
 * workspace (sweep_status(ws[i])).  Asynchronous on `stream`. */
int sweep_gradient_batch(int nprob, const sweep_problem* probs, const float* const* models,
                         const float* const* wavelets, const int32_t* const* srcs,
                         const int32_t* const* recs, const float* const* d_obs,
                         float* const* grads, double* const* misfits, void* const* ws,
                         const size_t* ws_bytes, void* stream);

/* Forward runs of several acoustic problems in one call, the same way:
 * problem i takes the arguments of sweep_forward (probs[i], models[i],
 * wavelets[i], srcs[i], recs[i], data[i]) and its own workspace ws[i] of
 * ws_bytes[i] >= sweep_workspace_bytes(&probs[i], SWEEP_MODE_FORWARD) bytes;
 * groups of up to 16 in lockstep, each time-step launch carrying the step of
 * every problem of the group.  Checks, errors and asynchrony as
 * sweep_gradient_batch. */
int sweep_forward_batch(int nprob, const sweep_problem* probs, const float* const* models,
                        const float* const* wavelets, const int32_t* const* srcs,
                        const int32_t* const* recs, float* const* data, void* const* ws,
                        const size_t* ws_bytes, void* stream);

/* FP64 dot product sum_i a[i] b[i] of two device float arrays a, b of n
 * elements into the device double *out, with fixed-order partial sums (the
 * same inputs give the same bits); used by the dot-product test of the
 * adjoint and by the misfit of an FWI line-search trial.  The paper has no
 * separate counterpart: it is the inner product that test is stated in.
 * ws: device scratch of at least sweep_dot_workspace_bytes() bytes, 8-byte
 * aligned, owned by the caller; calls that overlap on the GPU must not share
 * one.  n = 0 gives 0.  SWEEP_EINVAL (n < 0, NULL out, or NULL a or b with
 * n > 0) and SWEEP_EWORKSPACE are returned before any launch.  Asynchronous
 * on `stream`. */
size_t sweep_dot_workspace_bytes(void);
int sweep_dot(const float* a, const float* b, int64_t n, double* out, void* ws,
              size_t ws_bytes, void* stream);

/* The same FP64 dot product for callers that cannot allocate device memory
 * (a plugin whose host application owns the device-memory budget, a loop
 * that must not allocate after start-up).  The paper has no counterpart; this
 * is a library convenience.  No workspace: the partial sums live in a fixed
 * 64 KiB device array inside the library, held by every GPU that loads it
 * until the process exits.  n <= SWEEP_DOT_NOALLOC_MAX_N (32 Mi elements),
 * else SWEEP_ETOOBIG before any launch.  a, b, out are device pointers on the
 * device current on the calling thread.  The first call on a device looks up
 * the array's device address and caches it; make that first call before any
 * stream capture.  All calls share the array: calls that overlap on the GPU
 * race (serialise them on one stream).  Asynchronous on `stream`. */
#define SWEEP_DOT_NOALLOC_MAX_N 33554432LL
int sweep_dot_noalloc(const float* a, const float* b, int64_t n, double* out,
                      void* stream);

/* Synchronises `stream` and returns the status word latched in `ws` by the
 * last call that used it (SWEEP_OK or a negative code). */
int sweep_status(void* ws, void* stream);

/* Diagnostic of the device-side timeout path.  Every pipeline wait in the
 * kernels is bounded (0.5 s); a wait that runs out latches SWEEP_ETIMEOUT in
 * the workspace status word and its kernel returns, leaving the context
 * usable.  This call launches one kernel whose bounded wait on a barrier
 * that nothing completes runs out: afterwards sweep_status(ws) returns
 * SWEEP_ETIMEOUT (the next solver call on ws clears it).  ws: any workspace
 * of this library (256-byte aligned, >= 4 bytes); only its status word is
 * written.  Takes ~0.5 s of one SM.  Asynchronous on `stream`. */
int sweep_check_wait_timeout(void* ws, size_t ws_bytes, void* stream);

/* Diagnostic of the SWEEP_F_ONE_LAUNCH kernels' grid barrier: launches two
 * co-resident CTAs, one of which leaves without arriving, so the other's
 * bounded barrier wait runs out and latches SWEEP_ETIMEOUT in the status word
 * of ws.  ws: any workspace of this library (256-byte aligned, >= 128 bytes);
 * its status word and bytes 64..79 are written.  Takes ~2 s of one SM.
 * Asynchronous on `stream`. */
int sweep_check_barrier_timeout(void* ws, size_t ws_bytes, void* stream);

/* Static description of a code. */
const char* sweep_strerror(int code);

/* Number of kernels this library has launched in this process so far
 * (monotone counter, for accounting launches per step). */
unsigned long long sweep_kernel_launches(void);

/* CUDA-graph capture.  A job that repeats the same calls with the same
 * buffers (an FWI loop, a batch of equal problems) can record them once and
 * replay every kernel of them with one host call; the kernels keep their
 * programmatic-launch overlap inside the graph.  Library extension: the paper
 * has no counterpart; it names kernel launches as the cost of its time loop
 * (Sec. 2.2).
 *
 * sweep_capture_begin(stream) starts a thread-local capture on `stream` (not
 * the legacy default stream 0: SWEEP_EINVAL); the library calls that this
 * thread then makes on `stream` are recorded, not run, and may not allocate,
 * synchronise or call sweep_status.  sweep_capture_end(stream, &graph) ends
 * the capture and returns an instantiated graph in *graph (SWEEP_EINVAL
 * without an active capture on this thread, SWEEP_ECUDA if the capture was
 * invalidated, e.g. by a synchronising call, in which case *graph = NULL).
 * sweep_graph_launch(graph, stream) replays it on any stream (asynchronous;
 * the recorded calls' pointers are reused, so their buffers must stay
 * alive and their contents are read at replay time); sweep_graph_kernels
 * returns the number of kernel nodes (each launch adds it to
 * sweep_kernel_launches; recorded calls add nothing); sweep_graph_destroy
 * frees the graph (the caller makes sure no replay of it is pending or
 * running).  Graphs hold no device memory of the caller's. */
int sweep_capture_begin(void* stream);
int sweep_capture_end(void* stream, void** graph);
int sweep_graph_launch(void* graph, void* stream);
int sweep_graph_kernels(void* graph);
void sweep_graph_destroy(void* graph);

/* Kernel timing for benchmarks.  While enabled, every launch of a time-step
 * kernel class selected by the mask is bracketed by two CUDA events recorded
 * on the launching stream.  sweep_profile_enable(mask) clears earlier records
 * and records the classes k with bit (1 << k) set in `mask` (-1: all
 * classes); sweep_profile_enable(0) stops recording.
 * sweep_profile_read() synchronises on the recorded events and returns, for
 * kernel class `kernel` (SWEEP_K_*), the summed device time in ms and the
 * number of launches.  Cost: two event records per recorded launch, and an
 * event between two kernels ends their programmatic overlap. */
enum {
  SWEEP_K_AC_FWD = 0,     /* acoustic forward step (all its kernels)   */
  SWEEP_K_AC_BWD = 1,     /* acoustic backward step (all its kernels)  */
  SWEEP_K_EL_VEL = 2,     /* elastic velocity half step                */
  SWEEP_K_EL_STR = 3,     /* elastic stress step                       */
  SWEEP_K_AC_FWD_IN = 4,  /* acoustic forward, stencil kernel          */
  SWEEP_K_AC_FWD_FR = 5,  /* acoustic forward, CPML correction kernels */
  SWEEP_K_AC_BWD_IN = 6,  /* acoustic backward, stencil kernel         */
  SWEEP_K_AC_BWD_FR = 7,  /* acoustic backward, CPML correction kernels*/
  SWEEP_K_AC_FWD_LOOP = 8, /* a whole acoustic forward time loop (one
                              record per call, or per group of a batched
                              call: the events sit before its first and
                              after its last step, so the steps keep
                              their programmatic overlap)                */
  SWEEP_K_AC_BWD_LOOP = 9, /* a whole acoustic backward time loop        */
  SWEEP_K_EL_ADJ = 10,     /* elastic transposed step (stress half,
                              receiver injection, velocity half)         */
  SWEEP_K_COUNT = 11
};
int sweep_profile_enable(int mask);
int sweep_profile_read(int kernel, double* ms, long long* launches);

#ifdef __cplusplus
}
#endif
#endif
