// Host side of the C ABI declared in include/sweep.h: argument validation,
// workspace layout, TMA descriptors, and the time loops that launch the step
// kernels (the Propagator of Sec. 2.1).  No device memory is allocated here:
// every buffer is carved out of the caller's workspace.
#include <cudaTypedefs.h>

#include <atomic>
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>
#include <mutex>

#include "elastic_internal.cuh"
#include "tma.cuh"

#ifdef SWEEP_NVTX
#include <nvtx3/nvToolsExt.h>
#endif

namespace sweep {

// A named range on the host timeline around the enqueueing of one phase of
// a call (forward loop, backward loop), for Nsight tools; compiled in only
// with -DSWEEP_NVTX (build with SWEEP_NVTX=1), otherwise it is empty.
struct PhaseRange {
#ifdef SWEEP_NVTX
  explicit PhaseRange(const char* name) { nvtxRangePushA(name); }
  ~PhaseRange() { nvtxRangePop(); }
#else
  explicit PhaseRange(const char*) {}
#endif
  PhaseRange(const PhaseRange&) = delete;
  PhaseRange& operator=(const PhaseRange&) = delete;
};

std::atomic<unsigned long long> g_launches{0};
void note_launches(int k) {
  if (!t_capturing) g_launches.fetch_add((unsigned long long)k);
}

// ------------------------------------------------------------- tensor maps
namespace {
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}
}  // namespace

bool make_tensor_map(CUtensorMap* map, const float* base, int rank, uint64_t dim0,
                     uint64_t dim1, uint64_t dim2, uint64_t pitch0, uint64_t pitch1,
                     uint32_t box0, uint32_t box1, uint32_t box2) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {dim0, dim1, dim2};
  cuuint64_t strides[2] = {pitch0 * sizeof(float), pitch1 * sizeof(float)};
  cuuint32_t box[3] = {box0, box1, box2};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank,
                  const_cast<float*>(base), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool make_tensor_map_bf16(CUtensorMap* map, const void* base, int rank, const uint64_t* dims,
                          const uint64_t* strides_elems, const uint32_t* box,
                          int swizzle_bytes) {
  auto fn = encode_fn();
  if (!fn || rank < 1 || rank > 5) return false;
  cuuint64_t d[5];
  cuuint64_t st[4];
  cuuint32_t bx[5], es[5];
  for (int i = 0; i < rank; ++i) {
    d[i] = dims[i];
    bx[i] = box[i];
    es[i] = 1;
    if (i > 0) st[i - 1] = strides_elems[i - 1] * 2;  // bytes
  }
  const CUtensorMapSwizzle sw = swizzle_bytes == 128  ? CU_TENSOR_MAP_SWIZZLE_128B
                                : swizzle_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                : swizzle_bytes == 32 ? CU_TENSOR_MAP_SWIZZLE_32B
                                                      : CU_TENSOR_MAP_SWIZZLE_NONE;
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (cuuint32_t)rank, const_cast<void*>(base),
                  d, st, bx, es, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

namespace {

// Stability limits of the two schemes (leapfrog in time):
//   acoustic 8th order: v dt/dx <= 2 / sqrt(2 * 6.5015873) (Nyquist symbol of D2)
//   elastic 4th-order staggered: v dt/dx <= 1 / (sqrt(2) (9/8 + 1/24))
constexpr float kCflAcoustic = 0.5546324f;
constexpr float kCflElastic = 0.6060915f;

constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Layout {
  size_t status = 0, partial = 0, vmax = 0, K = 0;
  size_t ax = 0, bx = 0, az = 0, bz = 0, axh = 0, bxh = 0, azh = 0, bzh = 0;
  size_t u[2] = {0, 0}, psx[2] = {0, 0}, psz[2] = {0, 0}, zex = 0, zez = 0;
  size_t m[2] = {0, 0}, pbx[2] = {0, 0}, pbz[2] = {0, 0}, zbx[2] = {0, 0}, zbz[2] = {0, 0};
  size_t data = 0, save = 0, graw = 0, iraw = 0;
  size_t el_par[5] = {0, 0, 0, 0, 0};  // elastic coefficients
  size_t el_f[5] = {0, 0, 0, 0, 0};    // vx, vz, txx, tzz, txz
  size_t el_p[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  // elastic adjoint state (same 13 fields in the same order), scratch, the
  // per-shot coefficient adjoints, and the checkpoints / segment states of
  // the forward replay (each a copy of the range [fwd_lo, fwd_hi))
  size_t el_a = 0, el_ap2 = 0, el_g = 0, el_ck = 0, el_seg = 0;
  int el_ngrp = 0;  // FP64 accumulator blocks of the adjoint kernels
  int el_C = 0, el_ncp = 0;
  size_t loop = 0, loopbar = 0;   // acoustic time-loop arguments, barrier words
  size_t rtile = 0, rlist = 0;    // receiver lists of the backward stencil units
  size_t fwd_lo = 0, fwd_hi = 0;  // contiguous range of forward fields
  size_t adj_lo = 0, adj_hi = 0;  // contiguous range of adjoint fields
  size_t total = 0;
};

struct Bump {
  size_t off = 0;
  size_t take(size_t bytes) {
    size_t o = off;
    off = align_up(off + bytes);
    return o;
  }
};

Geom make_geom(const sweep_problem* p) {
  Geom g{};
  g.nz = p->nz;
  g.nx = p->nx;
  g.P = p->pml;
  g.NZ = p->nz + 2 * p->pml;
  g.NX = p->nx + 2 * p->pml;
  g.NXp = (g.NX + 31) / 32 * 32;
  g.nshot = p->nshot;
  g.nrec = p->nrec;
  g.nt = p->nt;
  g.ringw = p->pml < 4 ? p->pml : 4;
  const int w = g.ringw;
  g.nring = 2 * w * (g.nx + 2 * w) + 2 * g.nz * w;
  g.fstride = (long long)g.NZ * g.NXp;
  // the plain-stencil kernels cover the whole padded grid; the CPML terms
  // are added by the correction kernels
  g.fin = Region{0, g.NZ, 0, g.NXp};
  g.bin = Region{0, g.NZ, 0, g.NXp};
  return g;
}

bool valid_problem(const sweep_problem* p) {
  if (!p) return false;
  if (p->physics != SWEEP_ACOUSTIC && p->physics != SWEEP_ELASTIC) return false;
  if (p->nz < 1 || p->nx < 1 || p->pml < 0 || p->nt < 1 || p->nshot < 0 || p->nrec < 0)
    return false;
  if (!(p->dx > 0.f) || !std::isfinite(p->dx)) return false;
  if (!(p->dt > 0.f) || !std::isfinite(p->dt)) return false;
  if (!(p->f_ref >= 0.f) || !std::isfinite(p->f_ref)) return false;
  if (!std::isfinite(p->v_pml)) return false;
  if (p->flags & ~(SWEEP_F_PADDED_MODEL | SWEEP_F_RESIDUAL_IN | SWEEP_F_ROWS16 |
                   SWEEP_F_ONE_LAUNCH | SWEEP_F_DETERMINISTIC))
    return false;  // unknown bits
  // keep every index within one shot's field (z * NXp + x, on the padded
  // row pitch) and the count of (tile, shot) units within 32 bits
  const long long NZ = (long long)p->nz + 2LL * p->pml, NX = (long long)p->nx + 2LL * p->pml;
  if (NZ > (1 << 20) || NX > (1 << 20)) return false;
  const long long NXp = (NX + 31) / 32 * 32;
  if (NZ * NXp >= (1LL << 31)) return false;
  if (p->nshot > 65535) return false;  // gridDim.y / z
  const long long tiles = (NZ + 15) / 16 * ((NX + 127) / 128);  // smallest tiles in use
  if (tiles * p->nshot >= (1LL << 31)) return false;
  return true;
}

Layout layout(const sweep_problem* p, int mode) {
  const Geom g = make_geom(p);
  Layout L;
  Bump b;
  const size_t F = sizeof(float) * (size_t)g.fstride * (size_t)g.nshot;
  L.status = b.take(sizeof(int) * 4);
  L.vmax = b.take(sizeof(unsigned int));
  L.partial = b.take(sizeof(double) * RED_BLOCKS);
  L.K = b.take(sizeof(float) * (size_t)g.fstride);
  L.ax = b.take(sizeof(float) * g.NXp);
  L.bx = b.take(sizeof(float) * g.NXp);
  L.az = b.take(sizeof(float) * g.NZ);
  L.bz = b.take(sizeof(float) * g.NZ);
  L.axh = b.take(sizeof(float) * g.NXp);
  L.bxh = b.take(sizeof(float) * g.NXp);
  L.azh = b.take(sizeof(float) * g.NZ);
  L.bzh = b.take(sizeof(float) * g.NZ);
  if (p->physics == SWEEP_ELASTIC) {
    for (int i = 0; i < 5; ++i) L.el_par[i] = b.take(sizeof(float) * (size_t)g.fstride);
    L.fwd_lo = b.off;
    for (int i = 0; i < 5; ++i) L.el_f[i] = b.take(F);
    for (int i = 0; i < 8; ++i) L.el_p[i] = b.take(F);
    L.fwd_hi = b.off;
    if (mode == SWEEP_MODE_ADJOINT || mode == SWEEP_MODE_GRADIENT) {
      L.adj_lo = b.off;
      L.el_a = b.take(L.fwd_hi - L.fwd_lo);
      L.adj_hi = b.off;
      L.el_ap2 = b.take(8 * F);  // second buffer of the adjoint memory variables
    }
    if (mode == SWEEP_MODE_GRADIENT) {
      // sqrt(nt) checkpoints of the forward state, and one segment of
      // states replayed from a checkpoint
      int C = 1;
      while ((long long)C * C < g.nt) ++C;
      L.el_C = C;
      L.el_ncp = (g.nt + C - 1) / C;
      const int sg = el_adj_shot_group(g);
      L.el_ngrp = (g.nshot + sg - 1) / sg;
      // per shot group: compensated FP32 sums (hi and lo planes)
      L.el_g = b.take((size_t)L.el_ngrp * 10 * sizeof(float) * (size_t)g.fstride);
      L.data = b.take(sizeof(float) * (size_t)g.nshot * 2 * g.nrec * g.nt);
      L.el_ck = b.take((L.fwd_hi - L.fwd_lo) * (size_t)L.el_ncp);
      L.el_seg = b.take((L.fwd_hi - L.fwd_lo) * (size_t)C);
    }
    L.total = b.off;
    return L;
  }
  L.loop = b.take(sizeof(LoopProblem));  // time-loop kernels' arguments
  L.loopbar = b.take(sizeof(unsigned) * 4);
  if (mode == SWEEP_MODE_FORWARD || mode == SWEEP_MODE_GRADIENT) {
    L.fwd_lo = b.off;
    L.u[0] = b.take(F);
    L.u[1] = b.take(F);
    L.psx[0] = b.take(F);
    L.psx[1] = b.take(F);
    L.psz[0] = b.take(F);
    L.psz[1] = b.take(F);
    L.zex = b.take(F);
    L.zez = b.take(F);
    L.fwd_hi = b.off;
  }
  if (mode == SWEEP_MODE_ADJOINT || mode == SWEEP_MODE_GRADIENT) {
    // units of the smaller tile height bound those of either
    const size_t units = (size_t)((g.NZ + IN_BZ_SMALL - 1) / IN_BZ_SMALL) *
                         ((g.NXp + IN_BX - 1) / IN_BX) * (size_t)g.nshot;
    L.rtile = b.take(sizeof(int2) * units);
    L.rlist = b.take(sizeof(int4) * (size_t)g.nshot * g.nrec);
    L.adj_lo = b.off;
    L.m[0] = b.take(F);
    L.m[1] = b.take(F);
    L.pbx[0] = b.take(F);
    L.pbx[1] = b.take(F);
    L.pbz[0] = b.take(F);
    L.pbz[1] = b.take(F);
    L.zbx[0] = b.take(F);
    L.zbx[1] = b.take(F);
    L.zbz[0] = b.take(F);
    L.zbz[1] = b.take(F);
    L.adj_hi = b.off;
  }
  if (mode == SWEEP_MODE_GRADIENT) {
    L.data = b.take(sizeof(float) * (size_t)g.nshot * g.nrec * g.nt);
    L.save = b.take(sizeof(float) * ((size_t)g.nt + 1) * g.nshot * g.nring);
    L.graw = b.take(F);
    L.iraw = b.take(F);
  }
  L.total = b.off;
  return L;
}

template <class T>
T* at(void* ws, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(ws) + off);
}

int check_ws(const sweep_problem* p, int mode, void* ws, size_t ws_bytes) {
  if (!ws || (reinterpret_cast<uintptr_t>(ws) % kAlign) != 0) return SWEEP_EWORKSPACE;
  if (ws_bytes < layout(p, mode).total) return SWEEP_EWORKSPACE;
  return SWEEP_OK;
}

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? SWEEP_OK : SWEEP_ECUDA; }

SetupArgs setup_args(const sweep_problem* p, const Layout& L, void* ws, const float* model,
                     const int32_t* src, const int32_t* rec) {
  SetupArgs s{};
  s.g = make_geom(p);
  s.physics = p->physics;
  s.model = model;
  s.padded = (p->flags & SWEEP_F_PADDED_MODEL) ? 1 : 0;
  s.dx = p->dx;
  s.dt = p->dt;
  s.f_ref = p->f_ref;
  s.v_pml = p->v_pml;
  s.cfl_limit = p->physics == SWEEP_ELASTIC ? kCflElastic : kCflAcoustic;
  s.src = src;
  s.rec = rec;
  s.K = at<float>(ws, L.K);
  s.ax = at<float>(ws, L.ax);
  s.bx = at<float>(ws, L.bx);
  s.az = at<float>(ws, L.az);
  s.bz = at<float>(ws, L.bz);
  if (p->physics == SWEEP_ELASTIC) {
    s.axh = at<float>(ws, L.axh);
    s.bxh = at<float>(ws, L.bxh);
    s.azh = at<float>(ws, L.azh);
    s.bzh = at<float>(ws, L.bzh);
  }
  s.vmax_bits = at<unsigned int>(ws, L.vmax);
  s.status = at<int>(ws, L.status);
  return s;
}

// TMA descriptors of one per-shot field [S][NZ][NXp] for interior tiles of
// bz rows: halo box and centre box.
bool field_maps(const Geom& g, const float* base, CUtensorMap* halo, CUtensorMap* centre,
                int bz) {
  const uint64_t S = (uint64_t)(g.nshot > 0 ? g.nshot : 1);
  bool ok = true;
  if (halo)
    ok = ok && make_tensor_map(halo, base, 3, g.NX, g.NZ, S, g.NXp, (uint64_t)g.fstride, IN_HW,
                               bz + 8, 1);
  if (centre)
    ok = ok && make_tensor_map(centre, base, 3, g.NX, g.NZ, S, g.NXp, (uint64_t)g.fstride, IN_BX,
                               bz, 1);
  return ok;
}

// The CPML z part's copies of a per-shot field [S][NZ][NXp]: boxes of
// IN_BX columns and `rows` rows.
bool z_map(const Geom& g, const float* base, CUtensorMap* m, int rows) {
  const uint64_t S = (uint64_t)(g.nshot > 0 ? g.nshot : 1);
  return make_tensor_map(m, base, 3, g.NX, g.NZ, S, g.NXp, (uint64_t)g.fstride, IN_BX,
                         (uint32_t)rows, 1);
}

// The shared K grid [NZ][NXp] with box (bx, bz).
bool map2(CUtensorMap* m, const Geom& g, const float* base, uint32_t bx, uint32_t bz) {
  return make_tensor_map(m, base, 2, g.NX, g.NZ, 1, g.NXp, (uint64_t)g.fstride, bx, bz, 1);
}

// Deterministic mode of a problem: one writer per border cell and phase.
bool deterministic(const sweep_problem* p) {
  return (p->flags & SWEEP_F_DETERMINISTIC) != 0;
}

// Rows of the acoustic stencil tiles of a problem.
int tile_rows(const sweep_problem* p) {
  return (p->flags & SWEEP_F_ROWS16) ? IN_BZ_SMALL : IN_BZ;
}

int region_units(const Region& R, int nshot, int bz, int* ntx) {
  if (R.z1 <= R.z0 || R.x1 <= R.x0) {
    *ntx = 0;
    return 0;
  }
  *ntx = (R.x1 - R.x0 + IN_BX - 1) / IN_BX;
  const int ntz = (R.z1 - R.z0 + bz - 1) / bz;
  return *ntx * ntz * nshot;
}

// Forward time loop of the acoustic engine: per step the plain-stencil
// kernel over the whole padded grid, then one kernel adding both axes' CPML
// terms, recording the receivers and saving the ring of u^n.  On
// return the workspace holds u^{nt} in u[nt % 2] and u^{nt-1} in
// u[(nt + 1) % 2].  AcFwdLoop holds one problem's loop state and fills the
// two kernels' arguments of step n (the batched entry runs several
// problems' steps in the same launches).
struct AcFwdLoop {
  Geom g;
  const Layout* L = nullptr;
  void* ws = nullptr;
  float* save = nullptr;
  AcInFwdArgs in{};
  AcFixArgs fx{};
  CUtensorMap tu_h[2], tu_c[2];
  CUtensorMap zu[2], zp[2];  // CPML z part: u^n and psi_z windows

  int init(const sweep_problem* p, const Layout& lay, void* w, const float* wavelet,
           const int32_t* src, const int32_t* rec, float* data, bool save_ring,
           cudaStream_t st) {
    g = make_geom(p);
    L = &lay;
    ws = w;
    cudaMemsetAsync(at<char>(ws, L->fwd_lo), 0, L->fwd_hi - L->fwd_lo, st);
    save = save_ring ? at<float>(ws, L->save) : nullptr;
    if (save) cudaMemsetAsync(save, 0, sizeof(float) * (size_t)g.nshot * g.nring, st);
    int* status = at<int>(ws, L->status);
    in.g = g;
    in.bz = tile_rows(p);
    in.units = region_units(g.fin, g.nshot, in.bz, &in.ntx);
    for (int b = 0; b < 2; ++b)
      if (!field_maps(g, at<float>(ws, L->u[b]), &tu_h[b], &tu_c[b], in.bz))
        return SWEEP_ECUDA;
    if (!map2(&in.tK, g, at<float>(ws, L->K), IN_BX, in.bz)) return SWEEP_ECUDA;
    for (int b = 0; b < 2; ++b)
      if (!z_map(g, at<float>(ws, L->u[b]), &zu[b], ZCH_FWD + 8) ||
          !z_map(g, at<float>(ws, L->psz[b]), &zp[b], ZCH_FWD + 8))
        return SWEEP_ECUDA;
    if (!z_map(g, at<float>(ws, L->zez), &fx.tzz, ZCH_FWD) ||
        !map2(&fx.tzK, g, at<float>(ws, L->K), IN_BX, ZCH_FWD))
      return SWEEP_ECUDA;
    in.wavelet = wavelet;
    in.src = src;
    in.status = status;
    fx.g = g;
    fx.K = at<float>(ws, L->K);
    fx.ax = at<float>(ws, L->ax);
    fx.bx = at<float>(ws, L->bx);
    fx.az = at<float>(ws, L->az);
    fx.bz = at<float>(ws, L->bz);
    fx.zzin = fx.zzout = at<float>(ws, L->zez);
    fx.zxin = fx.zxout = at<float>(ws, L->zex);
    fx.rec = rec;
    fx.data = data;
    fx.own = deterministic(p);
    fx.status = status;
    return SWEEP_OK;
  }

  void step(int n) {
    const int A = n & 1, B = (n + 1) & 1;
    in.n = n;
    in.tu = tu_h[A];
    in.tup = tu_c[B];
    in.un = at<float>(ws, L->u[B]);
    fx.n = n;
    fx.u = at<float>(ws, L->u[A]);
    fx.un = at<float>(ws, L->u[B]);
    fx.tzu = zu[A];
    fx.tzp = zp[A];
    fx.pzin = at<float>(ws, L->psz[A]);
    fx.pzout = at<float>(ws, L->psz[B]);
    fx.pxin = at<float>(ws, L->psx[A]);
    fx.pxout = at<float>(ws, L->psx[B]);
    fx.save = save ? save + (size_t)n * g.nshot * g.nring : nullptr;  // ring of u^n
  }
};

int acoustic_forward_loop(const sweep_problem* p, const Layout& L, void* ws,
                          const float* wavelet, const int32_t* src, const int32_t* rec,
                          float* data, bool save_ring, cudaStream_t st) {
  PhaseRange r("sweep acoustic forward");
  AcFwdLoop f;
  const int rc = f.init(p, L, ws, wavelet, src, rec, data, save_ring, st);
  if (rc) return rc;
  void* loop = profile_begin(SWEEP_K_AC_FWD_LOOP, st);
  for (int n = 0; n < f.g.nt; ++n) {
    f.step(n);
    void* tok = profile_begin(SWEEP_K_AC_FWD, st);
    launch_ac_in_fwd(f.in, st);
    launch_ac_fix_fwd(f.fx, st);
    profile_end(tok, st);
  }
  profile_end(loop, st);
  return SWEEP_OK;
}

// Backward loop: adjoint propagation from the residual `res`; optionally the
// imaging condition with wavefield reconstruction (gradient) and/or the
// adjoint source gather (wgrad).  Per step the plain kernel over the whole
// grid (it also injects the residual at the receivers, from per-unit
// receiver lists built once per call), then one kernel adding both axes'
// CPML terms of mu^n and restoring the ring of u^{n-1}.  Steps run
// n = nt .. 0; AcBwdLoop::step(n) fills the arguments of step n and says
// which of the two kernels run.
struct AcBwdLoop {
  Geom g;
  const Layout* L = nullptr;
  void* ws = nullptr;
  float* save = nullptr;
  bool imaging = false;
  const float* wgrad = nullptr;
  AcInBwdArgs in{};
  AcFixArgs fx{};
  CUtensorMap tu_h[2], tu_c[2], tm_h[2], tm_c[2];


  int init(const sweep_problem* p, const Layout& lay, void* w, const float* wavelet,
           const int32_t* src, const int32_t* rec, const float* res, float* wg, bool img,
           bool illum, cudaStream_t st) {
    g = make_geom(p);
    L = &lay;
    ws = w;
    imaging = img;
    wgrad = wg;
    cudaMemsetAsync(at<char>(ws, L->adj_lo), 0, L->adj_hi - L->adj_lo, st);
    const size_t F = sizeof(float) * (size_t)g.fstride * (size_t)g.nshot;
    if (imaging) {
      cudaMemsetAsync(at<float>(ws, L->graw), 0, F, st);
      if (illum) cudaMemsetAsync(at<float>(ws, L->iraw), 0, F, st);
    }
    int* status = at<int>(ws, L->status);
    save = imaging ? at<float>(ws, L->save) : nullptr;
    in.g = g;
    in.bz = tile_rows(p);
    in.units = region_units(g.bin, g.nshot, in.bz, &in.ntx);
    for (int b = 0; b < 2; ++b) {
      if (imaging && !field_maps(g, at<float>(ws, L->u[b]), &tu_h[b], &tu_c[b], in.bz))
        return SWEEP_ECUDA;
      if (!field_maps(g, at<float>(ws, L->m[b]), &tm_h[b], &tm_c[b], in.bz))
        return SWEEP_ECUDA;
    }
    if (!map2(&in.tK, g, at<float>(ws, L->K), IN_BX, in.bz)) return SWEEP_ECUDA;
    if (imaging && !field_maps(g, at<float>(ws, L->graw), nullptr, &in.tG, in.bz))
      return SWEEP_ECUDA;

    in.graw = imaging ? at<float>(ws, L->graw) : nullptr;
    in.illum = (imaging && illum) ? at<float>(ws, L->iraw) : nullptr;
    in.wavelet = wavelet;
    in.src = src;
    in.wgrad = wg;
    in.status = status;
    const bool own = deterministic(p);
    if (own && res && g.nrec > 0) {  // the stencil kernel injects the residual
      in.res = res;
      in.rtile = at<int2>(ws, L->rtile);
      in.rlist = at<int4>(ws, L->rlist);
      launch_rec_tiles(g, rec, in.bz, in.ntx, const_cast<int2*>(in.rtile),
                       const_cast<int4*>(in.rlist), st);
      note_launches(1);
    }
    fx.g = g;
    fx.K = at<float>(ws, L->K);
    fx.ax = at<float>(ws, L->ax);
    fx.bx = at<float>(ws, L->bx);
    fx.az = at<float>(ws, L->az);
    fx.bz = at<float>(ws, L->bz);
    fx.rec = rec;
    fx.res = (!own && g.nrec > 0) ? res : nullptr;
    fx.own = own;
    fx.status = status;
    return SWEEP_OK;
  }

  // false: step n has no work; *adj: the CPML kernel runs too
  bool step(int n, bool* adj) {
    const int A = n & 1, B = (n + 1) & 1;  // u^n in u[A]; mu^{n+1} in m[B]
    const int do_adj = n >= 1;
    const int do_img = imaging && n <= g.nt - 1;
    const int do_rec = imaging && n >= 1 && n <= g.nt - 1;
    *adj = do_adj;
    if (!(do_adj || do_img || wgrad)) return false;
    in.n = n;
    in.do_adj = do_adj;
    in.do_img = do_img;
    in.do_rec = do_rec;
    if (imaging) {
      in.tuA = tu_h[A];
      in.tuB = tu_c[B];
    }
    in.tmA = tm_h[B];
    in.tmB = tm_c[A];
    in.uB = imaging ? at<float>(ws, L->u[B]) : nullptr;
    in.mB = at<float>(ws, L->m[A]);
    if (do_adj) {
      // CPML terms of mu^n and the residual injection mu^n(r) += K r^{n-1}
      fx.n = n;
      fx.u = at<float>(ws, L->m[B]);
      fx.un = at<float>(ws, L->m[A]);

      fx.pzin = at<float>(ws, L->pbz[A]);
      fx.pzout = at<float>(ws, L->pbz[B]);
      fx.zzin = at<float>(ws, L->zbz[A]);
      fx.zzout = at<float>(ws, L->zbz[B]);
      fx.pxin = at<float>(ws, L->pbx[A]);
      fx.pxout = at<float>(ws, L->pbx[B]);
      fx.zxin = at<float>(ws, L->zbx[A]);
      fx.zxout = at<float>(ws, L->zbx[B]);
      fx.save = do_rec && save ? save + (size_t)(n - 1) * g.nshot * g.nring : nullptr;
      fx.uring = do_rec ? at<float>(ws, L->u[B]) : nullptr;  // u^{n-1}
    }
    return true;
  }
};

int acoustic_backward_loop(const sweep_problem* p, const Layout& L, void* ws,
                           const float* wavelet, const int32_t* src, const int32_t* rec,
                           const float* res, float* wgrad, bool imaging, bool illum,
                           cudaStream_t st) {
  PhaseRange r("sweep acoustic backward");
  AcBwdLoop b;
  const int rc = b.init(p, L, ws, wavelet, src, rec, res, wgrad, imaging, illum, st);
  if (rc) return rc;
  void* loop = profile_begin(SWEEP_K_AC_BWD_LOOP, st);
  for (int n = b.g.nt; n >= 0; --n) {
    bool adj = false;
    if (!b.step(n, &adj)) continue;
    void* tok = profile_begin(SWEEP_K_AC_BWD, st);
    launch_ac_in_bwd(b.in, st);
    if (adj) launch_ac_fix_bwd(b.fx, st);
    profile_end(tok, st);
  }
  profile_end(loop, st);
  return SWEEP_OK;
}

// Elastic coefficients (once per call) and the step arguments on the
// forward state starting at `state` (a copy of the range [fwd_lo, fwd_hi)).
void elastic_params(const sweep_problem* p, const Layout& L, void* ws, const float* model,
                    cudaStream_t st) {
  ElParamArgs pa{};
  pa.g = make_geom(p);
  pa.model = model;
  pa.padded = (p->flags & SWEEP_F_PADDED_MODEL) ? 1 : 0;
  pa.dx = p->dx;
  pa.dt = p->dt;
  pa.cbx = at<float>(ws, L.el_par[0]);
  pa.cbz = at<float>(ws, L.el_par[1]);
  pa.cl2m = at<float>(ws, L.el_par[2]);
  pa.clam = at<float>(ws, L.el_par[3]);
  pa.cmu = at<float>(ws, L.el_par[4]);
  launch_el_params(pa, st);
}

float* state_field(const Layout& L, char* state, int k) {  // k: 0..4 fields, 5..12 p1..p8
  const size_t off = k < 5 ? L.el_f[k] : L.el_p[k - 5];
  return reinterpret_cast<float*>(state + (off - L.fwd_lo));
}

// The step's input state (fields 0..4 and p1..p8 of a state copy at `in`)
// and where it writes the state after the step.
void set_step_in(ElStepArgs& a, char* in, const Layout& L) {
  float** f[13] = {&a.vx, &a.vz, &a.txx, &a.tzz, &a.txz, &a.p1, &a.p2,
                   &a.p3, &a.p4, &a.p5, &a.p6, &a.p7, &a.p8};
  for (int i = 0; i < 13; ++i) *f[i] = state_field(L, in, i);
}
void set_step_out(ElStepArgs& a, char* out, const Layout& L) {
  float** f[13] = {&a.vx_o, &a.vz_o, &a.txx_o, &a.tzz_o, &a.txz_o, &a.p1_o, &a.p2_o,
                   &a.p3_o, &a.p4_o, &a.p5_o, &a.p6_o, &a.p7_o, &a.p8_o};
  for (int i = 0; i < 13; ++i) *f[i] = state_field(L, out, i);
}

ElStepArgs elastic_step_args(const sweep_problem* p, const Layout& L, void* ws, char* state,
                             const float* wavelet, const int32_t* src, const int32_t* rec,
                             float* data) {
  ElStepArgs a{};
  a.g = make_geom(p);
  a.vx = state_field(L, state, 0);
  a.vz = state_field(L, state, 1);
  a.txx = state_field(L, state, 2);
  a.tzz = state_field(L, state, 3);
  a.txz = state_field(L, state, 4);
  float** ps[8] = {&a.p1, &a.p2, &a.p3, &a.p4, &a.p5, &a.p6, &a.p7, &a.p8};
  for (int i = 0; i < 8; ++i) *ps[i] = state_field(L, state, 5 + i);
  set_step_out(a, state, L);  // in place
  a.cbx = at<float>(ws, L.el_par[0]);
  a.cbz = at<float>(ws, L.el_par[1]);
  a.cl2m = at<float>(ws, L.el_par[2]);
  a.clam = at<float>(ws, L.el_par[3]);
  a.cmu = at<float>(ws, L.el_par[4]);
  a.ax = at<float>(ws, L.ax);
  a.bx = at<float>(ws, L.bx);
  a.axh = at<float>(ws, L.axh);
  a.bxh = at<float>(ws, L.bxh);
  a.az = at<float>(ws, L.az);
  a.bz = at<float>(ws, L.bz);
  a.azh = at<float>(ws, L.azh);
  a.bzh = at<float>(ws, L.bzh);
  a.wavelet = wavelet;
  a.src = src;
  a.rec = rec;
  a.data = data;
  a.src_scale = (float)((double)p->dt / ((double)p->dx * p->dx));
  a.status = at<int>(ws, L.status);
  if (!el_step_maps(a)) a.units = -1;  // reported by the callers
  return a;
}

// Elastic forward time loop: velocity then stress kernel per step.  With
// checkpoints (gradient mode) the state before step k C is copied to
// checkpoint k.
int elastic_forward_loop(const sweep_problem* p, const Layout& L, void* ws, const float* model,
                         const float* wavelet, const int32_t* src, const int32_t* rec,
                         float* data, bool checkpoints, cudaStream_t st) {
  PhaseRange r("sweep elastic forward");
  const Geom g = make_geom(p);
  char* state = at<char>(ws, L.fwd_lo);
  const size_t sb = L.fwd_hi - L.fwd_lo;
  cudaMemsetAsync(state, 0, sb, st);
  elastic_params(p, L, ws, model, st);
  ElStepArgs a = elastic_step_args(p, L, ws, state, wavelet, src, rec, data);
  if (a.units < 0) return SWEEP_ECUDA;
  for (int n = 0; n < g.nt; ++n) {
    if (checkpoints && n % L.el_C == 0)
      cudaMemcpyAsync(at<char>(ws, L.el_ck) + (size_t)(n / L.el_C) * sb, state, sb,
                      cudaMemcpyDeviceToDevice, st);
    a.n = n;
    launch_el_step(a, st);
  }
  return SWEEP_OK;
}

// Elastic reverse loop: the transposed steps n = nt-1 .. 0 from the residual
// (or adjoint data) `res`.  gradient: replays each checkpoint segment of the
// forward, keeping the state after every step, and accumulates the
// coefficient adjoints; wgrad: wavelet adjoint.
int elastic_reverse_loop(const sweep_problem* p, const Layout& L, void* ws, const float* wavelet,
                         const int32_t* src, const int32_t* rec, const float* res, float* wgrad,
                         bool gradient, cudaStream_t st) {
  PhaseRange r("sweep elastic reverse");
  const Geom g = make_geom(p);
  char* adj = at<char>(ws, L.el_a);
  const size_t sb = L.fwd_hi - L.fwd_lo;
  cudaMemsetAsync(adj, 0, sb, st);
  ElAdjArgs a{};
  a.g = g;
  a.avx = state_field(L, adj, 0);
  a.avz = state_field(L, adj, 1);
  a.atxx = state_field(L, adj, 2);
  a.atzz = state_field(L, adj, 3);
  a.atxz = state_field(L, adj, 4);
  // adjoint memory variables: the state's p1..p8 and a second buffer,
  // read from one and written to the other, swapped every step
  float* apb[2][8];
  for (int i = 0; i < 8; ++i) {
    apb[0][i] = state_field(L, adj, 5 + i);
    apb[1][i] = at<float>(ws, L.el_ap2) + (size_t)i * g.fstride * g.nshot;
  }
  cudaMemsetAsync(at<char>(ws, L.el_ap2), 0, 8 * sizeof(float) * (size_t)g.fstride * g.nshot,
                  st);
  int cur = 0;
  auto set_ap = [&]() {
    for (int i = 0; i < 8; ++i) {
      a.ap_in[i] = apb[cur][i];
      a.ap_out[i] = apb[cur ^ 1][i];
    }
  };
  a.cbx = at<float>(ws, L.el_par[0]);
  a.cbz = at<float>(ws, L.el_par[1]);
  a.cl2m = at<float>(ws, L.el_par[2]);
  a.clam = at<float>(ws, L.el_par[3]);
  a.cmu = at<float>(ws, L.el_par[4]);
  a.ax = at<float>(ws, L.ax);
  a.bx = at<float>(ws, L.bx);
  a.axh = at<float>(ws, L.axh);
  a.bxh = at<float>(ws, L.bxh);
  a.az = at<float>(ws, L.az);
  a.bz = at<float>(ws, L.bz);
  a.azh = at<float>(ws, L.azh);
  a.bzh = at<float>(ws, L.bzh);
  a.res = g.nrec > 0 ? res : nullptr;
  a.src = src;
  a.rec = rec;
  a.wgrad = wgrad;
  a.src_scale = (float)((double)p->dt / ((double)p->dx * p->dx));
  a.status = at<int>(ws, L.status);
  if (!el_adj_maps(a)) return SWEEP_ECUDA;
  if (!gradient) {
    for (int n = g.nt - 1; n >= 0; --n) {
      a.n = n;
      set_ap();
      launch_el_adj_step(a, st);
      cur ^= 1;
    }
    return SWEEP_OK;
  }
  a.gacc = at<float>(ws, L.el_g);
  cudaMemsetAsync(a.gacc, 0, (size_t)a.ngrp * 10 * sizeof(float) * (size_t)g.fstride, st);
  char* state = at<char>(ws, L.fwd_lo);
  char* ck = at<char>(ws, L.el_ck);
  char* seg = at<char>(ws, L.el_seg);
  ElStepArgs fs = elastic_step_args(p, L, ws, state, wavelet, src, rec, nullptr);
  if (fs.units < 0) return SWEEP_ECUDA;
  for (int k = L.el_ncp - 1; k >= 0; --k) {
    const int n0 = k * L.el_C, n1 = std::min(n0 + L.el_C, g.nt);
    // replay the segment from checkpoint k, each step writing the state
    // after it into its own slot (a memory variable only on the tiles that
    // meet its strip: the adjoint reads it only where its profile is on)
    for (int n = n0; n < n1; ++n) {
      set_step_in(fs, n > n0 ? seg + (size_t)(n - n0 - 1) * sb : ck + (size_t)k * sb, L);
      set_step_out(fs, seg + (size_t)(n - n0) * sb, L);
      if (!el_step_maps(fs)) return SWEEP_ECUDA;
      fs.n = n;
      launch_el_step(fs, st);
    }
    for (int n = n1 - 1; n >= n0; --n) {
      char* after = seg + (size_t)(n - n0) * sb;
      char* before = n > n0 ? seg + (size_t)(n - n0 - 1) * sb : ck + (size_t)k * sb;
      a.fvx = state_field(L, after, 0);
      a.fvz = state_field(L, after, 1);
      for (int i = 0; i < 8; ++i) a.fp[i] = state_field(L, after, 5 + i);
      a.ftxx = state_field(L, before, 2);
      a.ftzz = state_field(L, before, 3);
      a.ftxz = state_field(L, before, 4);
      if (!el_adj_forward_maps(a)) return SWEEP_ECUDA;
      a.n = n;
      set_ap();
      launch_el_adj_step(a, st);
      cur ^= 1;
    }
  }
  return SWEEP_OK;
}

}  // namespace
}  // namespace sweep

using namespace sweep;

extern "C" {

size_t sweep_workspace_bytes(const sweep_problem* prob, int mode) {
  if (!valid_problem(prob)) return 0;
  if (mode < SWEEP_MODE_FORWARD || mode > SWEEP_MODE_GRADIENT) return 0;
  return layout(prob, mode).total;
}

static int begin(const sweep_problem* p, int mode, void* ws, size_t ws_bytes,
                 cudaStream_t st) {
  if (!valid_problem(p)) return SWEEP_EINVAL;
  int rc = check_ws(p, mode, ws, ws_bytes);
  if (rc) return rc;
  const Layout L = layout(p, mode);
  return cuda_rc(cudaMemsetAsync(at<int>(ws, L.status), 0, sizeof(int), st));
}

static int gradient_group(const sweep_problem* const* P, const float* const* models,
                          const float* const* wavelets, const int32_t* const* srcs,
                          const int32_t* const* recs, const float* const* d_obs,
                          float* const* grads, double* const* misfits, void* const* wss,
                          int np, cudaStream_t st);
static int forward_group(const sweep_problem* const* P, const float* const* models,
                         const float* const* wavelets, const int32_t* const* srcs,
                         const int32_t* const* recs, float* const* data, void* const* wss,
                         int np, cudaStream_t st);

static bool one_launch(const sweep_problem* p) {
  return p->physics == SWEEP_ACOUSTIC && (p->flags & SWEEP_F_ONE_LAUNCH);
}
// the time-loop kernels run the default mode only
static bool unsupported_combination(const sweep_problem* p) {
  return one_launch(p) && deterministic(p);
}

int sweep_forward(const sweep_problem* p, const float* model, const float* wavelet,
                  const int32_t* src, const int32_t* rec, float* data, void* ws,
                  size_t ws_bytes, void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!valid_problem(p) || !model) return SWEEP_EINVAL;
  if (p->nshot > 0 && (!wavelet || !src)) return SWEEP_EINVAL;
  if (p->nshot > 0 && p->nrec > 0 && (!rec || !data)) return SWEEP_EINVAL;
  if (unsupported_combination(p)) return SWEEP_EUNSUPPORTED;
  int rc = begin(p, SWEEP_MODE_FORWARD, ws, ws_bytes, st);
  if (rc) return rc;
  if (p->nshot == 0) return SWEEP_OK;
  if (one_launch(p)) {  // a group of one problem: the time-loop kernel
    rc = forward_group(&p, &model, &wavelet, &src, &rec, &data, &ws, 1, st);
    return rc ? rc : cuda_rc(cudaGetLastError());
  }
  const Layout L = layout(p, SWEEP_MODE_FORWARD);
  if (p->physics == SWEEP_ELASTIC) {
    SetupArgs sa = setup_args(p, L, ws, model, src, rec);
    sa.K = nullptr;  // no acoustic K for the elastic engine
    launch_setup(sa, st);
    rc = elastic_forward_loop(p, L, ws, model, wavelet, src, rec, p->nrec > 0 ? data : nullptr,
                              false, st);
    if (rc) return rc;
    return cuda_rc(cudaGetLastError());
  }
  launch_setup(setup_args(p, L, ws, model, src, rec), st);
  rc = acoustic_forward_loop(p, L, ws, wavelet, src, rec, p->nrec > 0 ? data : nullptr, false,
                             st);
  if (rc) return rc;
  return cuda_rc(cudaGetLastError());
}

int sweep_adjoint(const sweep_problem* p, const float* model, const float* adj_data,
                  const int32_t* src, const int32_t* rec, float* wavelet_grad, void* ws,
                  size_t ws_bytes, void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!valid_problem(p) || !model) return SWEEP_EINVAL;
  if (p->nshot > 0 && (!src || !wavelet_grad)) return SWEEP_EINVAL;
  if (p->nshot > 0 && p->nrec > 0 && (!rec || !adj_data)) return SWEEP_EINVAL;
  if (one_launch(p)) return SWEEP_EUNSUPPORTED;
  int rc = begin(p, SWEEP_MODE_ADJOINT, ws, ws_bytes, st);
  if (rc) return rc;
  if (p->nshot == 0) return SWEEP_OK;
  const Layout L = layout(p, SWEEP_MODE_ADJOINT);
  if (p->physics == SWEEP_ELASTIC) {
    SetupArgs sa = setup_args(p, L, ws, model, src, rec);
    sa.K = nullptr;
    launch_setup(sa, st);
    elastic_params(p, L, ws, model, st);
    rc = elastic_reverse_loop(p, L, ws, nullptr, src, rec, adj_data, wavelet_grad, false, st);
    if (rc) return rc;
    return cuda_rc(cudaGetLastError());
  }
  launch_setup(setup_args(p, L, ws, model, src, rec), st);
  // no imaging: the backward kernels never read the wavelet
  rc = acoustic_backward_loop(p, L, ws, nullptr, src, rec, adj_data, wavelet_grad, false, false,
                              st);
  if (rc) return rc;
  return cuda_rc(cudaGetLastError());
}

int sweep_gradient(const sweep_problem* p, const float* model, const float* wavelet,
                   const int32_t* src, const int32_t* rec, const float* d_obs, float* grad,
                   double* misfit, float* illum, void* ws, size_t ws_bytes, void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!valid_problem(p) || !model || !grad) return SWEEP_EINVAL;
  if (p->nshot > 0 && (!wavelet || !src)) return SWEEP_EINVAL;
  if (p->nshot > 0 && p->nrec > 0 && (!rec || !d_obs)) return SWEEP_EINVAL;
  if (p->physics == SWEEP_ELASTIC && illum) return SWEEP_EUNSUPPORTED;
  if (one_launch(p) && illum) return SWEEP_EUNSUPPORTED;
  if (unsupported_combination(p)) return SWEEP_EUNSUPPORTED;
  int rc = begin(p, SWEEP_MODE_GRADIENT, ws, ws_bytes, st);
  if (rc) return rc;
  const Geom g = make_geom(p);
  const int npar = p->physics == SWEEP_ELASTIC ? 3 : 1;
  if (p->nshot == 0) {
    cudaMemsetAsync(grad, 0, sizeof(float) * npar * (size_t)g.nz * g.nx, st);
    if (illum) cudaMemsetAsync(illum, 0, sizeof(float) * (size_t)g.nz * g.nx, st);
    if (misfit) cudaMemsetAsync(misfit, 0, sizeof(double), st);
    return cuda_rc(cudaGetLastError());
  }
  if (one_launch(p)) {  // a group of one problem: the time-loop kernels
    rc = gradient_group(&p, &model, &wavelet, &src, &rec, &d_obs, &grad, &misfit, &ws, 1, st);
    return rc ? rc : cuda_rc(cudaGetLastError());
  }
  const Layout L = layout(p, SWEEP_MODE_GRADIENT);
  if (p->physics == SWEEP_ELASTIC) {
    SetupArgs sa = setup_args(p, L, ws, model, src, rec);
    sa.K = nullptr;
    launch_setup(sa, st);
    float* d = at<float>(ws, L.data);
    rc = elastic_forward_loop(p, L, ws, model, wavelet, src, rec, p->nrec > 0 ? d : nullptr,
                              true, st);
    if (rc) return rc;
    const long long nd = (long long)g.nshot * 2 * g.nrec * g.nt;
    launch_residual_misfit(d, d_obs, d, nd, (p->flags & SWEEP_F_RESIDUAL_IN) ? 1 : 0,
                           at<double>(ws, L.partial), RED_BLOCKS, misfit, at<int>(ws, L.status),
                           st);
    note_launches(2);
    rc = elastic_reverse_loop(p, L, ws, wavelet, src, rec, d, nullptr, true, st);
    if (rc) return rc;
    launch_el_grad(g, at<float>(ws, L.el_g), L.el_ngrp, model,
                   (p->flags & SWEEP_F_PADDED_MODEL) ? 1 : 0, p->dx, p->dt, grad,
                   at<int>(ws, L.status), st);
    return cuda_rc(cudaGetLastError());
  }
  launch_setup(setup_args(p, L, ws, model, src, rec), st);
  float* d = at<float>(ws, L.data);
  rc = acoustic_forward_loop(p, L, ws, wavelet, src, rec, p->nrec > 0 ? d : nullptr, true, st);
  if (rc) return rc;
  const long long nd = (long long)g.nshot * g.nrec * g.nt;
  launch_residual_misfit(d, d_obs, d, nd, (p->flags & SWEEP_F_RESIDUAL_IN) ? 1 : 0,
                         at<double>(ws, L.partial), RED_BLOCKS, misfit, at<int>(ws, L.status),
                         st);
  note_launches(2);
  rc = acoustic_backward_loop(p, L, ws, wavelet, src, rec, d, nullptr, true, illum != nullptr,
                              st);
  if (rc) return rc;
  launch_grad_reduce(g, at<float>(ws, L.graw), illum ? at<float>(ws, L.iraw) : nullptr, model,
                     (p->flags & SWEEP_F_PADDED_MODEL) ? 1 : 0, grad, illum,
                     at<int>(ws, L.status), st);
  note_launches(1);
  return cuda_rc(cudaGetLastError());
}

// The time-loop kernels' path (SWEEP_F_ONE_LAUNCH): the arguments of both
// step parities of each live problem go into its workspace, then one
// launch runs the whole forward loop.  lp[i] keeps problem i's arguments
// for the backward half.
static int loop_forward(const sweep_problem* const* P, std::vector<AcFwdLoop>& F,
                        const std::vector<Layout>& Ls, void* const* wss,
                        const std::vector<int>& live, std::vector<LoopProblem>& lp, int ntmax,
                        cudaStream_t st) {
  LoopArgs la{};
  for (int i : live) {
    LoopProblem& h = lp[i];
    for (int k = 0; k < 2; ++k) {
      F[i].step(k);
      h.fin[k] = F[i].in;
      h.ffix[k] = F[i].fx;
      fix_fwd_split(h.ffix[k]);
    }
    h.fsave = F[i].save;
    h.slot = (long long)F[i].g.nshot * F[i].g.nring;
    h.nt = P[i]->nt;
    LoopProblem* d = at<LoopProblem>(wss[i], Ls[i].loop);
    launch_loop_install(h, d, st);
    la.p[la.np++] = d;
  }
  la.nsteps = ntmax;
  la.bar = at<unsigned>(wss[live[0]], Ls[live[0]].loopbar);
  cudaMemsetAsync(la.bar, 0, sizeof(unsigned) * 4, st);
  return launch_ac_loop_fwd(la, st);
}

static int loop_backward(const sweep_problem* const* P, std::vector<AcBwdLoop>& B,
                         const std::vector<Layout>& Ls, void* const* wss,
                         const std::vector<int>& live, std::vector<LoopProblem>& lp, int ntmax,
                         cudaStream_t st) {
  LoopArgs la{};
  for (int i : live) {
    LoopProblem& h = lp[i];
    for (int k = 0; k < 2; ++k) {
      bool adj = false;
      B[i].step(k + 2, &adj);  // buffers of the steps with n % 2 == k
      h.bin[k] = B[i].in;
      AcFixArgs& f = h.bfix[k];
      f = B[i].fx;
      f.n = 1;  // a step with a residual injection ...
      f.save = B[i].save;  // ... and a ring restore: slot n - 1 set per step
      f.uring = at<float>(wss[i], Ls[i].u[(k + 1) & 1]);
      fix_bwd_split(f);
    }
    LoopProblem* d = at<LoopProblem>(wss[i], Ls[i].loop);
    launch_loop_install(h, d, st);
    la.p[la.np++] = d;
  }
  la.nsteps = ntmax + 1;
  la.bar = at<unsigned>(wss[live[0]], Ls[live[0]].loopbar);
  cudaMemsetAsync(la.bar, 0, sizeof(unsigned) * 4, st);
  return launch_ac_loop_bwd(la, st);
}

// Gradients of up to kStepBatch acoustic problems in lockstep: every step
// kernel launch carries the step of each problem that has it (forward: step
// t for the problems with t < nt; backward: step nt - t of each).
static int gradient_group(const sweep_problem* const* P, const float* const* models,
                          const float* const* wavelets, const int32_t* const* srcs,
                          const int32_t* const* recs, const float* const* d_obs,
                          float* const* grads, double* const* misfits, void* const* wss,
                          int np, cudaStream_t st) {
  const bool one_launch = (P[0]->flags & SWEEP_F_ONE_LAUNCH) != 0;
  std::vector<Layout> Ls(np);
  std::vector<AcFwdLoop> F(np);
  std::vector<AcBwdLoop> Bk(np);
  std::vector<int> live;
  int ntmax = 0;
  for (int i = 0; i < np; ++i) {
    const sweep_problem* p = P[i];
    const Geom g = make_geom(p);
    if (p->nshot == 0) {
      cudaMemsetAsync(grads[i], 0, sizeof(float) * (size_t)g.nz * g.nx, st);
      cudaMemsetAsync(misfits[i], 0, sizeof(double), st);
      continue;
    }
    Ls[i] = layout(p, SWEEP_MODE_GRADIENT);
    launch_setup(setup_args(p, Ls[i], wss[i], models[i], srcs[i], recs[i]), st);
    float* d = at<float>(wss[i], Ls[i].data);
    const int rc = F[i].init(p, Ls[i], wss[i], wavelets[i], srcs[i], recs[i],
                             p->nrec > 0 ? d : nullptr, true, st);
    if (rc) return rc;
    live.push_back(i);
    ntmax = std::max(ntmax, p->nt);
  }
  if (live.empty()) return SWEEP_OK;
  AcInFwdArgs fin[kStepBatch];
  AcInBwdArgs bin[kStepBatch];
  AcFixArgs fix[kStepBatch];
  std::vector<LoopProblem> lp(one_launch ? np : 0);
  void* ftok = profile_begin(SWEEP_K_AC_FWD_LOOP, st);
  if (one_launch) {
    const int rc = loop_forward(P, F, Ls, wss, live, lp, ntmax, st);
    if (rc) return rc;
  } else {
    for (int t = 0; t < ntmax; ++t) {
      int k = 0;
      for (int i : live) {
        if (t >= P[i]->nt) continue;
        F[i].step(t);
        fin[k] = F[i].in;
        fix[k] = F[i].fx;
        ++k;
      }
      launch_ac_in_fwd_batch(fin, k, st);
      launch_ac_fix_fwd_batch(fix, k, st);
    }
  }
  profile_end(ftok, st);
  for (int i : live) {
    const sweep_problem* p = P[i];
    float* d = at<float>(wss[i], Ls[i].data);
    const long long nd = (long long)p->nshot * p->nrec * p->nt;
    launch_residual_misfit(d, d_obs[i], d, nd, (p->flags & SWEEP_F_RESIDUAL_IN) ? 1 : 0,
                           at<double>(wss[i], Ls[i].partial), RED_BLOCKS, misfits[i],
                           at<int>(wss[i], Ls[i].status), st);
    note_launches(2);
    const int rc = Bk[i].init(p, Ls[i], wss[i], wavelets[i], srcs[i], recs[i], d, nullptr,
                              true, false, st);
    if (rc) return rc;
  }
  void* btok = profile_begin(SWEEP_K_AC_BWD_LOOP, st);
  if (one_launch) {
    const int rc = loop_backward(P, Bk, Ls, wss, live, lp, ntmax, st);
    if (rc) return rc;
  } else {
    for (int t = 0; t <= ntmax; ++t) {
      int kb = 0, kf = 0;
      for (int i : live) {
        const int n = P[i]->nt - t;
        bool adj = false;
        if (n < 0 || !Bk[i].step(n, &adj)) continue;
        bin[kb++] = Bk[i].in;
        if (adj) fix[kf++] = Bk[i].fx;
      }
      launch_ac_in_bwd_batch(bin, kb, st);
      launch_ac_fix_bwd_batch(fix, kf, st);
    }
  }
  profile_end(btok, st);
  for (int i : live) {
    const sweep_problem* p = P[i];
    launch_grad_reduce(make_geom(p), at<float>(wss[i], Ls[i].graw), nullptr, models[i],
                       (p->flags & SWEEP_F_PADDED_MODEL) ? 1 : 0, grads[i], nullptr,
                       at<int>(wss[i], Ls[i].status), st);
    note_launches(1);
  }
  return SWEEP_OK;
}

// Forward runs of up to kStepBatch acoustic problems in lockstep.
static int forward_group(const sweep_problem* const* P, const float* const* models,
                         const float* const* wavelets, const int32_t* const* srcs,
                         const int32_t* const* recs, float* const* data, void* const* wss,
                         int np, cudaStream_t st) {
  std::vector<Layout> Ls(np);
  std::vector<AcFwdLoop> F(np);
  std::vector<int> live;
  int ntmax = 0;
  for (int i = 0; i < np; ++i) {
    const sweep_problem* p = P[i];
    if (p->nshot == 0) continue;
    Ls[i] = layout(p, SWEEP_MODE_FORWARD);
    launch_setup(setup_args(p, Ls[i], wss[i], models[i], srcs[i], recs[i]), st);
    const int rc = F[i].init(p, Ls[i], wss[i], wavelets[i], srcs[i], recs[i],
                             p->nrec > 0 ? data[i] : nullptr, false, st);
    if (rc) return rc;
    live.push_back(i);
    ntmax = std::max(ntmax, p->nt);
  }
  if (live.empty()) return SWEEP_OK;
  if (P[0]->flags & SWEEP_F_ONE_LAUNCH) {
    std::vector<LoopProblem> lp(np);
    return loop_forward(P, F, Ls, wss, live, lp, ntmax, st);
  }
  AcInFwdArgs fin[kStepBatch];
  AcFixArgs fix[kStepBatch];
  for (int t = 0; t < ntmax; ++t) {
    int k = 0;
    for (int i : live) {
      if (t >= P[i]->nt) continue;
      F[i].step(t);
      fin[k] = F[i].in;
      fix[k] = F[i].fx;
      ++k;
    }
    launch_ac_in_fwd_batch(fin, k, st);
    launch_ac_fix_fwd_batch(fix, k, st);
  }
  return SWEEP_OK;
}

int sweep_forward_batch(int nprob, const sweep_problem* probs, const float* const* models,
                        const float* const* wavelets, const int32_t* const* srcs,
                        const int32_t* const* recs, float* const* data, void* const* ws,
                        const size_t* ws_bytes, void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (nprob < 0) return SWEEP_EINVAL;
  if (nprob == 0) return SWEEP_OK;
  if (!probs || !models || !wavelets || !srcs || !recs || !data || !ws || !ws_bytes)
    return SWEEP_EINVAL;
  for (int i = 0; i < nprob; ++i) {  // every problem checked before any launch
    const sweep_problem* p = &probs[i];
    if (!valid_problem(p)) return SWEEP_EINVAL;
    if (p->physics != SWEEP_ACOUSTIC) return SWEEP_EUNSUPPORTED;
    if ((p->flags ^ probs[0].flags) & (SWEEP_F_ONE_LAUNCH | SWEEP_F_DETERMINISTIC))
      return SWEEP_EINVAL;  // the problems of one launch share these modes
    if (unsupported_combination(p)) return SWEEP_EUNSUPPORTED;
    const int rc = check_ws(p, SWEEP_MODE_FORWARD, ws[i], ws_bytes[i]);
    if (rc) return rc;
    if (!models[i]) return SWEEP_EINVAL;
    if (p->nshot > 0 && (!wavelets[i] || !srcs[i])) return SWEEP_EINVAL;
    if (p->nshot > 0 && p->nrec > 0 && (!recs[i] || !data[i])) return SWEEP_EINVAL;
    for (int j = 0; j < i; ++j)
      if (ws[j] == ws[i]) return SWEEP_EWORKSPACE;
  }
  for (int i = 0; i < nprob; ++i) {
    const int rc = begin(&probs[i], SWEEP_MODE_FORWARD, ws[i], ws_bytes[i], st);
    if (rc) return rc;
  }
  const sweep_problem* P[kStepBatch];
  for (int g0 = 0; g0 < nprob; g0 += kStepBatch) {
    const int np = std::min(kStepBatch, nprob - g0);
    for (int i = 0; i < np; ++i) P[i] = &probs[g0 + i];
    const int rc = forward_group(P, models + g0, wavelets + g0, srcs + g0, recs + g0,
                                 data + g0, ws + g0, np, st);
    if (rc) return rc;
  }
  return cuda_rc(cudaGetLastError());
}

int sweep_gradient_batch(int nprob, const sweep_problem* probs, const float* const* models,
                         const float* const* wavelets, const int32_t* const* srcs,
                         const int32_t* const* recs, const float* const* d_obs,
                         float* const* grads, double* const* misfits, void* const* ws,
                         const size_t* ws_bytes, void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (nprob < 0) return SWEEP_EINVAL;
  if (nprob == 0) return SWEEP_OK;
  if (!probs || !models || !wavelets || !srcs || !recs || !d_obs || !grads || !misfits ||
      !ws || !ws_bytes)
    return SWEEP_EINVAL;
  // every problem checked on the host before anything is launched
  for (int i = 0; i < nprob; ++i) {
    const sweep_problem* p = &probs[i];
    if (!valid_problem(p)) return SWEEP_EINVAL;
    if (p->physics != SWEEP_ACOUSTIC) return SWEEP_EUNSUPPORTED;
    if ((p->flags ^ probs[0].flags) & (SWEEP_F_ONE_LAUNCH | SWEEP_F_DETERMINISTIC))
      return SWEEP_EINVAL;  // the problems of one launch share these modes
    if (unsupported_combination(p)) return SWEEP_EUNSUPPORTED;
    const int rc = check_ws(p, SWEEP_MODE_GRADIENT, ws[i], ws_bytes[i]);
    if (rc) return rc;
    if (!models[i] || !grads[i] || !misfits[i]) return SWEEP_EINVAL;
    if (p->nshot > 0 && (!wavelets[i] || !srcs[i])) return SWEEP_EINVAL;
    if (p->nshot > 0 && p->nrec > 0 && (!recs[i] || !d_obs[i])) return SWEEP_EINVAL;
    for (int j = 0; j < i; ++j)
      if (ws[j] == ws[i]) return SWEEP_EWORKSPACE;  // one workspace per problem
  }
  for (int i = 0; i < nprob; ++i) {
    const int rc = begin(&probs[i], SWEEP_MODE_GRADIENT, ws[i], ws_bytes[i], st);
    if (rc) return rc;
  }
  const sweep_problem* P[kStepBatch];
  for (int g0 = 0; g0 < nprob; g0 += kStepBatch) {
    const int np = std::min(kStepBatch, nprob - g0);
    for (int i = 0; i < np; ++i) P[i] = &probs[g0 + i];
    const int rc = gradient_group(P, models + g0, wavelets + g0, srcs + g0, recs + g0,
                                  d_obs + g0, grads + g0, misfits + g0, ws + g0, np, st);
    if (rc) return rc;
  }
  return cuda_rc(cudaGetLastError());
}

size_t sweep_dot_workspace_bytes(void) { return sizeof(double) * RED_BLOCKS; }

int sweep_dot(const float* a, const float* b, int64_t n, double* out, void* ws,
              size_t ws_bytes, void* stream) {
  if (n < 0 || !out || (n > 0 && (!a || !b))) return SWEEP_EINVAL;
  if (!ws || ws_bytes < sweep_dot_workspace_bytes() ||
      (reinterpret_cast<uintptr_t>(ws) % 8) != 0)
    return SWEEP_EWORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  launch_dot(a, b, n, static_cast<double*>(ws), RED_BLOCKS, out, st);
  note_launches(2);
  return cuda_rc(cudaGetLastError());
}

int sweep_status(void* ws, void* stream) {
  if (!ws) return SWEEP_EWORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, ws, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return SWEEP_ECUDA;
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return SWEEP_ECUDA;
  return h;
}

unsigned long long sweep_kernel_launches(void) { return g_launches.load(); }

const char* sweep_strerror(int code) {
  switch (code) {
    case SWEEP_OK: return "ok";
    case SWEEP_EINVAL: return "invalid argument";
    case SWEEP_ECFL: return "time step above the stability (CFL) limit";
    case SWEEP_EBOUNDS: return "source or receiver outside the interior grid";
    case SWEEP_EWORKSPACE: return "workspace missing, misaligned or too small";
    case SWEEP_ECUDA: return "CUDA runtime error";
    case SWEEP_ETIMEOUT: return "bounded device-side wait timed out";
    case SWEEP_ENONFINITE: return "non-finite model value or misfit";
    case SWEEP_EMODEL: return "non-physical model value";
    case SWEEP_EUNSUPPORTED: return "not implemented for this physics";
    case SWEEP_ETOOBIG: return "size above a fixed internal capacity";
    default: return "unknown error";
  }
}

}  // extern "C"
