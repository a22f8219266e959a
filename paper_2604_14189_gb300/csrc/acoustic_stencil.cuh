// Device code of the acoustic stencil kernels (acoustic_interior.cu), shared
// with the time-loop kernels of acoustic_loop.cu: the tile shapes, the unit
// descriptors and one CTA's share of a forward or backward stencil step
// (fwd_body, bwd_body).  A body reads the step's scalars from a StepCtl.
// PDL = true: the body runs in a per-step kernel started by programmatic
// dependent launch (it waits for the previous kernel after its prologue and
// lets the next one start before its last unit); false: it runs inside a
// kernel that orders its phases with grid barriers, so it fences the
// generic-proxy writes of earlier phases before its TMA reads and
// invalidates its mbarriers on return.
#pragma once

#include <algorithm>

#include "acoustic_common.cuh"
#include "tma.cuh"

namespace sweep {
namespace {


constexpr int FWD_THREADS = 256;
constexpr int BWD_ROLE_WARPS = 8;  // backward: 8 adjoint + 8 imaging warps
constexpr int BWD_THREADS = 64 * BWD_ROLE_WARPS;

// Shared-memory stages of a tile height BZ.  Heights and stage counts chosen
// by sweeps on GB300 (301x901+40, 20 shots): forward 32 rows x 4 stages
// (16 x 6, 32 x 3, 48 x 2, 64 x 2 no better); backward 32 rows x 2 stages,
// 230 KB of shared memory with the static tables (16 x 3 was 0.5 % slower
// over the whole gradient).  The 16-row tiles (forward 7 stages, backward
// 3) give small grids twice the units.
template <int BZ>
struct FwdTile {
  static constexpr int RPW = BZ / (FWD_THREADS / 32);  // rows per warp
  static constexpr int HF = IN_HW * (BZ + 8);          // floats, halo tile
  static constexpr int CF = IN_BX * BZ;                // floats, centre tile
  static constexpr int STAGES = BZ == IN_BZ ? 4 : 7;
  static constexpr uint32_t BYTES = (HF + 2 * CF) * 4;
  struct __align__(128) Stage {
    float u[HF];   // u^n with halo
    float up[CF];  // u^{n-1}
    float k[CF];   // K
  };
  static constexpr size_t SMEM = STAGES * sizeof(Stage) + 8 * STAGES;
  static_assert((HF * 4) % 128 == 0 && (CF * 4) % 128 == 0, "alignment");
  static_assert(RPW * (FWD_THREADS / 32) == BZ, "rows per warp");
};
template <int BZ>
struct BwdTile {
  static constexpr int RPW = BZ / BWD_ROLE_WARPS;
  static constexpr int HF = IN_HW * (BZ + 8);
  static constexpr int CF = IN_BX * BZ;
  static constexpr int STAGES = BZ == IN_BZ ? 2 : 3;
  struct __align__(128) Stage {
    float ua[HF];  // u^n with halo
    float ma[HF];  // mu^{n+1} with halo
    float ub[CF];  // u^{n+1}
    float mb[CF];  // mu^{n+2}
    float k[CF];   // K
    float gr[CF];  // imaging accumulator of this shot
  };
  static constexpr size_t SMEM = STAGES * sizeof(Stage) + 8 * STAGES;
  static_assert((HF * 4) % 128 == 0 && (CF * 4) % 128 == 0, "alignment");
  static_assert(RPW * BWD_ROLE_WARPS == BZ, "rows per warp");
  static_assert(STAGES >= 2, "the ring prefetch reads a descriptor written two barriers earlier");
};
constexpr size_t kFwdSmem = std::max(FwdTile<IN_BZ>::SMEM, FwdTile<IN_BZ_SMALL>::SMEM);
constexpr size_t kBwdSmem = std::max(BwdTile<IN_BZ>::SMEM, BwdTile<IN_BZ_SMALL>::SMEM);
constexpr int kMaxStages = 7;
static_assert(FwdTile<IN_BZ_SMALL>::STAGES <= kMaxStages && BwdTile<IN_BZ_SMALL>::STAGES <= kMaxStages,
              "descriptor ring");

__device__ __forceinline__ float4 lds4(const float* t, int pitch, int r, int c) {
  return *reinterpret_cast<const float4*>(t + r * pitch + c);
}

struct UnitPos {
  int s, z0, x0;
};

// What a backward unit touches: interior cells (imaging, reconstruction).
struct BwdFlags {
  bool imgt, needu1;
};
__device__ __forceinline__ BwdFlags bwd_flags(const Geom& g, bool img, bool rec,
                                              const UnitPos& p, int bz) {
  const int z1 = p.z0 + bz, x1 = p.x0 + IN_BX;
  const bool touch_int = z1 > g.P && p.z0 < g.P + g.nz && x1 > g.P && p.x0 < g.P + g.nx;
  BwdFlags f;
  f.imgt = img && touch_int;
  f.needu1 = rec && f.imgt;
  return f;
}

__device__ __forceinline__ UnitPos unit_pos(const Region& R, int S, int ntx, int bz, int unit) {
  const int tile = unit / S;
  UnitPos p;
  p.s = unit - tile * S;
  const int tz = tile / ntx, tx = tile - tz * ntx;
  p.z0 = R.z0 + tz * bz;
  p.x0 = R.x0 + tx * IN_BX;
  return p;
}

// The scalars of one step that a body reads (the per-step kernels take
// them from their arguments, the time-loop kernels from the loop counter).
struct StepCtl {
  int n;
  int do_adj, do_img, do_rec;  // backward only
};

// Per-unit facts, computed once by the thread that issues the unit's
// transfers and read by every thread from shared memory.
enum : int {
  U_IMG = 1,   // meets the interior: imaging (backward)
  U_U1 = 4,    // needs u^{n+1} (reconstruction, backward)
  U_SRC = 8,   // holds the source cell
  U_REC = 16,  // holds receivers (backward): their count is flags >> 8
};
struct UnitDesc {
  int s, z0, x0, flags;
  int sz, sx;  // source cell (padded coordinates)
  float fn;    // wavelet sample of this step (0 where not needed)
  int rec;     // U_REC: offset of the unit's receivers in rlist
};
// Descriptors of a CTA's first kUnitTable units are computed by all its
// threads in the prologue; later units (large batches) are described by the
// issuing thread into a ring beside the stages.
constexpr int kUnitTable = 256;

__device__ __forceinline__ UnitDesc make_desc(const Region& R, const Geom& g, const ShotTable& T,
                                              const AcInFwdArgs* af, const AcInBwdArgs* ab,
                                              const StepCtl& c, int bz, int unit) {
  const int S = g.nshot;
  const int ntx = af ? af->ntx : ab->ntx;
  const UnitPos p = unit_pos(R, S, ntx, bz, unit);
  const bool img = ab && c.do_img;
  const ShotInfo si =
      af ? shot_info(T, g, af->src, af->wavelet, c.n, p.s)
         : shot_info(T, g, ab->src, img ? ab->wavelet : nullptr, c.n, p.s);
  UnitDesc d;
  d.s = p.s;
  d.z0 = p.z0;
  d.x0 = p.x0;
  d.sz = si.sz;
  d.sx = si.sx;
  d.fn = si.fn;
  d.rec = 0;
  int f = 0;
  if (si.sz >= p.z0 && si.sz < p.z0 + bz && si.sx >= p.x0 && si.sx < p.x0 + IN_BX &&
      in_region(R, si.sz, si.sx))
    f |= U_SRC;
  if (ab) {
    const BwdFlags b = bwd_flags(g, img, c.do_rec != 0, p, bz);
    f |= (b.imgt ? U_IMG : 0) | (b.needu1 ? U_U1 : 0);
    if (ab->rtile && c.do_adj) {
      const int2 oc = ab->rtile[unit];
      if (oc.y > 0) {
        f |= U_REC | (oc.y << 8);
        d.rec = oc.x;
      }
    }
  }
  d.flags = f;
  return d;
}

// -------------------------------------------------------------- forward
// Invalidates a body's mbarriers once no transfer is in flight (the next
// body run by the same CTA initialises them again).
__device__ __forceinline__ void release_barriers(uint64_t* bar, int D) {
  __syncthreads();
  if (threadIdx.x == 0)
    for (int i = 0; i < D; ++i) mbar_inval(&bar[i]);
  __syncthreads();
}

// One CTA's units of a forward step, for tiles of BZ rows.  T, desc and
// utab are the kernel's static shared tables (one set for both heights).
// Returns false when a transfer never landed (SWEEP_ETIMEOUT latched).
template <int BZ, bool PDL>
__device__ __forceinline__ bool fwd_body(const AcInFwdArgs& a, const StepCtl& c, int bx, int G,
                                         ShotTable& T, UnitDesc* desc, UnitDesc* utab,
                                         unsigned char* smem_raw) {
  using C = FwdTile<BZ>;
  using Stage = typename C::Stage;
  constexpr int D = C::STAGES;
  Stage* stg = reinterpret_cast<Stage*>(smem_raw);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + D * sizeof(Stage));
  const Geom& g = a.g;
  const Region& R = g.fin;
  const int count = (a.units - bx + G - 1) / G;  // units b, b+G, ...
  if (count <= 0) {
    if constexpr (PDL) grid_dep_wait();
    return true;
  }
  load_shot_table(T, g, a.src, a.wavelet, c.n);
  __syncthreads();  // shot table visible
  for (int i = threadIdx.x; i < count && i < kUnitTable; i += FWD_THREADS)
    utab[i] = make_desc(R, g, T, &a, nullptr, c, BZ, bx + i * G);
  if (threadIdx.x == 0) {
    for (int i = 0; i < D; ++i) mbar_init(&bar[i], 1);
    fence_barrier_init();
  }
  // The prologue above reads only the call's inputs (geometry, sources,
  // wavelets), which no kernel of the library writes, so it overlaps the
  // previous kernel's tail; the fields are read after this wait.
  if constexpr (PDL) grid_dep_wait();
  // (time loop) every thread's generic use of the stage memory in the
  // previous phase before the copies below write it
  if constexpr (!PDL) fence_proxy_async_smem();
  if (__syncthreads_or(threadIdx.x == 0 && *a.status != 0)) {
    if constexpr (!PDL) release_barriers(bar, D);
    return true;
  }
  // the unit's descriptor is stored before the arrive on its barrier, so a
  // thread that has waited on the barrier sees it
  auto issue = [&](int k) {
    UnitDesc d;
    if (k < kUnitTable) {
      d = utab[k];
    } else {
      d = make_desc(R, g, T, &a, nullptr, c, BZ, bx + k * G);
      desc[k % D] = d;
    }
    Stage& sg = stg[k % D];
    uint64_t* b = &bar[k % D];
    mbar_arrive_expect_tx(b, C::BYTES);
    tma_load_3d(sg.u, &a.tu, b, d.x0 - 4, d.z0 - 4, d.s);
    tma_load_3d(sg.up, &a.tup, b, d.x0, d.z0, d.s);
    tma_load_2d(sg.k, &a.tK, b, d.x0, d.z0);
  };
  if (threadIdx.x == 0) {
    if constexpr (!PDL) {
      fence_proxy_async_global();  // earlier phases' stores before these loads
      fence_proxy_async_smem();    // and the stage memory's generic use
    }
    for (int k = 0; k < D && k < count; ++k) issue(k);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lx = 4 * lane, r0 = warp * C::RPW;
  int k = 0;
  for (; k < count; ++k) {
    if constexpr (PDL)
      if (k == count - 1) grid_dep_trigger();  // the next kernel may start
    // one CTA barrier per unit: each thread waits for the stage itself, and
    // the barrier after the unit both releases the stage and agrees on a
    // transfer that never landed
    const bool got = mbar_wait(&bar[k % D], (k / D) & 1);
    const UnitDesc d = k < kUnitTable ? utab[k] : desc[k % D];
    const Stage& sg = stg[k % D];
    const long long so = (long long)d.s * g.fstride;
    const int gx = d.x0 + lx;
    if (got) {
    float w[9][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) f4a(lds4(sg.u, IN_HW, r0 + j, lx + 4), w[j]);
#pragma unroll
    for (int q = 0; q < C::RPW; ++q) {
      f4a(lds4(sg.u, IN_HW, r0 + q + 8, lx + 4), w[8]);
      const int gz = d.z0 + r0 + q;
      if (gz < R.z1 && gx < R.x1) {
        float e[12], up[4], kk[4], out[4];
        f4a(lds4(sg.u, IN_HW, r0 + q + 4, lx), e);
        f4a(lds4(sg.u, IN_HW, r0 + q + 4, lx + 8), e + 8);
#pragma unroll
        for (int c = 0; c < 4; ++c) e[4 + c] = w[4][c];
        f4a(lds4(sg.up, IN_BX, r0 + q, lx), up);
        f4a(lds4(sg.k, IN_BX, r0 + q, lx), kk);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float lap =
              d2(e[c], e[c + 1], e[c + 2], e[c + 3], e[c + 4], e[c + 5], e[c + 6], e[c + 7],
                 e[c + 8]) +
              d2(w[0][c], w[1][c], w[2][c], w[3][c], w[4][c], w[5][c], w[6][c], w[7][c], w[8][c]);
          out[c] = 2.f * w[4][c] - up[c] + kk[c] * lap;
        }
        if ((d.flags & U_SRC) && gz == d.sz) {
#pragma unroll
          for (int c = 0; c < 4; ++c)
            if (gx + c == d.sx) out[c] += kk[c] * d.fn;
        }
        *reinterpret_cast<float4*>(a.un + so + (long long)gz * g.NXp + gx) =
            make_float4(out[0], out[1], out[2], out[3]);
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
#pragma unroll
        for (int c = 0; c < 4; ++c) w[j][c] = w[j + 1][c];
      }
    }
    }  // got
    if (__syncthreads_or(!got)) break;  // stage released
    if (threadIdx.x == 0 && k + D < count) {
      fence_proxy_async_smem();
      issue(k + D);
    }
  }
  if (k < count) {
    if (threadIdx.x == 0) {
      // a transfer never landed: report, drain what is still in flight
      latch(a.status, SWEEP_ETIMEOUT);
      for (int j = k; j < count && j < k + D; ++j) mbar_wait(&bar[j % D], (j / D) & 1);
    }
    return false;
  }
  if constexpr (!PDL) release_barriers(bar, D);
  return true;
}

// -------------------------------------------------------------- backward
// INJ: deterministic mode, the adjoint warps inject the residual at the
// unit's receivers (a.rtile / a.rlist) instead of the CPML kernel.
template <int BZ, bool PDL, bool INJ>
__device__ __forceinline__ bool bwd_body(const AcInBwdArgs& a, const StepCtl& c, int bx, int G,
                                         ShotTable& T, UnitDesc* desc, UnitDesc* utab,
                                         unsigned char* smem_raw) {
  using C = BwdTile<BZ>;
  using Stage = typename C::Stage;
  constexpr int D = C::STAGES;
  constexpr int HF = C::HF, CF = C::CF, RPW = C::RPW;
  Stage* stg = reinterpret_cast<Stage*>(smem_raw);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + D * sizeof(Stage));
  const Geom& g = a.g;
  const Region& R = g.bin;
  const int count = (a.units - bx + G - 1) / G;
  if (count <= 0) {
    if constexpr (PDL) grid_dep_wait();
    return true;
  }
  const bool img = c.do_img != 0, adj = c.do_adj != 0;
  load_shot_table(T, g, a.src, img ? a.wavelet : nullptr, c.n);
  __syncthreads();  // shot table visible
  for (int i = threadIdx.x; i < count && i < kUnitTable; i += BWD_THREADS)
    utab[i] = make_desc(R, g, T, nullptr, &a, c, BZ, bx + i * G);
  if (threadIdx.x == 0) {
    for (int i = 0; i < D; ++i) mbar_init(&bar[i], 1);
    fence_barrier_init();
  }
  // inputs only above (see the forward body); the fields after the wait
  if constexpr (PDL) grid_dep_wait();
  // (time loop) every thread's generic use of the stage memory in the
  // previous phase before the copies below write it
  if constexpr (!PDL) fence_proxy_async_smem();
  if (__syncthreads_or(threadIdx.x == 0 && *a.status != 0)) {
    if constexpr (!PDL) release_barriers(bar, D);
    return true;
  }
  auto issue = [&](int k) {
    UnitDesc d;
    if (k < kUnitTable) {
      d = utab[k];
    } else {
      d = make_desc(R, g, T, nullptr, &a, c, BZ, bx + k * G);
      desc[k % D] = d;
    }
    Stage& sg = stg[k % D];
    uint64_t* b = &bar[k % D];
    const bool imgt = d.flags & U_IMG;
    mbar_arrive_expect_tx(b, (HF + CF) * 4 + (imgt ? (HF + CF) * 4 : 0) +
                                 ((d.flags & U_U1) ? CF * 4 : 0) + (adj ? CF * 4 : 0));
    tma_load_3d(sg.ma, &a.tmA, b, d.x0 - 4, d.z0 - 4, d.s);
    tma_load_2d(sg.k, &a.tK, b, d.x0, d.z0);
    if (imgt) {
      tma_load_3d(sg.ua, &a.tuA, b, d.x0 - 4, d.z0 - 4, d.s);
      tma_load_3d(sg.gr, &a.tG, b, d.x0, d.z0, d.s);
    }
    if (d.flags & U_U1) tma_load_3d(sg.ub, &a.tuB, b, d.x0, d.z0, d.s);
    if (adj) tma_load_3d(sg.mb, &a.tmB, b, d.x0, d.z0, d.s);
  };
  if (threadIdx.x == 0) {
    if constexpr (!PDL) {
      fence_proxy_async_global();  // earlier phases' stores before these loads
      fence_proxy_async_smem();    // and the stage memory's generic use
    }
    for (int k = 0; k < D && k < count; ++k) issue(k);
  }
  __syncthreads();  // first descriptors visible before the ring prefetch below
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // warps 0..7: adjoint update of mu; warps 8..15: imaging and the
  // reconstruction of u.  Each owns RPW rows of the tile.
  const bool adj_warp = warp < BWD_ROLE_WARPS;
  const int lx = 4 * lane, r0 = (warp % BWD_ROLE_WARPS) * RPW;
  int k = 0;
  for (; k < count; ++k) {
    if constexpr (PDL)
      // the next (CPML) kernel may start with this CTA's second-to-last unit:
      // its blocks fit beside the stencil CTA and issue their loads during
      // the tail (measured: one unit earlier 230.5 ms per gradient, the last
      // unit 232.0, two units earlier 233.9)
      if (k == (count > 1 ? count - 2 : 0)) grid_dep_trigger();
    const UnitDesc d = k < kUnitTable ? utab[k] : desc[k % D];
    const bool imgt = d.flags & U_IMG, needu1 = d.flags & U_U1;
    const int gx = d.x0 + lx;
    // one CTA barrier per unit (see the forward body)
    const bool got = mbar_wait(&bar[k % D], (k / D) & 1);
    const Stage& sg = stg[k % D];
    const long long so = (long long)d.s * g.fstride;
    if (!got) {
      // a transfer never landed: the barrier below ends the loop
    } else if (adj_warp) {
      if (adj) {
        // mu^n = 2 mu^{n+1} - mu^{n+2} + K Lap mu^{n+1} + K R^T r^{n-1}: the
        // residual of this warp's receivers gathered first, in receiver
        // order (a cell holding two receivers takes both)
        float inj[RPW][4];
#pragma unroll
        for (int q = 0; q < RPW; ++q)
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) inj[q][cc] = 0.f;
        if (INJ && (d.flags & U_REC)) {
          // the unit's receivers 32 at a time, one per lane; those in this
          // warp's rows are handed to the lane owning their column, in list
          // order (a cell holding two receivers takes both, always in the
          // same order)
          const int cnt = d.flags >> 8;
          const int4* rl = a.rlist + d.rec;
          for (int j0 = 0; j0 < cnt; j0 += 32) {
            const int j = j0 + lane;
            int qr = -1, cr = 0;
            float v = 0.f;
            if (j < cnt) {
              const int4 e = rl[j];  // (receiver, z, x)
              qr = e.y - (d.z0 + r0);
              cr = e.z - d.x0;
              if (qr >= 0 && qr < RPW)
                v = a.res[((long long)d.s * g.nrec + e.x) * g.nt + (c.n - 1)];
              else
                qr = -1;
            }
            unsigned todo = __ballot_sync(0xffffffffu, qr >= 0);
            while (todo) {
              const int src = __ffs(todo) - 1;
              todo &= todo - 1;
              const int q2 = __shfl_sync(0xffffffffu, qr, src);
              const int c2 = __shfl_sync(0xffffffffu, cr, src);
              const float v2 = __shfl_sync(0xffffffffu, v, src);
              const float add = (c2 >> 2) == lane ? v2 : 0.f;  // the owning lane's
#pragma unroll
              for (int q = 0; q < RPW; ++q)
#pragma unroll
                for (int cc = 0; cc < 4; ++cc)
                  inj[q][cc] += (q == q2 && cc == (c2 & 3)) ? add : 0.f;
            }
          }
        }
        float wm[9][4];
#pragma unroll
        for (int j = 0; j < 8; ++j) f4a(lds4(sg.ma, IN_HW, r0 + j, lx + 4), wm[j]);
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
          f4a(lds4(sg.ma, IN_HW, r0 + q + 8, lx + 4), wm[8]);
          const int gz = d.z0 + r0 + q;
          if (gz < R.z1 && gx < R.x1) {
            float e[12], m2[4], kk[4], out[4];
            f4a(lds4(sg.ma, IN_HW, r0 + q + 4, lx), e);
            f4a(lds4(sg.ma, IN_HW, r0 + q + 4, lx + 8), e + 8);
#pragma unroll
            for (int c = 0; c < 4; ++c) e[4 + c] = wm[4][c];
            f4a(lds4(sg.mb, IN_BX, r0 + q, lx), m2);
            f4a(lds4(sg.k, IN_BX, r0 + q, lx), kk);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              const float lap =
                  d2(e[c], e[c + 1], e[c + 2], e[c + 3], e[c + 4], e[c + 5], e[c + 6],
                     e[c + 7], e[c + 8]) +
                  d2(wm[0][c], wm[1][c], wm[2][c], wm[3][c], wm[4][c], wm[5][c], wm[6][c],
                     wm[7][c], wm[8][c]);
              out[c] = 2.f * wm[4][c] - m2[c] + kk[c] * lap;
              if (INJ && (d.flags & U_REC)) out[c] += kk[c] * inj[q][c];
            }
            *reinterpret_cast<float4*>(a.mB + so + (long long)gz * g.NXp + gx) =
                make_float4(out[0], out[1], out[2], out[3]);
          }
#pragma unroll
          for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int c = 0; c < 4; ++c) wm[j][c] = wm[j + 1][c];
        }
      }
    } else if (imgt) {
      // interior columns among this lane's 4 cells
      unsigned cmask = 0;
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (gx + c >= g.P && gx + c < g.P + g.nx) cmask |= 1u << c;
      float wu[9][4];
      if (imgt) {
#pragma unroll
        for (int j = 0; j < 8; ++j) f4a(lds4(sg.ua, IN_HW, r0 + j, lx + 4), wu[j]);
      }
#pragma unroll
      for (int q = 0; q < RPW; ++q) {
        if (imgt) f4a(lds4(sg.ua, IN_HW, r0 + q + 8, lx + 4), wu[8]);
        const int gz = d.z0 + r0 + q;
        if (gz < R.z1 && gx < R.x1) {
          const long long ci = so + (long long)gz * g.NXp + gx;
          // interior cells of this lane in this row
          const unsigned im = (imgt && gz >= g.P && gz < g.P + g.nz) ? cmask : 0u;
          float lap[4] = {0.f, 0.f, 0.f, 0.f};
          if (im) {
            // imaging: graw += mu^{n+1} (Lap u^n + f^n delta_s)
            float e[12], m1[4], gvv[4];
            f4a(lds4(sg.ua, IN_HW, r0 + q + 4, lx), e);
            f4a(lds4(sg.ua, IN_HW, r0 + q + 4, lx + 8), e + 8);
#pragma unroll
            for (int c = 0; c < 4; ++c) e[4 + c] = wu[4][c];
#pragma unroll
            for (int c = 0; c < 4; ++c)
              lap[c] = d2(e[c], e[c + 1], e[c + 2], e[c + 3], e[c + 4], e[c + 5], e[c + 6],
                          e[c + 7], e[c + 8]) +
                       d2(wu[0][c], wu[1][c], wu[2][c], wu[3][c], wu[4][c], wu[5][c],
                          wu[6][c], wu[7][c], wu[8][c]);
            if ((d.flags & U_SRC) && gz == d.sz) {
#pragma unroll
              for (int c = 0; c < 4; ++c)
                if (gx + c == d.sx) lap[c] += d.fn;
            }
            f4a(lds4(sg.ma, IN_HW, r0 + q + 4, lx + 4), m1);
            f4a(lds4(sg.gr, IN_BX, r0 + q, lx), gvv);
#pragma unroll
            for (int c = 0; c < 4; ++c)
              if ((im >> c) & 1u) gvv[c] += m1[c] * lap[c];
            *reinterpret_cast<float4*>(a.graw + ci) =
                make_float4(gvv[0], gvv[1], gvv[2], gvv[3]);
            if (a.illum) {
              float iv[4];
              f4a(*reinterpret_cast<const float4*>(a.illum + ci), iv);
#pragma unroll
              for (int c = 0; c < 4; ++c)
                if ((im >> c) & 1u) iv[c] += wu[4][c] * wu[4][c];
              *reinterpret_cast<float4*>(a.illum + ci) =
                  make_float4(iv[0], iv[1], iv[2], iv[3]);
            }
          }
          if (needu1 && im) {
            // u^{n-1} on interior cells; the ring is restored from the
            // forward save by the step's second kernel, and cells beyond it
            // are never read again (they keep u^{n+1})
            float u1[4], kk[4], out[4];
            f4a(lds4(sg.ub, IN_BX, r0 + q, lx), u1);
            f4a(lds4(sg.k, IN_BX, r0 + q, lx), kk);
#pragma unroll
            for (int c = 0; c < 4; ++c)
              out[c] = ((im >> c) & 1u) ? 2.f * wu[4][c] - u1[c] + kk[c] * lap[c] : u1[c];
            *reinterpret_cast<float4*>(a.uB + ci) = make_float4(out[0], out[1], out[2], out[3]);
          }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
          for (int c = 0; c < 4; ++c) wu[j][c] = wu[j + 1][c];
      }
    }
    // adjoint source gather: f-bar^n = mu^{n+1}(s)
    if (got && a.wgrad && threadIdx.x == 0 && c.n < g.nt && (d.flags & U_SRC))
      a.wgrad[(long long)d.s * g.nt + c.n] =
          sg.ma[(d.sz - d.z0 + 4) * IN_HW + (d.sx - d.x0 + 4)];
    if (__syncthreads_or(!got)) break;  // stage released
    if (threadIdx.x == 0 && k + D < count) {
      fence_proxy_async_smem();
      issue(k + D);
    }
  }
  if (k < count) {
    if (threadIdx.x == 0) {
      latch(a.status, SWEEP_ETIMEOUT);
      for (int j = k; j < count && j < k + D; ++j) mbar_wait(&bar[j % D], (j / D) & 1);
    }
    return false;
  }
  if constexpr (!PDL) release_barriers(bar, D);
  return true;
}

}  // namespace
}  // namespace sweep
