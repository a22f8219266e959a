/*
 * FP64 CPU oracle: isotropic elastic velocity-stress engine (Sec. 3.5,
 * Eq. 12; test infrastructure only).
 *
 * Staggered grid, cell (i, j) = (z, x):
 *   txx, tzz, lambda, mu at (i, j);  vx at (i, j+1/2);  vz at (i+1/2, j);
 *   txz at (i+1/2, j+1/2).
 * Buoyancy at a velocity point is the inverse of the arithmetic mean of the
 * two neighbouring densities; mu at a txz point is the harmonic mean of the
 * four neighbouring mu (0 if any is 0); neighbours past the grid edge are
 * clamped to the edge.  lambda = rho (vp^2 - 2 vs^2), mu = rho vs^2.
 * Differences: 4th-order staggered, coefficients 9/8 and -1/24.
 * Leapfrog: velocities live at n+1/2, stresses at n.  One step n:
 *   v^{n+1/2} = v^{n-1/2} + dt b (div tau^n)           (Eq. 12, rows 1-2)
 *   record vx, vz at n+1/2
 *   tau^{n+1} = tau^n + dt C (grad v^{n+1/2})         (Eq. 12, rows 3-5)
 *   explosive source: txx(s), tzz(s) += dt f^n / dx^2
 * Convolutional PML: every spatial derivative d/dx F taken at a point with
 * profile (a, b) is replaced by d/dx F + psi with psi = a psi + b d/dx F
 * (updated before use); the profile is sampled at the point's own (integer
 * or half-cell) position.
 */
#include "oracle_internal.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int NZ, NX, P;
  double* lam;  /* [NZ][NX] at (i, j) */
  double* mu;   /* [NZ][NX] at (i, j) */
  double* bux;  /* buoyancy at vx points */
  double* buz;  /* buoyancy at vz points */
  double* muxz; /* mu at txz points */
  double *ax, *bx, *axh, *bxh, *az, *bz, *azh, *bzh;
} egrid;

static inline double G(const egrid* g, const double* f, int i, int j) {
  if (i < 0 || i >= g->NZ || j < 0 || j >= g->NX) return 0.0;
  return f[(size_t)i * g->NX + j];
}
static inline int clampi(int v, int hi) { return v < 0 ? 0 : (v > hi ? hi : v); }

static void egrid_init(egrid* g, const oracle_problem* p, const double* m) {
  g->P = p->pml;
  g->NZ = p->nz + 2 * p->pml;
  g->NX = p->nx + 2 * p->pml;
  const int NZ = g->NZ, NX = g->NX;
  const size_t N = (size_t)NZ * NX;
  const double* vp = m;
  const double* vs = m + N;
  const double* rho = m + 2 * N;
  g->lam = malloc(N * sizeof(double));
  g->mu = malloc(N * sizeof(double));
  g->bux = malloc(N * sizeof(double));
  g->buz = malloc(N * sizeof(double));
  g->muxz = malloc(N * sizeof(double));
  double vmax = 0.0;
  for (size_t c = 0; c < N; ++c) {
    g->lam[c] = rho[c] * (vp[c] * vp[c] - 2.0 * vs[c] * vs[c]);
    g->mu[c] = rho[c] * vs[c] * vs[c];
    if (vp[c] > vmax) vmax = vp[c];
  }
  for (int i = 0; i < NZ; ++i)
    for (int j = 0; j < NX; ++j) {
      const size_t c = (size_t)i * NX + j;
      const int j1 = clampi(j + 1, NX - 1), i1 = clampi(i + 1, NZ - 1);
      g->bux[c] = 2.0 / (rho[c] + rho[(size_t)i * NX + j1]);
      g->buz[c] = 2.0 / (rho[c] + rho[(size_t)i1 * NX + j]);
      const double m00 = g->mu[c], m01 = g->mu[(size_t)i * NX + j1];
      const double m10 = g->mu[(size_t)i1 * NX + j], m11 = g->mu[(size_t)i1 * NX + j1];
      g->muxz[c] = (m00 == 0.0 || m01 == 0.0 || m10 == 0.0 || m11 == 0.0)
                       ? 0.0
                       : 4.0 / (1.0 / m00 + 1.0 / m01 + 1.0 / m10 + 1.0 / m11);
    }
  if (p->v_pml > 0.0) vmax = p->v_pml;
  g->ax = malloc(NX * sizeof(double)); g->bx = malloc(NX * sizeof(double));
  g->axh = malloc(NX * sizeof(double)); g->bxh = malloc(NX * sizeof(double));
  g->az = malloc(NZ * sizeof(double)); g->bz = malloc(NZ * sizeof(double));
  g->azh = malloc(NZ * sizeof(double)); g->bzh = malloc(NZ * sizeof(double));
  oracle_cpml_profile(p->nx, p->pml, p->dx, p->dt, vmax, p->f_ref, 0, g->ax, g->bx);
  oracle_cpml_profile(p->nx, p->pml, p->dx, p->dt, vmax, p->f_ref, 1, g->axh, g->bxh);
  oracle_cpml_profile(p->nz, p->pml, p->dx, p->dt, vmax, p->f_ref, 0, g->az, g->bz);
  oracle_cpml_profile(p->nz, p->pml, p->dx, p->dt, vmax, p->f_ref, 1, g->azh, g->bzh);
}

static void egrid_free(egrid* g) {
  free(g->lam); free(g->mu); free(g->bux); free(g->buz); free(g->muxz);
  free(g->ax); free(g->bx); free(g->axh); free(g->bxh);
  free(g->az); free(g->bz); free(g->azh); free(g->bzh);
}

/* staggered differences on the stored arrays, unit spacing */
/* forward: value at +1/2 from integer-indexed samples j, j+1 */
static inline double dpx(const egrid* g, const double* f, int i, int j) {
  return ORC_S1 * (G(g, f, i, j + 1) - G(g, f, i, j)) +
         ORC_S2 * (G(g, f, i, j + 2) - G(g, f, i, j - 1));
}
static inline double dmx(const egrid* g, const double* f, int i, int j) {
  return ORC_S1 * (G(g, f, i, j) - G(g, f, i, j - 1)) +
         ORC_S2 * (G(g, f, i, j + 1) - G(g, f, i, j - 2));
}
static inline double dpz(const egrid* g, const double* f, int i, int j) {
  return ORC_S1 * (G(g, f, i + 1, j) - G(g, f, i, j)) +
         ORC_S2 * (G(g, f, i + 2, j) - G(g, f, i - 1, j));
}
static inline double dmz(const egrid* g, const double* f, int i, int j) {
  return ORC_S1 * (G(g, f, i, j) - G(g, f, i - 1, j)) +
         ORC_S2 * (G(g, f, i + 1, j) - G(g, f, i - 2, j));
}

int oracle_elastic_forward(const oracle_problem* p, const double* model,
                           const double* wavelet, const int32_t* src,
                           const int32_t* rec, double* data, double* wavefield) {
  int rc = orc_check(p, src, rec);
  if (rc) return rc;
  double* m = orc_pad_model(p, model, 3);
  egrid g;
  egrid_init(&g, p, m);
  const int NZ = g.NZ, NX = g.NX, P = g.P, nt = p->nt;
  const size_t N = (size_t)NZ * NX;
  const double dt = p->dt, idx = 1.0 / p->dx;
#pragma omp parallel for schedule(dynamic, 1)
  for (int s = 0; s < p->nshot; ++s) {
    double* f = calloc(13 * N, sizeof(double));
    double *vx = f, *vz = f + N, *txx = f + 2 * N, *tzz = f + 3 * N, *txz = f + 4 * N;
    double *p1 = f + 5 * N, *p2 = f + 6 * N, *p3 = f + 7 * N, *p4 = f + 8 * N;
    double *p5 = f + 9 * N, *p6 = f + 10 * N, *p7 = f + 11 * N, *p8 = f + 12 * N;
    const size_t cs = (size_t)(src[2 * s] + P) * NX + src[2 * s + 1] + P;
    if (wavefield) memset(wavefield + (size_t)s * (nt + 1) * 5 * N, 0, 5 * N * sizeof(double));
    for (int n = 0; n < nt; ++n) {
      /* velocities from tau^n */
      for (int i = 0; i < NZ; ++i)
        for (int j = 0; j < NX; ++j) {
          const size_t c = (size_t)i * NX + j;
          const double dxt = dpx(&g, txx, i, j) * idx; /* at (i, j+1/2) */
          const double dzt = dmz(&g, txz, i, j) * idx; /* at (i, j+1/2) */
          p1[c] = g.axh[j] * p1[c] + g.bxh[j] * dxt;
          p2[c] = g.az[i] * p2[c] + g.bz[i] * dzt;
          vx[c] += dt * g.bux[c] * (dxt + p1[c] + dzt + p2[c]);
        }
      for (int i = 0; i < NZ; ++i)
        for (int j = 0; j < NX; ++j) {
          const size_t c = (size_t)i * NX + j;
          const double dxt = dmx(&g, txz, i, j) * idx; /* at (i+1/2, j) */
          const double dzt = dpz(&g, tzz, i, j) * idx; /* at (i+1/2, j) */
          p3[c] = g.ax[j] * p3[c] + g.bx[j] * dxt;
          p4[c] = g.azh[i] * p4[c] + g.bzh[i] * dzt;
          vz[c] += dt * g.buz[c] * (dxt + p3[c] + dzt + p4[c]);
        }
      for (int r = 0; r < p->nrec; ++r) {
        const int32_t* q = rec + 2 * ((size_t)s * p->nrec + r);
        const size_t cr = (size_t)(q[0] + P) * NX + q[1] + P;
        data[(((size_t)s * 2 + 0) * p->nrec + r) * nt + n] = vx[cr];
        data[(((size_t)s * 2 + 1) * p->nrec + r) * nt + n] = vz[cr];
      }
      /* stresses from v^{n+1/2} */
      for (int i = 0; i < NZ; ++i)
        for (int j = 0; j < NX; ++j) {
          const size_t c = (size_t)i * NX + j;
          const double exx = dmx(&g, vx, i, j) * idx; /* at (i, j) */
          const double ezz = dmz(&g, vz, i, j) * idx;
          p5[c] = g.ax[j] * p5[c] + g.bx[j] * exx;
          p6[c] = g.az[i] * p6[c] + g.bz[i] * ezz;
          const double ex = exx + p5[c], ez = ezz + p6[c];
          const double l2m = g.lam[c] + 2.0 * g.mu[c];
          txx[c] += dt * (l2m * ex + g.lam[c] * ez);
          tzz[c] += dt * (g.lam[c] * ex + l2m * ez);
        }
      for (int i = 0; i < NZ; ++i)
        for (int j = 0; j < NX; ++j) {
          const size_t c = (size_t)i * NX + j;
          const double ezx = dpz(&g, vx, i, j) * idx; /* at (i+1/2, j+1/2) */
          const double exz = dpx(&g, vz, i, j) * idx;
          p7[c] = g.azh[i] * p7[c] + g.bzh[i] * ezx;
          p8[c] = g.axh[j] * p8[c] + g.bxh[j] * exz;
          txz[c] += dt * g.muxz[c] * (ezx + p7[c] + exz + p8[c]);
        }
      const double amp = dt * wavelet[(size_t)s * nt + n] * idx * idx;
      txx[cs] += amp;
      tzz[cs] += amp;
      if (wavefield)
        memcpy(wavefield + ((size_t)s * (nt + 1) + n + 1) * 5 * N, f,
               5 * N * sizeof(double));
    }
    free(f);
  }
  egrid_free(&g);
  free(m);
  return 0;
}

/* ------------------------------------------------------------------------
 * Reverse mode: the exact transpose of the recurrence above, for the
 * adjoint-state gradient (Sec. 1 motivates gradients by the adjoint state;
 * here it is written out for this discrete scheme).
 *
 * One forward step, with the quantities its transpose needs:
 *   sx = dxt + p1' + dzt + p2'  (bracket of the vx update, p' = updated psi)
 *   sz = dxt + p3' + dzt + p4'  (bracket of the vz update)
 *   ex = exx + p5', ez = ezz + p6'  (normal strains)
 *   sxz = ezx + p7' + exz + p8'  (bracket of the txz update)
 * ------------------------------------------------------------------------ */
static void estep(const egrid* g, double dt, double idx, double* f, double amp, size_t cs,
                  double* sx, double* sz, double* ex, double* ez, double* sxz) {
  const int NZ = g->NZ, NX = g->NX;
  const size_t N = (size_t)NZ * NX;
  double *vx = f, *vz = f + N, *txx = f + 2 * N, *tzz = f + 3 * N, *txz = f + 4 * N;
  double *p1 = f + 5 * N, *p2 = f + 6 * N, *p3 = f + 7 * N, *p4 = f + 8 * N;
  double *p5 = f + 9 * N, *p6 = f + 10 * N, *p7 = f + 11 * N, *p8 = f + 12 * N;
  for (int i = 0; i < NZ; ++i)
    for (int j = 0; j < NX; ++j) {
      const size_t c = (size_t)i * NX + j;
      const double dxt = dpx(g, txx, i, j) * idx, dzt = dmz(g, txz, i, j) * idx;
      p1[c] = g->axh[j] * p1[c] + g->bxh[j] * dxt;
      p2[c] = g->az[i] * p2[c] + g->bz[i] * dzt;
      sx[c] = dxt + p1[c] + dzt + p2[c];
    }
  for (int i = 0; i < NZ; ++i)
    for (int j = 0; j < NX; ++j) {
      const size_t c = (size_t)i * NX + j;
      const double dxt = dmx(g, txz, i, j) * idx, dzt = dpz(g, tzz, i, j) * idx;
      p3[c] = g->ax[j] * p3[c] + g->bx[j] * dxt;
      p4[c] = g->azh[i] * p4[c] + g->bzh[i] * dzt;
      sz[c] = dxt + p3[c] + dzt + p4[c];
    }
  for (size_t c = 0; c < N; ++c) {
    vx[c] += dt * g->bux[c] * sx[c];
    vz[c] += dt * g->buz[c] * sz[c];
  }
  for (int i = 0; i < NZ; ++i)
    for (int j = 0; j < NX; ++j) {
      const size_t c = (size_t)i * NX + j;
      const double exx = dmx(g, vx, i, j) * idx, ezz = dmz(g, vz, i, j) * idx;
      p5[c] = g->ax[j] * p5[c] + g->bx[j] * exx;
      p6[c] = g->az[i] * p6[c] + g->bz[i] * ezz;
      ex[c] = exx + p5[c];
      ez[c] = ezz + p6[c];
      const double ezx = dpz(g, vx, i, j) * idx, exz = dpx(g, vz, i, j) * idx;
      p7[c] = g->azh[i] * p7[c] + g->bzh[i] * ezx;
      p8[c] = g->axh[j] * p8[c] + g->bxh[j] * exz;
      sxz[c] = ezx + p7[c] + exz + p8[c];
    }
  for (size_t c = 0; c < N; ++c) {
    const double l2m = g->lam[c] + 2.0 * g->mu[c];
    txx[c] += dt * (l2m * ex[c] + g->lam[c] * ez[c]);
    tzz[c] += dt * (g->lam[c] * ex[c] + l2m * ez[c]);
    txz[c] += dt * g->muxz[c] * sxz[c];
  }
  txx[cs] += amp;
  tzz[cs] += amp;
}

/* add w * (staggered forward / backward difference) transposed: the sample
 * that the forward difference at (i, j) reads at offset k gets the weight */
static inline void sadd(const egrid* g, double* f, int i, int j, double w) {
  if (i >= 0 && i < g->NZ && j >= 0 && j < g->NX) f[(size_t)i * g->NX + j] += w;
}
/* transpose of y = dpx(f)(i, j) * idx: taps j+1, j (S1) and j+2, j-1 (S2) */
static void tdpx(const egrid* g, double* f, int i, int j, double y) {
  sadd(g, f, i, j + 1, ORC_S1 * y); sadd(g, f, i, j, -ORC_S1 * y);
  sadd(g, f, i, j + 2, ORC_S2 * y); sadd(g, f, i, j - 1, -ORC_S2 * y);
}
static void tdmx(const egrid* g, double* f, int i, int j, double y) {
  sadd(g, f, i, j, ORC_S1 * y); sadd(g, f, i, j - 1, -ORC_S1 * y);
  sadd(g, f, i, j + 1, ORC_S2 * y); sadd(g, f, i, j - 2, -ORC_S2 * y);
}
static void tdpz(const egrid* g, double* f, int i, int j, double y) {
  sadd(g, f, i + 1, j, ORC_S1 * y); sadd(g, f, i, j, -ORC_S1 * y);
  sadd(g, f, i + 2, j, ORC_S2 * y); sadd(g, f, i - 1, j, -ORC_S2 * y);
}
static void tdmz(const egrid* g, double* f, int i, int j, double y) {
  sadd(g, f, i, j, ORC_S1 * y); sadd(g, f, i - 1, j, -ORC_S1 * y);
  sadd(g, f, i + 1, j, ORC_S2 * y); sadd(g, f, i - 2, j, -ORC_S2 * y);
}

/* Transpose of the stress half of a step (in reverse order of the forward):
 * a holds the adjoints of (vx, vz, txx, tzz, txz, p1 .. p8) of the state
 * after the step; on return the stress and p5..p8 adjoints are those of the
 * state before the stress update, and the velocity adjoints have received
 * the strain terms.  gr (optional) accumulates d J / d (lam, mu, muxz). */
static void estep_adj_stress(const egrid* g, double dt, double idx, double* a,
                             const double* ex, const double* ez, const double* sxz,
                             double* glam, double* gmu, double* gmxz) {
  const int NZ = g->NZ, NX = g->NX;
  const size_t N = (size_t)NZ * NX;
  double *avx = a, *avz = a + N, *atxx = a + 2 * N, *atzz = a + 3 * N, *atxz = a + 4 * N;
  double *ap5 = a + 9 * N, *ap6 = a + 10 * N, *ap7 = a + 11 * N, *ap8 = a + 12 * N;
  for (int i = 0; i < NZ; ++i)
    for (int j = 0; j < NX; ++j) {
      const size_t c = (size_t)i * NX + j;
      /* txz += dt muxz (ezx + p7' + exz + p8') */
      const double T = dt * g->muxz[c] * atxz[c];
      if (gmxz) gmxz[c] += dt * atxz[c] * sxz[c];
      const double P7 = ap7[c] + T, P8 = ap8[c] + T;
      const double aezx = T + g->bzh[i] * P7, aexz = T + g->bxh[j] * P8;
      ap7[c] = g->azh[i] * P7;
      ap8[c] = g->axh[j] * P8;
      tdpz(g, avx, i, j, aezx * idx);
      tdpx(g, avz, i, j, aexz * idx);
      /* txx += dt (l2m ex + lam ez); tzz += dt (lam ex + l2m ez) */
      const double l2m = g->lam[c] + 2.0 * g->mu[c];
      const double Ex = dt * (l2m * atxx[c] + g->lam[c] * atzz[c]);
      const double Ez = dt * (g->lam[c] * atxx[c] + l2m * atzz[c]);
      if (glam) {
        glam[c] += dt * (atxx[c] + atzz[c]) * (ex[c] + ez[c]);
        gmu[c] += 2.0 * dt * (atxx[c] * ex[c] + atzz[c] * ez[c]);
      }
      const double P5 = ap5[c] + Ex, P6 = ap6[c] + Ez;
      const double aexx = Ex + g->bx[j] * P5, aezz = Ez + g->bz[i] * P6;
      ap5[c] = g->ax[j] * P5;
      ap6[c] = g->az[i] * P6;
      tdmx(g, avx, i, j, aexx * idx);
      tdmz(g, avz, i, j, aezz * idx);
    }
}

/* Transpose of the velocity half: the velocity adjoints (complete for this
 * step) feed the stress adjoints and p1..p4; gbx, gbz (optional) accumulate
 * d J / d (buoyancy at vx, vz points). */
static void estep_adj_velocity(const egrid* g, double dt, double idx, double* a,
                               const double* sx, const double* sz, double* gbx,
                               double* gbz) {
  const int NZ = g->NZ, NX = g->NX;
  const size_t N = (size_t)NZ * NX;
  double *avx = a, *avz = a + N, *atxx = a + 2 * N, *atzz = a + 3 * N, *atxz = a + 4 * N;
  double *ap1 = a + 5 * N, *ap2 = a + 6 * N, *ap3 = a + 7 * N, *ap4 = a + 8 * N;
  for (int i = 0; i < NZ; ++i)
    for (int j = 0; j < NX; ++j) {
      const size_t c = (size_t)i * NX + j;
      /* vx += dt bux (dxt + p1' + dzt + p2') */
      const double Q = dt * g->bux[c] * avx[c];
      if (gbx) gbx[c] += dt * avx[c] * sx[c];
      const double P1 = ap1[c] + Q, P2 = ap2[c] + Q;
      const double adxt = Q + g->bxh[j] * P1, adzt = Q + g->bz[i] * P2;
      ap1[c] = g->axh[j] * P1;
      ap2[c] = g->az[i] * P2;
      tdpx(g, atxx, i, j, adxt * idx);
      tdmz(g, atxz, i, j, adzt * idx);
      /* vz += dt buz (dxt + p3' + dzt + p4') */
      const double Qz = dt * g->buz[c] * avz[c];
      if (gbz) gbz[c] += dt * avz[c] * sz[c];
      const double P3 = ap3[c] + Qz, P4 = ap4[c] + Qz;
      const double adxt3 = Qz + g->bx[j] * P3, adzt4 = Qz + g->bzh[i] * P4;
      ap3[c] = g->ax[j] * P3;
      ap4[c] = g->azh[i] * P4;
      tdmx(g, atxz, i, j, adxt3 * idx);
      tdpz(g, atzz, i, j, adzt4 * idx);
    }
}

/* Reverse pass over all steps of one shot.  res [2][nrec][nt] is injected at
 * the receivers (transpose of the recording).  With H (the states before
 * each step, [nt][13][N]) the parameter adjoints are accumulated into g5
 * (glam, gmu, gbx, gbz, gmuxz, each [N]); wg (optional) receives the
 * wavelet adjoint.  Returns nothing: the arrays are the output. */
static void elastic_reverse_shot(const egrid* g, const oracle_problem* p, double idx,
                                 const double* H, const double* res, const int32_t* rec_s,
                                 size_t cs, double* wg, double* g5) {
  const int nt = p->nt, P = g->P, NX = g->NX;
  const size_t N = (size_t)g->NZ * g->NX;
  const double dt = p->dt;
  double* a = calloc(13 * N, sizeof(double));
  double* tmp = H ? malloc(13 * N * sizeof(double)) : NULL;
  double* q = H ? malloc(5 * N * sizeof(double)) : NULL;
  for (int n = nt - 1; n >= 0; --n) {
    double *sx = NULL, *sz = NULL, *ex = NULL, *ez = NULL, *sxz = NULL;
    if (H) {
      /* forward step n again from the stored state, for its intermediates */
      memcpy(tmp, H + (size_t)n * 13 * N, 13 * N * sizeof(double));
      sx = q; sz = q + N; ex = q + 2 * N; ez = q + 3 * N; sxz = q + 4 * N;
      estep(g, dt, idx, tmp, 0.0, 0, sx, sz, ex, ez, sxz);
    }
    /* source: txx(s), tzz(s) += dt f^n / dx^2 */
    if (wg) wg[n] = dt * idx * idx * (a[2 * N + cs] + a[3 * N + cs]);
    estep_adj_stress(g, dt, idx, a, ex, ez, sxz, H ? g5 : NULL, H ? g5 + N : NULL,
                     H ? g5 + 4 * N : NULL);
    /* recording: d[0][r][n] = vx(r), d[1][r][n] = vz(r) */
    for (int r = 0; r < p->nrec; ++r) {
      const size_t cr = (size_t)(rec_s[2 * r] + P) * NX + rec_s[2 * r + 1] + P;
      a[cr] += res[(size_t)r * nt + n];
      a[N + cr] += res[((size_t)p->nrec + r) * nt + n];
    }
    estep_adj_velocity(g, dt, idx, a, sx, sz, H ? g5 + 2 * N : NULL, H ? g5 + 3 * N : NULL);
  }
  free(a);
  free(tmp);
  free(q);
}

int oracle_elastic_adjoint(const oracle_problem* p, const double* model,
                           const double* adj_data, const int32_t* src,
                           const int32_t* rec, double* wavelet_grad) {
  int rc = orc_check(p, src, rec);
  if (rc) return rc;
  double* m = orc_pad_model(p, model, 3);
  egrid g;
  egrid_init(&g, p, m);
  const double idx = 1.0 / p->dx;
#pragma omp parallel for schedule(dynamic, 1)
  for (int s = 0; s < p->nshot; ++s) {
    const size_t cs = (size_t)(src[2 * s] + g.P) * g.NX + src[2 * s + 1] + g.P;
    elastic_reverse_shot(&g, p, idx, NULL, adj_data + (size_t)s * 2 * p->nrec * p->nt,
                         rec + (size_t)s * 2 * p->nrec, cs,
                         wavelet_grad + (size_t)s * p->nt, NULL);
  }
  egrid_free(&g);
  free(m);
  return 0;
}

int oracle_elastic_gradient(const oracle_problem* p, const double* model,
                            const double* wavelet, const int32_t* src,
                            const int32_t* rec, const double* d_obs, double* grad,
                            double* misfit) {
  int rc = orc_check(p, src, rec);
  if (rc) return rc;
  double* m = orc_pad_model(p, model, 3);
  egrid g;
  egrid_init(&g, p, m);
  const int NZ = g.NZ, NX = g.NX, P = g.P, nt = p->nt, R = p->nrec;
  const size_t N = (size_t)NZ * NX;
  const double dt = p->dt, idx = 1.0 / p->dx;
  double* gsum = calloc(5 * N, sizeof(double)); /* glam, gmu, gbx, gbz, gmuxz */
  double J = 0.0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : J)
  for (int s = 0; s < p->nshot; ++s) {
    const size_t cs = (size_t)(src[2 * s] + P) * NX + src[2 * s + 1] + P;
    const int32_t* rs = rec + (size_t)s * 2 * R;
    double* H = malloc((size_t)nt * 13 * N * sizeof(double));
    double* f = calloc(13 * N, sizeof(double));
    double* q = malloc(5 * N * sizeof(double));
    double* res = malloc((size_t)2 * R * nt * sizeof(double));
    for (int n = 0; n < nt; ++n) {
      memcpy(H + (size_t)n * 13 * N, f, 13 * N * sizeof(double));
      /* the trace sample n is v^{n+1/2}: record after the velocity half */
      estep(&g, dt, idx, f, dt * wavelet[(size_t)s * nt + n] * idx * idx, cs, q, q + N,
            q + 2 * N, q + 3 * N, q + 4 * N);
      for (int r = 0; r < R; ++r) {
        const size_t cr = (size_t)(rs[2 * r] + P) * NX + rs[2 * r + 1] + P;
        /* the velocities are not changed by the stress half */
        for (int k = 0; k < 2; ++k) {
          const size_t o = ((size_t)k * R + r) * nt + n;
          const double d = f[(size_t)k * N + cr];
          const double ob = d_obs[((size_t)s * 2 * R) * nt + o];
          res[o] = (p->flags & ORACLE_F_RESIDUAL_IN) ? ob : d - ob;
          J += 0.5 * res[o] * res[o];
        }
      }
    }
    double* g5 = calloc(5 * N, sizeof(double));
    elastic_reverse_shot(&g, p, idx, H, res, rs, cs, NULL, g5);
#pragma omp critical
    for (size_t c = 0; c < 5 * N; ++c) gsum[c] += g5[c];
    free(g5);
    free(H);
    free(f);
    free(q);
    free(res);
  }
  /* chain rule to (vp, vs, rho) on the padded grid; the padding is held
   * fixed, so only interior cells are reported */
  const double* vp = m;
  const double* vs = m + N;
  const double* rho = m + 2 * N;
  double* gvp = calloc(N, sizeof(double));
  double* gvs = calloc(N, sizeof(double));
  double* grho = calloc(N, sizeof(double));
  double* gmu = calloc(N, sizeof(double));
  const double *glam = gsum, *gmu0 = gsum + N, *gbx = gsum + 2 * N, *gbz = gsum + 3 * N,
               *gmxz = gsum + 4 * N;
  for (int i = 0; i < NZ; ++i)
    for (int j = 0; j < NX; ++j) {
      const size_t c = (size_t)i * NX + j;
      const int j1 = clampi(j + 1, NX - 1), i1 = clampi(i + 1, NZ - 1);
      const size_t cx = (size_t)i * NX + j1, cz = (size_t)i1 * NX + j, cxz = (size_t)i1 * NX + j1;
      gmu[c] += gmu0[c];
      /* bux = 2 / (rho_c + rho_cx), buz = 2 / (rho_c + rho_cz) */
      const double sx2 = rho[c] + rho[cx], sz2 = rho[c] + rho[cz];
      grho[c] += -2.0 / (sx2 * sx2) * gbx[c] - 2.0 / (sz2 * sz2) * gbz[c];
      grho[cx] += -2.0 / (sx2 * sx2) * gbx[c];
      grho[cz] += -2.0 / (sz2 * sz2) * gbz[c];
      /* muxz = 4 / sum(1 / mu_k): d muxz / d mu_k = muxz^2 / (4 mu_k^2) */
      const double mk[4] = {g.mu[c], g.mu[cx], g.mu[cz], g.mu[cxz]};
      const size_t ck[4] = {c, cx, cz, cxz};
      if (g.muxz[c] != 0.0)
        for (int k = 0; k < 4; ++k)
          gmu[ck[k]] += gmxz[c] * g.muxz[c] * g.muxz[c] / (4.0 * mk[k] * mk[k]);
    }
  for (size_t c = 0; c < N; ++c) {
    /* lam = rho (vp^2 - 2 vs^2), mu = rho vs^2 */
    gvp[c] = glam[c] * 2.0 * rho[c] * vp[c];
    gvs[c] = glam[c] * (-4.0 * rho[c] * vs[c]) + gmu[c] * 2.0 * rho[c] * vs[c];
    grho[c] += glam[c] * (vp[c] * vp[c] - 2.0 * vs[c] * vs[c]) + gmu[c] * vs[c] * vs[c];
  }
  for (int i = 0; i < p->nz; ++i)
    for (int j = 0; j < p->nx; ++j) {
      const size_t c = (size_t)(i + P) * NX + (j + P), o = (size_t)i * p->nx + j;
      const size_t M = (size_t)p->nz * p->nx;
      grad[o] = gvp[c];
      grad[M + o] = gvs[c];
      grad[2 * M + o] = grho[c];
    }
  if (misfit) *misfit = J;
  free(gvp); free(gvs); free(grho); free(gmu); free(gsum);
  egrid_free(&g);
  free(m);
  return 0;
}
