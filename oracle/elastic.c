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
