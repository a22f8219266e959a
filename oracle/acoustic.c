/*
 * FP64 CPU oracle: constant-density acoustic engine (test infrastructure
 * only; see oracle.h for the readings of the paper it implements).
 *
 * Forward step (Eq. 2 with the update form of the Sec. 2.1 listing), on the
 * padded grid, per cell, with fields zero outside the grid:
 *   Wx      = D2x u^n + mx * D1x psi_x^{n-1}     (mx = 1 inside the x border)
 *   zeta_x^n = ax zeta_x^{n-1} + bx Wx
 *   psi_x^n  = ax psi_x^{n-1}  + bx D1x u^n
 *   (same for z)
 *   u^{n+1} = 2 u^n - u^{n-1} + K (Wx + zeta_x^n + Wz + zeta_z^n),
 *   K = v^2 dt^2 / dx^2,
 *   then u^{n+1}(s) += K(s) f^n and trace sample n = u^{n+1}(receiver).
 * This is the second-order convolutional PML: u_xx is replaced by
 * u_xx + d/dx psi_x + zeta_x, with the psi derivative taken one step behind so
 * that one pass per step suffices.
 *
 * Adjoint: the transpose of every statement above, applied in reverse order
 * (reverse-mode differentiation written out by hand, scatter form).  Velocity
 * gradient: dJ/dK(c) = sum_n lambda^{n+1}(c) (bracket^n(c) + f^n delta_{c,s}),
 * dK/dv = 2 v dt^2 / dx^2, interior cells only (padding frozen).  Long runs
 * use uniform checkpoints of the full state and recompute each segment.
 */
#include "oracle_internal.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Every field is stored with a 4-cell halo of zeros around the padded grid
 * (storage rows SX = NX + 8), so that stencil reads past the grid edge read 0
 * (the Dirichlet condition).  Scatter writes that land in the halo are
 * contributions to cells outside the grid and are never read back. */
#define H 4
typedef struct {
  int nz, nx, P, NZ, NX, SX;
  size_t NS;                       /* storage size (NZ+8)*(NX+8) */
  const double* K;                 /* storage layout, v^2 dt^2 / dx^2 */
  double *ax, *bx, *az, *bz;       /* CPML profiles */
  unsigned char *mx, *mz;          /* 1 inside the border along that axis */
} agrid;

typedef struct {
  double *u, *up, *psx, *psz, *zex, *zez; /* X^n = (u^n, u^{n-1}, psi^{n-1}, zeta^{n-1}) */
} astate;

static double* zalloc(size_t n) { return (double*)calloc(n, sizeof(double)); }

static void state_alloc(astate* s, size_t n) {
  s->u = zalloc(n); s->up = zalloc(n);
  s->psx = zalloc(n); s->psz = zalloc(n);
  s->zex = zalloc(n); s->zez = zalloc(n);
}
static void state_free(astate* s) {
  free(s->u); free(s->up); free(s->psx); free(s->psz); free(s->zex); free(s->zez);
}
static void state_copy(astate* d, const astate* s, size_t n) {
  memcpy(d->u, s->u, n * sizeof(double)); memcpy(d->up, s->up, n * sizeof(double));
  memcpy(d->psx, s->psx, n * sizeof(double)); memcpy(d->psz, s->psz, n * sizeof(double));
  memcpy(d->zex, s->zex, n * sizeof(double)); memcpy(d->zez, s->zez, n * sizeof(double));
}

static inline size_t ix(const agrid* g, int i, int j) {
  return (size_t)(i + H) * g->SX + (j + H);
}
static inline double at(const agrid* g, const double* f, int i, int j) {
  return f[ix(g, i, j)];
}

/* One forward step X^n -> X^{n+1} without the source.  `out` receives
 * (u^{n+1}, u^n, psi^n, zeta^n).  bracket (optional) receives
 * Wx + zeta_x^n + Wz + zeta_z^n per cell. */
static void step_forward(const agrid* g, const astate* in, astate* out,
                         double* bracket) {
  const int NZ = g->NZ, NX = g->NX;
  for (int i = 0; i < NZ; ++i)
    for (int j = 0; j < NX; ++j) {
      const size_t c = ix(g, i, j);
      double d2x = ORC_C2[0] * in->u[c], d2z = ORC_C2[0] * in->u[c];
      double d1xu = 0, d1zu = 0, d1xp = 0, d1zp = 0;
      for (int k = 1; k <= 4; ++k) {
        d2x += ORC_C2[k] * (at(g, in->u, i, j + k) + at(g, in->u, i, j - k));
        d2z += ORC_C2[k] * (at(g, in->u, i + k, j) + at(g, in->u, i - k, j));
        d1xu += ORC_C1[k] * (at(g, in->u, i, j + k) - at(g, in->u, i, j - k));
        d1zu += ORC_C1[k] * (at(g, in->u, i + k, j) - at(g, in->u, i - k, j));
        d1xp += ORC_C1[k] * (at(g, in->psx, i, j + k) - at(g, in->psx, i, j - k));
        d1zp += ORC_C1[k] * (at(g, in->psz, i + k, j) - at(g, in->psz, i - k, j));
      }
      const double Wx = d2x + (g->mx[j] ? d1xp : 0.0);
      const double Wz = d2z + (g->mz[i] ? d1zp : 0.0);
      const double zx = g->ax[j] * in->zex[c] + g->bx[j] * Wx;
      const double zz = g->az[i] * in->zez[c] + g->bz[i] * Wz;
      out->psx[c] = g->ax[j] * in->psx[c] + g->bx[j] * d1xu;
      out->psz[c] = g->az[i] * in->psz[c] + g->bz[i] * d1zu;
      out->zex[c] = zx;
      out->zez[c] = zz;
      const double br = Wx + zx + Wz + zz;
      out->u[c] = 2.0 * in->u[c] - in->up[c] + g->K[c] * br;
      if (bracket) bracket[c] = br;
    }
  memcpy(out->up, in->u, g->NS * sizeof(double));
}

static inline void acc(const agrid* g, double* f, int i, int j, double v) {
  f[ix(g, i, j)] += v;
}

/* Transpose of step_forward: given the adjoint of X^{n+1} (`ain`, whose u
 * already contains the receiver injection), produce the adjoint of X^n. */
static void step_adjoint(const agrid* g, const astate* ain, astate* aout) {
  const int NZ = g->NZ, NX = g->NX;
  const size_t N = g->NS;
  memset(aout->u, 0, N * sizeof(double));
  memset(aout->up, 0, N * sizeof(double));
  memset(aout->psx, 0, N * sizeof(double));
  memset(aout->psz, 0, N * sizeof(double));
  memset(aout->zex, 0, N * sizeof(double));
  memset(aout->zez, 0, N * sizeof(double));
  for (int i = 0; i < NZ; ++i)
    for (int j = 0; j < NX; ++j) {
      const size_t c = ix(g, i, j);
      const double lun = ain->u[c];          /* adjoint of u^{n+1}      */
      /* out->up = in->u (u^n passed on as next step's u^{n-1}) */
      aout->u[c] += ain->up[c];
      /* u^{n+1} = 2 u^n - u^{n-1} + K * bracket */
      aout->u[c] += 2.0 * lun;
      aout->up[c] += -lun;
      const double q = g->K[c] * lun;       /* adjoint of bracket      */
      /* bracket = Wx + zeta_x^n + ...; zeta_x^n = ax zeta_x + bx Wx */
      const double tzx = ain->zex[c] + q, tzz = ain->zez[c] + q;
      const double wx = q + g->bx[j] * tzx, wz = q + g->bz[i] * tzz;
      aout->zex[c] += g->ax[j] * tzx;
      aout->zez[c] += g->az[i] * tzz;
      /* psi^n = a psi^{n-1} + b D1 u^n */
      aout->psx[c] += g->ax[j] * ain->psx[c];
      aout->psz[c] += g->az[i] * ain->psz[c];
      const double gx = g->bx[j] * ain->psx[c], gz = g->bz[i] * ain->psz[c];
      /* Wx = D2x u + mx D1x psi_x */
      acc(g, aout->u, i, j, ORC_C2[0] * (wx + wz));
      for (int k = 1; k <= 4; ++k) {
        acc(g, aout->u, i, j + k, ORC_C2[k] * wx);
        acc(g, aout->u, i, j - k, ORC_C2[k] * wx);
        acc(g, aout->u, i + k, j, ORC_C2[k] * wz);
        acc(g, aout->u, i - k, j, ORC_C2[k] * wz);
        acc(g, aout->u, i, j + k, ORC_C1[k] * gx);
        acc(g, aout->u, i, j - k, -ORC_C1[k] * gx);
        acc(g, aout->u, i + k, j, ORC_C1[k] * gz);
        acc(g, aout->u, i - k, j, -ORC_C1[k] * gz);
        if (g->mx[j]) {
          acc(g, aout->psx, i, j + k, ORC_C1[k] * wx);
          acc(g, aout->psx, i, j - k, -ORC_C1[k] * wx);
        }
        if (g->mz[i]) {
          acc(g, aout->psz, i + k, j, ORC_C1[k] * wz);
          acc(g, aout->psz, i - k, j, -ORC_C1[k] * wz);
        }
      }
    }
}

/* Build the padded grid: K, profiles, masks.  vp is the padded velocity
 * [NZ][NX]; K is stored in the halo layout. */
static void grid_init(agrid* g, const oracle_problem* p, const double* vp) {
  g->nz = p->nz; g->nx = p->nx; g->P = p->pml;
  g->NZ = p->nz + 2 * p->pml; g->NX = p->nx + 2 * p->pml;
  g->SX = g->NX + 2 * H;
  g->NS = (size_t)(g->NZ + 2 * H) * g->SX;
  double* K = zalloc(g->NS);
  double vmax = 0.0;
  for (int i = 0; i < g->NZ; ++i)
    for (int j = 0; j < g->NX; ++j) {
      const double v = vp[(size_t)i * g->NX + j];
      K[ix(g, i, j)] = v * v * p->dt * p->dt / (p->dx * p->dx);
      if (v > vmax) vmax = v;
    }
  g->K = K;
  if (p->v_pml > 0.0) vmax = p->v_pml;
  g->ax = zalloc(g->NX); g->bx = zalloc(g->NX);
  g->az = zalloc(g->NZ); g->bz = zalloc(g->NZ);
  oracle_cpml_profile(p->nx, p->pml, p->dx, p->dt, vmax, p->f_ref, 0, g->ax, g->bx);
  oracle_cpml_profile(p->nz, p->pml, p->dx, p->dt, vmax, p->f_ref, 0, g->az, g->bz);
  g->mx = (unsigned char*)calloc(g->NX, 1);
  g->mz = (unsigned char*)calloc(g->NZ, 1);
  for (int j = 0; j < g->NX; ++j) g->mx[j] = (j < p->pml || j >= p->pml + p->nx);
  for (int i = 0; i < g->NZ; ++i) g->mz[i] = (i < p->pml || i >= p->pml + p->nz);
}

static void grid_free(agrid* g) {
  free((void*)g->K); free(g->ax); free(g->bx); free(g->az); free(g->bz);
  free(g->mx); free(g->mz);
}

/* storage index of an interior position (z, x) */
static size_t cell_of(const agrid* g, const int32_t* zx) {
  return ix(g, zx[0] + g->P, zx[1] + g->P);
}

/* copy the padded grid [NZ][NX] out of a halo-layout field */
static void unhalo(const agrid* g, const double* f, double* out) {
  for (int i = 0; i < g->NZ; ++i)
    memcpy(out + (size_t)i * g->NX, f + ix(g, i, 0), g->NX * sizeof(double));
}

static agrid setup(const oracle_problem* p, const double* model) {
  double* vp = orc_pad_model(p, model, 1);
  agrid g;
  grid_init(&g, p, vp);
  free(vp);
  return g;
}

int oracle_acoustic_forward(const oracle_problem* p, const double* model,
                            const double* wavelet, const int32_t* src,
                            const int32_t* rec, double* data, double* wavefield) {
  int rc = orc_check(p, src, rec);
  if (rc) return rc;
  agrid g = setup(p, model);
  const size_t NP = (size_t)g.NZ * g.NX;
#pragma omp parallel for schedule(dynamic, 1)
  for (int s = 0; s < p->nshot; ++s) {
    astate a, b;
    state_alloc(&a, g.NS);
    state_alloc(&b, g.NS);
    astate *cur = &a, *nxt = &b;
    const size_t cs = cell_of(&g, src + 2 * s);
    if (wavefield) memset(wavefield + (size_t)s * (p->nt + 1) * NP, 0, NP * sizeof(double));
    for (int n = 0; n < p->nt; ++n) {
      step_forward(&g, cur, nxt, NULL);
      nxt->u[cs] += g.K[cs] * wavelet[(size_t)s * p->nt + n];
      for (int r = 0; r < p->nrec; ++r) {
        const size_t cr = cell_of(&g, rec + 2 * ((size_t)s * p->nrec + r));
        data[((size_t)s * p->nrec + r) * p->nt + n] = nxt->u[cr];
      }
      if (wavefield) unhalo(&g, nxt->u, wavefield + ((size_t)s * (p->nt + 1) + n + 1) * NP);
      astate* t = cur; cur = nxt; nxt = t;
    }
    state_free(&a);
    state_free(&b);
  }
  grid_free(&g);
  return 0;
}

int oracle_acoustic_adjoint(const oracle_problem* p, const double* model,
                            const double* adj_data, const int32_t* src,
                            const int32_t* rec, double* wavelet_grad) {
  int rc = orc_check(p, src, rec);
  if (rc) return rc;
  agrid g = setup(p, model);
#pragma omp parallel for schedule(dynamic, 1)
  for (int s = 0; s < p->nshot; ++s) {
    astate a, b;
    state_alloc(&a, g.NS);  /* zero: adjoint of the final state */
    state_alloc(&b, g.NS);
    astate *cur = &a, *nxt = &b;
    const size_t cs = cell_of(&g, src + 2 * s);
    for (int n = p->nt - 1; n >= 0; --n) {
      /* cur = adjoint of X^{n+1}; sample n of each trace is u^{n+1} */
      for (int r = 0; r < p->nrec; ++r) {
        const size_t cr = cell_of(&g, rec + 2 * ((size_t)s * p->nrec + r));
        cur->u[cr] += adj_data[((size_t)s * p->nrec + r) * p->nt + n];
      }
      /* u^{n+1}(s) += K(s) f^n */
      wavelet_grad[(size_t)s * p->nt + n] = g.K[cs] * cur->u[cs];
      step_adjoint(&g, cur, nxt);
      astate* t = cur; cur = nxt; nxt = t;
    }
    state_free(&a);
    state_free(&b);
  }
  grid_free(&g);
  return 0;
}

int oracle_acoustic_gradient(const oracle_problem* p, const double* model,
                             const double* wavelet, const int32_t* src,
                             const int32_t* rec, const double* d_obs,
                             double* grad, double* misfit) {
  int rc = orc_check(p, src, rec);
  if (rc) return rc;
  agrid g = setup(p, model);
  const size_t NS = g.NS;
  const int nt = p->nt, nz = p->nz, nx = p->nx, P = p->pml;
  const size_t nint = (size_t)nz * nx;
  int seg = (int)ceil(sqrt((double)nt));
  if (seg < 1) seg = 1;
  const int nseg = (nt + seg - 1) / seg;
  double* gK = zalloc((size_t)(p->nshot > 0 ? p->nshot : 1) * nint); /* per-shot dJ/dK */
  double* Jshot = zalloc(p->nshot > 0 ? p->nshot : 1);

#pragma omp parallel for schedule(dynamic, 1)
  for (int s = 0; s < p->nshot; ++s) {
    const size_t cs = cell_of(&g, src + 2 * s);
    const double* f = wavelet + (size_t)s * nt;
    double* res = zalloc((size_t)p->nrec * nt);
    /* checkpoints of the full state at n = k * seg */
    astate* ck = (astate*)malloc(sizeof(astate) * nseg);
    astate a, b;
    state_alloc(&a, NS);
    state_alloc(&b, NS);
    astate *cur = &a, *nxt = &b;
    for (int n = 0; n < nt; ++n) {
      if (n % seg == 0) {
        state_alloc(&ck[n / seg], NS);
        state_copy(&ck[n / seg], cur, NS);
      }
      step_forward(&g, cur, nxt, NULL);
      nxt->u[cs] += g.K[cs] * f[n];
      for (int r = 0; r < p->nrec; ++r) {
        const size_t cr = cell_of(&g, rec + 2 * ((size_t)s * p->nrec + r));
        res[(size_t)r * nt + n] = nxt->u[cr];
      }
      astate* t = cur; cur = nxt; nxt = t;
    }
    /* residual r = d - d_obs (or the given residual), J = 1/2 sum r^2 */
    double J = 0.0;
    for (int r = 0; r < p->nrec; ++r)
      for (int n = 0; n < nt; ++n) {
        const size_t o = ((size_t)s * p->nrec + r) * nt + n;
        const double rv = (p->flags & ORACLE_F_RESIDUAL_IN)
                              ? d_obs[o]
                              : res[(size_t)r * nt + n] - d_obs[o];
        res[(size_t)r * nt + n] = rv;
        J += 0.5 * rv * rv;
      }
    Jshot[s] = J;
    /* backward over segments, recomputing each from its checkpoint */
    double* br = (double*)malloc(sizeof(double) * (size_t)seg * nint);
    double* full = zalloc(NS);
    astate adj, adj2, rs, rs2;
    state_alloc(&adj, NS);
    state_alloc(&adj2, NS);
    state_alloc(&rs, NS);
    state_alloc(&rs2, NS);
    astate *ac = &adj, *an = &adj2;
    double* gks = gK + (size_t)s * nint;
    for (int k = nseg - 1; k >= 0; --k) {
      const int n0 = k * seg;
      const int n1 = (n0 + seg < nt) ? n0 + seg : nt;
      state_copy(&rs, &ck[k], NS);
      astate *rc0 = &rs, *rc1 = &rs2;
      for (int n = n0; n < n1; ++n) {
        step_forward(&g, rc0, rc1, full);
        /* the source term enters u^{n+1} multiplied by K as well */
        full[cs] += f[n];
        for (int i = 0; i < nz; ++i)
          memcpy(br + (size_t)(n - n0) * nint + (size_t)i * nx,
                 full + ix(&g, i + P, P), nx * sizeof(double));
        rc1->u[cs] += g.K[cs] * f[n];
        astate* t = rc0; rc0 = rc1; rc1 = t;
      }
      for (int n = n1 - 1; n >= n0; --n) {
        for (int r = 0; r < p->nrec; ++r) {
          const size_t cr = cell_of(&g, rec + 2 * ((size_t)s * p->nrec + r));
          ac->u[cr] += res[(size_t)r * nt + n];
        }
        /* dJ/dK(c) += lambda^{n+1}(c) * (bracket^n(c) + f^n delta_{c,s}) */
        const double* bn = br + (size_t)(n - n0) * nint;
        for (int i = 0; i < nz; ++i)
          for (int j = 0; j < nx; ++j)
            gks[(size_t)i * nx + j] += ac->u[ix(&g, i + P, j + P)] * bn[(size_t)i * nx + j];
        step_adjoint(&g, ac, an);
        astate* t = ac; ac = an; an = t;
      }
      state_free(&ck[k]);
    }
    free(ck);
    free(br);
    free(full);
    free(res);
    state_free(&a); state_free(&b);
    state_free(&adj); state_free(&adj2);
    state_free(&rs); state_free(&rs2);
  }
  double J = 0.0;
  for (int s = 0; s < p->nshot; ++s) J += Jshot[s];
  if (misfit) *misfit = J;
  /* dK/dv = 2 v dt^2 / dx^2 = 2 K / v */
  double* vp = orc_pad_model(p, model, 1);
  for (int i = 0; i < nz; ++i)
    for (int j = 0; j < nx; ++j) {
      double sum = 0.0;
      for (int s = 0; s < p->nshot; ++s) sum += gK[(size_t)s * nint + (size_t)i * nx + j];
      const double v = vp[(size_t)(i + P) * g.NX + j + P];
      grad[(size_t)i * nx + j] = sum * 2.0 * v * p->dt * p->dt / (p->dx * p->dx);
    }
  free(vp);
  free(gK);
  free(Jshot);
  grid_free(&g);
  return 0;
}
