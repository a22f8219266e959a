/*
 * FP64 CPU oracle: pieces common to both engines (test infrastructure only;
 * see oracle.h).  Plain loops, no blocking, no fusion.
 */
#include "oracle_internal.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Taylor coefficients of the centred 8th-order second derivative,
 * f''(0) ~ sum_{k=-4..4} C2[|k|] f(k).  Pinned by exactness on x^k, k <= 9. */
const double ORC_C2[5] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0,
                          -1.0 / 560.0};
/* centred 8th-order first derivative, f'(0) ~ sum_k C1[k] (f(k) - f(-k)). */
const double ORC_C1[5] = {0.0, 4.0 / 5.0, -1.0 / 5.0, 4.0 / 105.0,
                          -1.0 / 280.0};
/* staggered 4th-order first derivative over half-cell offsets:
 * f'(0) ~ [S1 (f(1/2) - f(-1/2)) + S2 (f(3/2) - f(-3/2))] / h.              */
const double ORC_S1 = 9.0 / 8.0;
const double ORC_S2 = -1.0 / 24.0;

static double at1(const double* f, int n, int j) {
  return (j >= 0 && j < n) ? f[j] : 0.0;
}

void oracle_stencil_1d(int kind, int n, const double* f, double* out) {
  for (int j = 0; j < n; ++j) {
    double s = 0.0;
    if (kind == 0) {
      s = ORC_C2[0] * f[j];
      for (int k = 1; k <= 4; ++k)
        s += ORC_C2[k] * (at1(f, n, j + k) + at1(f, n, j - k));
    } else if (kind == 1) {
      for (int k = 1; k <= 4; ++k)
        s += ORC_C1[k] * (at1(f, n, j + k) - at1(f, n, j - k));
    } else if (kind == 2) {
      /* derivative at j + 1/2 from integer samples */
      s = ORC_S1 * (at1(f, n, j + 1) - at1(f, n, j)) +
          ORC_S2 * (at1(f, n, j + 2) - at1(f, n, j - 1));
    } else {
      /* derivative at j - 1/2 from integer samples */
      s = ORC_S1 * (at1(f, n, j) - at1(f, n, j - 1)) +
          ORC_S2 * (at1(f, n, j + 1) - at1(f, n, j - 2));
    }
    out[j] = s;
  }
}

void oracle_cpml_profile(int n_int, int pml, double dx, double dt, double vmax,
                         double f_ref, int half, double* a, double* b) {
  const int n = n_int + 2 * pml;
  const double R = 1e-3; /* target reflection coefficient */
  const double sigma_max =
      pml > 0 ? 3.0 * vmax * log(1.0 / R) / (2.0 * pml * dx) : 0.0;
  for (int j = 0; j < n; ++j) {
    const double x = half ? j + 0.5 : (double)j;
    double d = 0.0; /* depth into the border, cells */
    if (x < pml)
      d = pml - x;
    else if (x > pml + n_int - 1)
      d = x - (pml + n_int - 1);
    if (d <= 0.0 || pml == 0) {
      a[j] = 0.0;
      b[j] = 0.0;
      continue;
    }
    double rho = d / pml;
    if (rho > 1.0) rho = 1.0;
    const double sigma = sigma_max * rho * rho;
    const double alpha = M_PI * f_ref * (1.0 - rho);
    a[j] = exp(-(sigma + alpha) * dt);
    b[j] = sigma / (sigma + alpha) * (a[j] - 1.0);
  }
}

double* orc_pad_model(const oracle_problem* p, const double* model, int npar) {
  const int NZ = p->nz + 2 * p->pml, NX = p->nx + 2 * p->pml;
  double* out = (double*)malloc(sizeof(double) * (size_t)npar * NZ * NX);
  for (int c = 0; c < npar; ++c) {
    double* o = out + (size_t)c * NZ * NX;
    if (p->flags & ORACLE_F_PADDED_MODEL) {
      memcpy(o, model + (size_t)c * NZ * NX, sizeof(double) * (size_t)NZ * NX);
      continue;
    }
    const double* m = model + (size_t)c * p->nz * p->nx;
    for (int i = 0; i < NZ; ++i) {
      int ii = i - p->pml;
      if (ii < 0) ii = 0;
      if (ii > p->nz - 1) ii = p->nz - 1;
      for (int j = 0; j < NX; ++j) {
        int jj = j - p->pml;
        if (jj < 0) jj = 0;
        if (jj > p->nx - 1) jj = p->nx - 1;
        o[(size_t)i * NX + j] = m[(size_t)ii * p->nx + jj];
      }
    }
  }
  return out;
}

int orc_check(const oracle_problem* p, const int32_t* src, const int32_t* rec) {
  if (!p || p->nz < 1 || p->nx < 1 || p->pml < 0 || p->nt < 1 ||
      p->nshot < 0 || p->nrec < 0 || !(p->dx > 0.0) || !(p->dt > 0.0))
    return ORC_EINVAL;
  for (int s = 0; s < p->nshot; ++s) {
    if (src[2 * s] < 0 || src[2 * s] >= p->nz || src[2 * s + 1] < 0 ||
        src[2 * s + 1] >= p->nx)
      return ORC_EBOUNDS;
    for (int r = 0; r < p->nrec; ++r) {
      const int32_t* q = rec + 2 * ((size_t)s * p->nrec + r);
      if (q[0] < 0 || q[0] >= p->nz || q[1] < 0 || q[1] >= p->nx)
        return ORC_EBOUNDS;
    }
  }
  return 0;
}
