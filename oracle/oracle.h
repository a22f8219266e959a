/*
 * FP64 CPU oracle for the 2D finite-difference wave solvers of SWEEP
 * (Wang & Alkhalifah, "SWEEP: A Unified Solver Framework for Differentiable
 * Wave Physics").
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, plain, obviously
 * correct statement of what the GPU library computes.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or constant with the CUDA path.
 *
 * Everything is double precision, host memory, row-major with x fastest.
 *
 * Acoustic engine: constant-density 2nd-order wave equation (Sec. 3.1.2,
 * Eq. 2) stepped as in the listing of Sec. 2.1:
 *     u^{n+1} = 2 u^n - u^{n-1} + v^2 dt^2 Lap(u^n),
 * with an 8th-order Laplacian, a convolutional PML written for the
 * second-order form (memory variables psi, zeta per axis), point-source
 * injection and receiver recording (Sec. 2.1, Source / Receiver modules).
 * Elastic engine: velocity-stress system of Sec. 3.5 (Eq. 12) on a staggered
 * grid with 4th-order differences and a convolutional PML.
 *
 * The paper fixes none of: FD order, absorbing boundary, source scaling,
 * wavelet delay, record timing.  The readings implemented here:
 *   - padding: the interior model is edge-replicated into a border of `pml`
 *     cells on every side; the padding is frozen (the gradient is taken with
 *     respect to interior cells, padded values held fixed);
 *   - outside the padded grid every field is zero (Dirichlet);
 *   - CPML profile per axis: depth d (cells, measured at cell centres) into
 *     the border, rho = d/pml, sigma = sigma_max rho^2,
 *     sigma_max = 3 vmax ln(1/1e-3) / (2 pml dx), alpha = pi f_ref (1-rho),
 *     vmax = v_pml if given, else the largest vp of the padded model; the
 *     profile is held fixed when differentiating (like the padding);
 *     a = exp(-(sigma+alpha) dt), b = sigma/(sigma+alpha) (a-1); a=b=0 where
 *     d = 0;
 *   - source: u^{n+1}(s) += v(s)^2 dt^2 / dx^2 * f^n (unit-area point source);
 *   - recording: trace sample n is u^{n+1} (time (n+1) dt).
 */
#ifndef SWEEP_ORACLE_H
#define SWEEP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORACLE_ACOUSTIC = 0, ORACLE_ELASTIC = 1 };
/* model is given on the padded grid [npar][nz+2pml][nx+2pml] */
#define ORACLE_F_PADDED_MODEL 0x1
/* in oracle_*_gradient, d_obs holds the data residual itself */
#define ORACLE_F_RESIDUAL_IN 0x2

typedef struct {
  int32_t physics;
  int32_t nz, nx;     /* interior grid */
  int32_t pml;        /* border width per side */
  double dx, dt;      /* dz == dx */
  int32_t nt;         /* time steps == samples per trace */
  int32_t nshot, nrec;
  double f_ref;       /* CPML alpha reference frequency (Hz) */
  double v_pml;       /* CPML reference velocity (m/s); <= 0: max of vp */
  int32_t flags;
} oracle_problem;

/* 1D operators on a zero-padded line of n samples, unit spacing.
 * kind 0: 8th-order centred second derivative
 * kind 1: 8th-order centred first derivative
 * kind 2: 4th-order staggered forward difference, out[j] ~ f'(j+1/2)
 * kind 3: 4th-order staggered backward difference, out[j] ~ f'(j-1/2)   */
void oracle_stencil_1d(int kind, int n, const double* f, double* out);

/* CPML coefficients along one axis of n_int interior cells plus pml on each
 * side; a, b have n_int + 2 pml entries.  half != 0 evaluates the profile at
 * the half-cell points j + 1/2 (staggered grids).                           */
void oracle_cpml_profile(int n_int, int pml, double dx, double dt, double vmax,
                         double f_ref, int half, double* a, double* b);

/* Acoustic forward.  model: vp [nz][nx] (or padded).  wavelet [nshot][nt].
 * src [nshot][2] (z,x) interior indices.  rec [nshot][nrec][2].
 * data out [nshot][nrec][nt].  wavefield (optional, NULL to skip):
 * [nshot][nt+1][NZ][NX], u^0 ... u^nt.  Returns 0 or a negative code.      */
int oracle_acoustic_forward(const oracle_problem* p, const double* model,
                            const double* wavelet, const int32_t* src,
                            const int32_t* rec, double* data, double* wavefield);

/* Adjoint of the forward map wavelet -> data (model fixed):
 * wavelet_grad[s][n] = sum_{r,m} adj_data[s][r][m] * d data[s][r][m] / d wavelet[s][n]. */
int oracle_acoustic_adjoint(const oracle_problem* p, const double* model,
                            const double* adj_data, const int32_t* src,
                            const int32_t* rec, double* wavelet_grad);

/* L2 misfit J = 1/2 sum (d - d_obs)^2 and its gradient with respect to the
 * interior velocity, grad [nz][nx] (sum over shots).  With
 * ORACLE_F_RESIDUAL_IN, d_obs is the residual r and the gradient is
 * (dd/dv)^T r, misfit = 1/2 sum r^2.                                        */
int oracle_acoustic_gradient(const oracle_problem* p, const double* model,
                             const double* wavelet, const int32_t* src,
                             const int32_t* rec, const double* d_obs,
                             double* grad, double* misfit);

/* Elastic forward.  model [3][nz][nx] = (vp, vs, rho) (or padded).
 * data out [nshot][2][nrec][nt] = (vx, vz) at n+1/2.  wavefield optional:
 * [nshot][nt+1][5][NZ][NX] (vx, vz, txx, tzz, txz) after each step.       */
int oracle_elastic_forward(const oracle_problem* p, const double* model,
                           const double* wavelet, const int32_t* src,
                           const int32_t* rec, double* data, double* wavefield);

/* Elastic adjoint of the map wavelet -> data (model fixed): adj_data
 * [nshot][2][nrec][nt] in the layout of the data, wavelet_grad [nshot][nt].
 * The exact transpose of the recurrence, run backwards in time.            */
int oracle_elastic_adjoint(const oracle_problem* p, const double* model,
                           const double* adj_data, const int32_t* src,
                           const int32_t* rec, double* wavelet_grad);

/* Elastic L2 misfit J = 1/2 sum (d - d_obs)^2 over both components and its
 * gradient with respect to the interior (vp, vs, rho), grad [3][nz][nx]
 * (sum over shots); padding and CPML profiles held fixed (set v_pml).
 * Keeps every forward state in memory: small problems only.                */
int oracle_elastic_gradient(const oracle_problem* p, const double* model,
                            const double* wavelet, const int32_t* src,
                            const int32_t* rec, const double* d_obs, double* grad,
                            double* misfit);

#ifdef __cplusplus
}
#endif
#endif
