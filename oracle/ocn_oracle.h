/*
 * Plain FP64 CPU oracle for the nonhydrostatic Boussinesq RK3 substep on a
 * staggered C-grid (arXiv 2502.14148, Sec. 3.1, Appendix A.1-A.2, Appendix B).
 *
 * ORACLE / TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA library; the CUDA library never links
 * or calls it.
 *
 * Layout (x fastest): centre fields and u, v are [Nz][Ny][Nx]; w is
 * [Nz+1][Ny][Nx] with w[0] = w[Nz] = 0 (impenetrable walls).  Face index i is
 * left of cell index i (Appendix B.1).  x, y periodic and uniform; z bounded,
 * described by ascending face heights zf[0..Nz].
 *
 * Parity unpinned (fixed by decision, checked only oracle-vs-GPU): the WENO-Z
 * constants (epsilon = 1e-8, tau = |beta_0 - beta_{r-1}|), the AMD and
 * Smagorinsky-Lilly constants and averaging stencils, the Coriolis 4-point
 * average, the linear-EOS constants and the flux-BC sign convention.
 */
#ifndef OCN_ORACLE_H
#define OCN_ORACLE_H
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_CLOSURE_NONE = 0, ORC_CLOSURE_SCALAR = 1, ORC_CLOSURE_SMAG = 2, ORC_CLOSURE_AMD = 3 };
enum { ORC_EOS_BUOYANCY_TRACER = 0, ORC_EOS_LINEAR_TS = 1 };
enum { ORC_MAX_TRACERS = 4 };

typedef struct {
  int Nx, Ny, Nz;
  double Lx, Ly;
  const double* zf;          /* Nz+1 ascending face heights (copied) */
  int weno_order;            /* 1, 3, 5, 7 or 9 (odd); the advecting velocity uses centered order weno_order-1 (>=2) */
  int closure;               /* ORC_CLOSURE_* */
  double nu, kappa;          /* ScalarDiffusivity */
  double Cs, Cb, Pr;         /* Smagorinsky-Lilly */
  double C_amd;              /* AMD Poincare constant (buoyancy modification not modelled) */
  double f;                  /* FPlane Coriolis parameter */
  int n_tracers;
  int eos;                   /* ORC_EOS_* ; BUOYANCY_TRACER: tracer 0 is b.  LINEAR_TS: tracers 0,1 are T,S */
  double g, alpha, beta, T0, S0;
  double top_flux[2 + ORC_MAX_TRACERS];     /* u, v, tracers: upward flux through the top face */
  double bottom_flux[2 + ORC_MAX_TRACERS];  /* u, v, tracers: upward flux through the bottom face */
  int nthreads;              /* OpenMP threads (<=0: default) */
} orc_params;

typedef struct orc_model orc_model;

orc_model* orc_create(const orc_params* p);
void orc_destroy(orc_model* m);

/* field ids: 0=u 1=v 2=w 3..3+n_tracers-1 = tracers, 10=p, 20+f = G^{m-1} of field f */
enum { ORC_U = 0, ORC_V = 1, ORC_W = 2, ORC_C0 = 3, ORC_P = 10, ORC_G = 20 };
size_t orc_field_len(const orc_model* m, int field);
void orc_set(orc_model* m, int field, const double* src);
void orc_get(const orc_model* m, int field, double* dst);

/* Pressure projection of the current velocity (paper Eq. pressure-poisson and
 * Eq. pressure-correction with the stage step dt_stage): solves
 * lap p = div(u)/dt_stage and sets u -= dt_stage grad p. */
void orc_project(orc_model* m, double dt_stage);

/* nsteps full RK3 steps (Appendix A.1 Eq. rk3, three substages each). */
void orc_time_step(orc_model* m, double dt, int nsteps);

/* Tendencies G of every prognostic field at the current state (no stepping).
 * Output buffers have the field layouts above (Gw has Nz+1 levels, walls 0). */
void orc_tendencies(orc_model* m, double* Gu, double* Gv, double* Gw, double* Gc /* n_tracers fields */);
/* One tendency value, computed from scratch at one point. */
double orc_tendency_at(orc_model* m, int field, int i, int j, int k);
/* Eddy viscosity nu_e (closure >= SMAG) or tracer diffusivity (which = 1 + tracer) at one centre. */
double orc_diffusivity_at(orc_model* m, int which, int i, int j, int k);

/* Diagnostics: out[0..n_tracers-1] = sum V c_n; then sum V u, sum V v, sum V w,
 * max |div u|, max(|u|/dx,|v|/dy,|w|/dz_f)*dt, nonfinite count. */
void orc_diagnostics(const orc_model* m, double dt, double* out);
/* Conservative regridding of cell averages between two column grids covering the same interval:
 * out[j] = (1/dz_out_j) sum_i in[i] |cell_i of the input ∩ cell_j of the output| (finite-volume
 * averaging, Sec. B listing "finite-volumes"). */
void orc_regrid(const double* zf_in, int nin, const double* in, const double* zf_out, int nout, double* out);
/* Coarse-graining diagnostics (horizontal means over the periodic plane):
 *   out[0*Nz + k] = <b>, out[1*Nz + k] = <u>, out[2*Nz + k] = <v> at level k (b = tracer 0 or the EOS);
 *   out[3*Nz + f*(Nz+1) + k], f = 0,1,2: the horizontal mean of the model's upward face flux of b, u, v
 *   through face k = 0..Nz (advective + closure flux; the prescribed fluxes at the walls).
 * out holds 3*Nz + 3*(Nz+1) values. */
void orc_profiles(orc_model* m, double* out);

/* Discrete divergence at centres, [Nz][Ny][Nx]. */
void orc_divergence(const orc_model* m, double* out);

/* --- building blocks exposed for the analytic pins --- */
/* z metrics: centres zc[Nz], cell thickness dzc[Nz], centre spacing dzf[Nz+1] (dzf[k] = zc[k]-zc[k-1], 1<=k<Nz). */
void orc_grid_metrics(const orc_model* m, double* zc, double* dzc, double* dzf);
/* WENO(2r-1) reconstruction at the interface between s[r-1] and s[r] from the
 * 2r values s[0..2r-1] (cells m-r .. m+r-1), upwinded by the sign of vel. */
double orc_weno(const double* s, int r, double vel);
/* The pieces of orc_weno in the upwind frame: substencil values q[0..r-1] and
 * smoothness indicators beta[0..r-1] (substencil 0 the most upwind). */
void orc_weno_parts(const double* s, int r, double vel, double* q, double* beta);
/* Centered reconstruction of order 2p at the interface between s[p-1] and s[p]. */
double orc_centered(const double* s, int p);
/* Complex FFT in place, any length, sign -1 forward / +1 backward (unnormalised). */
void orc_fft(double* re, double* im, int n, int sign);
/* Solve the discrete Poisson problem lap p = rhs (Nz x Ny x Nx) with the
 * FFT + tridiagonal method, Neumann walls, zero-volume-mean gauge. */
void orc_poisson(orc_model* m, const double* rhs, double* p);

#ifdef __cplusplus
}
#endif
#endif
