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
 * constants (epsilon = 1e-8, tau = |beta_0 - beta_{r-1}|), the values of the
 * AMD and Smagorinsky-Lilly constants, which edges are averaged onto a centre
 * (linear fields cannot tell averaging stencils apart), the Coriolis 4-point
 * average, the linear-EOS constants and the flux-BC sign convention.  The two
 * closure formulas themselves (Smagorinsky-Lilly with its stratification
 * factor, AMD viscosity and tracer diffusivity) are pinned by closed forms on
 * linear velocity and tracer fields.
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
  /* time stepper: ORC_RK3 (Eq. rk3) or ORC_QAB2 (Eq. qab2 with chi; the first step after orc_set of a
   * state field is forward Euler, chi = -1/2; orc_set of a G field marks the run as continuing) */
  int timestepper;
  double chi;
  /* vertical diffusivity profiles at the w-faces (Nz+1 values each, copied; NULL = none): nu_z for
   * u, v, w and kappa_z for every tracer (Eqs. tracer-with-tendency, momentum-tendency-definition);
   * vertical_implicit = 1 treats them with the semi-implicit step of Eq. tracer-time-discretization /
   * predictor-velocity, 0 adds them to the explicit tendency */
  const double* nu_z;
  const double* kappa_z;
  int vertical_implicit;
} orc_params;
enum { ORC_RK3 = 0, ORC_QAB2 = 1 };

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

/* --- learned column closure (an extension: the paper motivates closures calibrated on LES,
 * Sec. 3.2.3, but prints no network).  Column quantities: b, ubar = (u_i + u_{i+1})/2 and
 * vbar = (v_j + v_{j+1})/2 at cell centres; fluxes are upward through the w-faces of the
 * cell-centre columns, zero at the walls, arrays [3][Nz+1][Ny][Nx] (b, ubar, vbar). --- */
enum { ORC_NF = 32, ORC_NF_USED = 20 };
/* Raw features of every w-face (sample (k, j, i), i fastest; ORC_NF values each, zero padded):
 *   0-4   db/dz at faces k-2..k+2, 5-9 dubar/dz, 10-14 dvbar/dz (0 for faces outside 1..Nz-1)
 *   15    surface buoyancy flux (top_flux of tracer 0), 16 f, 17 N2_background,
 *   18    depth of the face below the top, zf[Nz] - zf[k],
 *   19    column mixed-layer depth estimate h = sum_{q=1}^{Nz-1} max(0, 1 - (db/dz)_q / N2_background) dzf[q]
 *         (0 when N2_background <= 0). */
void orc_closure_features(orc_model* m, double N2_background, double* X);
/* The closure's own vertical flux of b, ubar, vbar through the interior faces:
 * -kappa_f dq/dz for b, -nu_f dq/dz for ubar and vbar, face diffusivities the mean of the two
 * adjacent centres (ScalarDiffusivity: kappa, nu; LINEAR_TS: g (alpha F_T - beta F_S)). */
void orc_column_sgs_flux(orc_model* m, double* F);
/* Box filter of the state onto a cx x cy coarse horizontal grid (Nx % cx == 0, Ny % cy == 0; the
 * vertical grid is kept).  out = [u_c Nz*cy*cx][v_c Nz*cy*cx][w_c (Nz+1)*cy*cx][b_c Nz*cy*cx]
 * [tau 3*(Nz+1)*cy*cx]: u_c the mean of u over the fine faces on coarse x-face I (rx = Nx/cx fine
 * columns), v_c likewise, w_c and b_c box means, and the subfilter vertical flux of q in {b, ubar,
 * vbar} at the interior faces, tau_q = <w q_f> - <w><q_f> + <F_sgs,q> with q_f = (q_{k-1} + q_k)/2
 * and F_sgs as in orc_column_sgs_flux (0 at the walls). */
void orc_coarse_grain(orc_model* m, int cx, int cy, double* out);
/* Hook: when set, every tendency evaluation of the time stepper (and orc_tendencies) calls
 * fn(ctx, m, F) with the stage state in m, takes F [3][Nz+1][Ny][Nx] (wall faces forced to 0) and
 * adds -dF_b/dz to the tendency of tracer 0 and -dF/dz of the ubar/vbar fluxes averaged onto the u
 * and v columns to G_u and G_v (buoyancy-tracer models).  fn = NULL removes it. */
typedef void (*orc_face_flux_fn)(void* ctx, orc_model* m, double* F);
void orc_set_face_flux(orc_model* m, orc_face_flux_fn fn, void* ctx);
/* Hook of a learned closure in diffusivity form: at the start of every stage of the time stepper,
 * fn(ctx, m, K) with the stage's initial state in m fills K [3][Nz+1][Ny][Nx] with the eddy
 * diffusivity of the tracers (K[0]) and of momentum (K[1]) at every w-face of every column (K[2]
 * unused); their horizontal means over the grid at the interior faces (0 at the walls) become the
 * vertical diffusivity profiles of that stage's semi-implicit column solve (Eq.
 * tracer-time-discretization, Eq. predictor-velocity): kappa for every tracer, nu for u, v, w.
 * Setting it makes the model's vertical diffusion implicit; fn = NULL removes it (the profiles
 * of the last stage stay). */
void orc_set_face_diffusivity(orc_model* m, orc_face_flux_fn fn, void* ctx);

/* Vertical diffusion operator D(q) = d/dz (kappa dq/dz) of one column with no flux through the walls,
 * second order (fluxes -kappa_f (q_k - q_{k-1})/dz_f at the interior faces, divergence over dz_c):
 * staggering 0 = q at centres (Nz values, kappa at the Nz+1 faces), 1 = q at the faces (Nz+1 values,
 * walls held at 0, diffusivity at the centres = mean of the two faces).  The implicit solve returns
 * q with (I - dtau D) q = rhs (Thomas algorithm in FP64). */
void orc_vertical_diffusion(const orc_model* m, int staggering, const double* kappa_faces, const double* q, double* out);
void orc_vertical_implicit_solve(const orc_model* m, int staggering, const double* kappa_faces, double dtau,
                                 const double* rhs, double* q);

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
