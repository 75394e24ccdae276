/*
 * Plain FP64 CPU oracle for the nonhydrostatic Boussinesq RK3 substep.
 *
 * ORACLE / TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares nothing with the
 * CUDA library.
 *
 * Every tendency value is computed "from scratch" at its point: both fluxes of
 * each direction are evaluated by the flux functions below, which follow the
 * paper's finite-volume statements term by term:
 *   - flux-form advection, Eq. flux-form-advection and Eq.
 *     advection-flux-divergence; momentum per Sec. B.2.1 (centered advecting
 *     velocity of order N-1, WENO advected velocity of order N);
 *   - WENO reconstruction, Eq. fifth-order-weno generalised to order 2r-1 with
 *     Jiang-Shu smoothness indicators and WENO-Z weights (Sec. B.2);
 *   - flux divergence (1/V) sum delta(A J), Eq. flux-divergence;
 *   - closures, Sec. 3.1.1 (ScalarDiffusivity Laplacian form; eddy-viscosity
 *     stress form for Smagorinsky-Lilly and AMD);
 *   - RK3, Eq. rk3 (gamma, zeta); pressure correction, Eqs. predictor-velocity,
 *     pressure-correction, pressure-poisson; FFT + tridiagonal Poisson solve
 *     (Appendix A.2 and the eigenfunction expansion described there).
 * Parity unpinned: WENO-Z epsilon and tau, the closures' constants and
 * averaging stencils (their formulas are pinned in closed form on linear
 * fields), the Coriolis 4-point average, EOS constants, the flux sign
 * convention (decisions, see ocn_oracle.h).
 */
#include "ocn_oracle.h"
#include "coeffs.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define WENO_EPS 1e-8

struct orc_model {
  orc_params p;
  int Nx, Ny, Nz, R, P, nt;
  double dx, dy;
  double *zf, *zc, *dzc, *dzf;      /* dzf[k] = zc[k]-zc[k-1] for 1<=k<=Nz-1 */
  double *u, *v, *w, *c[ORC_MAX_TRACERS], *pr;
  double *Gu, *Gv, *Gw, *Gc[ORC_MAX_TRACERS];       /* G^{m-1} */
  double *Hu, *Hv, *Hw, *Hc[ORC_MAX_TRACERS];       /* G^m work */
  double *nue, *kape[ORC_MAX_TRACERS];              /* diffusivities at centres */
  double *work;                                     /* Nz*Ny*Nx scratch */
  int have_diff;
  double *nuz, *kapz;                               /* vertical diffusivity profiles at faces (or NULL) */
  int ab_started;                                   /* QAB2: a previous tendency exists */
  orc_face_flux_fn flux_fn;                         /* column closure hook (or NULL) */
  void* flux_ctx;
  orc_face_flux_fn diff_fn;                         /* learned-diffusivity hook (or NULL) */
  void* diff_ctx;
  double* Fcol;                                     /* [3][Nz+1][Ny][Nx] face fluxes of b, ubar, vbar */
};

/* ------------------------------------------------------------------ */
/* indexing                                                            */
static inline int wrapn(int i, int n) { i %= n; return i < 0 ? i + n : i; }
static inline size_t ID(const orc_model* m, int i, int j, int k) {
  return ((size_t)k * m->Ny + (size_t)wrapn(j, m->Ny)) * m->Nx + (size_t)wrapn(i, m->Nx);
}
static inline double A3(const orc_model* m, const double* a, int i, int j, int k) { return a[ID(m, i, j, k)]; }

/* ------------------------------------------------------------------ */
/* reconstruction (Sec. B.2)                                           */
double orc_centered(const double* s, int p) {
  double acc = 0.0;
  for (int n = 0; n < 2 * p; ++n) acc += ORC_CENTERED[p][n] * s[n];
  return acc;
}

void orc_weno_parts(const double* s, int r, double vel, double* q, double* beta) {
  /* t[n] = value of the cell at offset -r+n from the interface, in the frame
   * where the flow goes in +x (mirror the stencil when vel < 0). */
  double t[2 * ORC_RMAX];
  for (int n = 0; n < 2 * r; ++n) t[n] = (vel >= 0.0) ? s[n] : s[2 * r - 1 - n];
  for (int sidx = 0; sidx < r; ++sidx) {
    double acc = 0.0, b = 0.0;
    for (int n = 0; n < r; ++n) acc += ORC_SUB[r][sidx][n] * t[sidx + n];
    for (int a = 0; a < r; ++a)
      for (int bb = 0; bb < r; ++bb) b += ORC_BETA[r][sidx][a][bb] * t[sidx + a] * t[sidx + bb];
    q[sidx] = acc;
    beta[sidx] = b;
  }
}

double orc_weno(const double* s, int r, double vel) {
  double q[ORC_RMAX], beta[ORC_RMAX];
  orc_weno_parts(s, r, vel, q, beta);
  double tau = fabs(beta[0] - beta[r - 1]);
  double num = 0.0, den = 0.0;
  for (int sidx = 0; sidx < r; ++sidx) {
    double ratio = tau / (beta[sidx] + WENO_EPS);
    double alpha = ORC_D[r][sidx] * (1.0 + ratio * ratio);
    num += alpha * q[sidx];
    den += alpha;
  }
  return num / den;
}

/* largest usable half-width at interface m of a line whose valid indices are lo..hi */
static inline int reduce_halfwidth(int want, int m, int lo, int hi) {
  int r = want;
  if (m - lo < r) r = m - lo;
  if (hi - m + 1 < r) r = hi - m + 1;
  return r;
}

/* Lines: gather q(m-h .. m+h-1) along a direction through (i,j,k). */
static void line_x(const orc_model* M, const double* a, int m, int j, int k, int h, double* out) {
  for (int n = 0; n < 2 * h; ++n) out[n] = A3(M, a, m - h + n, j, k);
}
static void line_y(const orc_model* M, const double* a, int i, int m, int k, int h, double* out) {
  for (int n = 0; n < 2 * h; ++n) out[n] = A3(M, a, i, m - h + n, k);
}
static void line_z(const orc_model* M, const double* a, int i, int j, int m, int h, double* out) {
  for (int n = 0; n < 2 * h; ++n) out[n] = A3(M, a, i, j, m - h + n);
}

/* centered / WENO at interface m of periodic x or y lines */
static double cen_x(const orc_model* M, const double* a, int m, int j, int k) {
  double s[2 * ORC_PMAX]; line_x(M, a, m, j, k, M->P, s); return orc_centered(s, M->P);
}
static double cen_y(const orc_model* M, const double* a, int i, int m, int k) {
  double s[2 * ORC_PMAX]; line_y(M, a, i, m, k, M->P, s); return orc_centered(s, M->P);
}
static double weno_x(const orc_model* M, const double* a, int m, int j, int k, double vel) {
  double s[2 * ORC_RMAX]; line_x(M, a, m, j, k, M->R, s); return orc_weno(s, M->R, vel);
}
static double weno_y(const orc_model* M, const double* a, int i, int m, int k, double vel) {
  double s[2 * ORC_RMAX]; line_y(M, a, i, m, k, M->R, s); return orc_weno(s, M->R, vel);
}
/* bounded z: valid indices 0..hi (hi = Nz-1 for centre fields, Nz for w) */
static double cen_z(const orc_model* M, const double* a, int i, int j, int m, int hi) {
  int p = reduce_halfwidth(M->P, m, 0, hi);
  double s[2 * ORC_PMAX]; line_z(M, a, i, j, m, p, s); return orc_centered(s, p);
}
static double weno_z(const orc_model* M, const double* a, int i, int j, int m, int hi, double vel) {
  int r = reduce_halfwidth(M->R, m, 0, hi);
  double s[2 * ORC_RMAX]; line_z(M, a, i, j, m, r, s); return orc_weno(s, r, vel);
}

/* ------------------------------------------------------------------ */
/* buoyancy (Eq. buoyancy; BuoyancyTracer or LinearEquationOfState)   */
static double buoyancy(const orc_model* M, int i, int j, int k) {
  if (M->p.eos == ORC_EOS_BUOYANCY_TRACER) return A3(M, M->c[0], i, j, k);
  double T = A3(M, M->c[0], i, j, k), S = A3(M, M->c[1], i, j, k);
  return M->p.g * (M->p.alpha * (T - M->p.T0) - M->p.beta * (S - M->p.S0));
}

/* ------------------------------------------------------------------ */
/* velocity gradients at their natural staggered locations             */
static double dudx_ccc(const orc_model* M, int i, int j, int k) { return (A3(M, M->u, i + 1, j, k) - A3(M, M->u, i, j, k)) / M->dx; }
static double dvdy_ccc(const orc_model* M, int i, int j, int k) { return (A3(M, M->v, i, j + 1, k) - A3(M, M->v, i, j, k)) / M->dy; }
static double dwdz_ccc(const orc_model* M, int i, int j, int k) { return (A3(M, M->w, i, j, k + 1) - A3(M, M->w, i, j, k)) / M->dzc[k]; }
static double dudy_ffc(const orc_model* M, int i, int j, int k) { return (A3(M, M->u, i, j, k) - A3(M, M->u, i, j - 1, k)) / M->dy; }
static double dvdx_ffc(const orc_model* M, int i, int j, int k) { return (A3(M, M->v, i, j, k) - A3(M, M->v, i - 1, j, k)) / M->dx; }
/* z-face gradients: zero at the walls (free slip, w = 0 there) */
static double dudz_fcf(const orc_model* M, int i, int j, int k) {
  if (k <= 0 || k >= M->Nz) return 0.0;
  return (A3(M, M->u, i, j, k) - A3(M, M->u, i, j, k - 1)) / M->dzf[k];
}
static double dvdz_cff(const orc_model* M, int i, int j, int k) {
  if (k <= 0 || k >= M->Nz) return 0.0;
  return (A3(M, M->v, i, j, k) - A3(M, M->v, i, j, k - 1)) / M->dzf[k];
}
static double dwdx_fcf(const orc_model* M, int i, int j, int k) { return (A3(M, M->w, i, j, k) - A3(M, M->w, i - 1, j, k)) / M->dx; }
static double dwdy_cff(const orc_model* M, int i, int j, int k) { return (A3(M, M->w, i, j, k) - A3(M, M->w, i, j - 1, k)) / M->dy; }
static double S12_ffc(const orc_model* M, int i, int j, int k) { return 0.5 * (dudy_ffc(M, i, j, k) + dvdx_ffc(M, i, j, k)); }
static double S13_fcf(const orc_model* M, int i, int j, int k) { return 0.5 * (dudz_fcf(M, i, j, k) + dwdx_fcf(M, i, j, k)); }
static double S23_cff(const orc_model* M, int i, int j, int k) { return 0.5 * (dvdz_cff(M, i, j, k) + dwdy_cff(M, i, j, k)); }

/* tracer gradient across a z-face (zero at walls) */
static double dcdz_ccf(const orc_model* M, const double* c, int i, int j, int k) {
  if (k <= 0 || k >= M->Nz) return 0.0;
  return (A3(M, c, i, j, k) - A3(M, c, i, j, k - 1)) / M->dzf[k];
}
static double dbdz_ccf(const orc_model* M, int i, int j, int k) {
  if (k <= 0 || k >= M->Nz) return 0.0;
  return (buoyancy(M, i, j, k) - buoyancy(M, i, j, k - 1)) / M->dzf[k];
}

/* ------------------------------------------------------------------ */
/* eddy diffusivities at cell centres (Sec. 3.1.1)                      */
static void velocity_gradient_ccc(const orc_model* M, int i, int j, int k, double G[3][3]) {
  /* G[a][b] = d u_a / d x_b, averaged onto the centre from its natural location */
  G[0][0] = dudx_ccc(M, i, j, k);
  G[1][1] = dvdy_ccc(M, i, j, k);
  G[2][2] = dwdz_ccc(M, i, j, k);
  G[0][1] = 0.25 * (dudy_ffc(M, i, j, k) + dudy_ffc(M, i + 1, j, k) + dudy_ffc(M, i, j + 1, k) + dudy_ffc(M, i + 1, j + 1, k));
  G[1][0] = 0.25 * (dvdx_ffc(M, i, j, k) + dvdx_ffc(M, i + 1, j, k) + dvdx_ffc(M, i, j + 1, k) + dvdx_ffc(M, i + 1, j + 1, k));
  G[0][2] = 0.25 * (dudz_fcf(M, i, j, k) + dudz_fcf(M, i + 1, j, k) + dudz_fcf(M, i, j, k + 1) + dudz_fcf(M, i + 1, j, k + 1));
  G[2][0] = 0.25 * (dwdx_fcf(M, i, j, k) + dwdx_fcf(M, i + 1, j, k) + dwdx_fcf(M, i, j, k + 1) + dwdx_fcf(M, i + 1, j, k + 1));
  G[1][2] = 0.25 * (dvdz_cff(M, i, j, k) + dvdz_cff(M, i, j + 1, k) + dvdz_cff(M, i, j, k + 1) + dvdz_cff(M, i, j + 1, k + 1));
  G[2][1] = 0.25 * (dwdy_cff(M, i, j, k) + dwdy_cff(M, i, j + 1, k) + dwdy_cff(M, i, j, k + 1) + dwdy_cff(M, i, j + 1, k + 1));
}

static double smagorinsky_nu(const orc_model* M, int i, int j, int k) {
  /* Strain rate S = (grad u + grad u^T)/2; off-diagonal parts averaged from edges. */
  double S11 = dudx_ccc(M, i, j, k), S22 = dvdy_ccc(M, i, j, k), S33 = dwdz_ccc(M, i, j, k);
  double S12 = 0.25 * (S12_ffc(M, i, j, k) + S12_ffc(M, i + 1, j, k) + S12_ffc(M, i, j + 1, k) + S12_ffc(M, i + 1, j + 1, k));
  double S13 = 0.25 * (S13_fcf(M, i, j, k) + S13_fcf(M, i + 1, j, k) + S13_fcf(M, i, j, k + 1) + S13_fcf(M, i + 1, j, k + 1));
  double S23 = 0.25 * (S23_cff(M, i, j, k) + S23_cff(M, i, j + 1, k) + S23_cff(M, i, j, k + 1) + S23_cff(M, i, j + 1, k + 1));
  double SS = 2.0 * (S11 * S11 + S22 * S22 + S33 * S33 + 2.0 * (S12 * S12 + S13 * S13 + S23 * S23)); /* |S|^2 */
  if (!(SS > 0.0)) return 0.0;
  double N2 = 0.5 * (dbdz_ccf(M, i, j, k) + dbdz_ccf(M, i, j, k + 1));
  double Delta = cbrt(M->dx * M->dy * M->dzc[k]);
  double CD = M->p.Cs * Delta;
  double stab = 1.0 - M->p.Cb * N2 / (M->p.Pr * SS);
  if (stab < 0.0) stab = 0.0;
  return CD * CD * sqrt(SS) * sqrt(stab);
}

static double amd_nu(const orc_model* M, int i, int j, int k) {
  double G[3][3];
  velocity_gradient_ccc(M, i, j, k, G);
  double D2[3] = {M->dx * M->dx, M->dy * M->dy, M->dzc[k] * M->dzc[k]};
  double num = 0.0, den = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double Sab = 0.5 * (G[a][b] + G[b][a]);
      for (int kk = 0; kk < 3; ++kk) num += D2[kk] * G[a][kk] * G[b][kk] * Sab;
      den += G[a][b] * G[a][b];
    }
  if (!(den > 0.0)) return 0.0;
  double nu = -M->p.C_amd * num / den;
  return nu > 0.0 ? nu : 0.0;
}

static double amd_kappa(const orc_model* M, const double* c, int i, int j, int k) {
  double G[3][3];
  velocity_gradient_ccc(M, i, j, k, G);
  double D2[3] = {M->dx * M->dx, M->dy * M->dy, M->dzc[k] * M->dzc[k]};
  double dc[3];
  dc[0] = 0.5 * ((A3(M, c, i, j, k) - A3(M, c, i - 1, j, k)) + (A3(M, c, i + 1, j, k) - A3(M, c, i, j, k))) / M->dx;
  dc[1] = 0.5 * ((A3(M, c, i, j, k) - A3(M, c, i, j - 1, k)) + (A3(M, c, i, j + 1, k) - A3(M, c, i, j, k))) / M->dy;
  dc[2] = 0.5 * (dcdz_ccf(M, c, i, j, k) + dcdz_ccf(M, c, i, j, k + 1));
  double num = 0.0, den = 0.0;
  for (int kk = 0; kk < 3; ++kk)
    for (int a = 0; a < 3; ++a) num += D2[kk] * G[a][kk] * dc[kk] * dc[a];
  for (int a = 0; a < 3; ++a) den += dc[a] * dc[a];
  if (!(den > 0.0)) return 0.0;
  double kap = -M->p.C_amd * num / den;
  return kap > 0.0 ? kap : 0.0;
}

double orc_diffusivity_at(orc_model* M, int which, int i, int j, int k) {
  if (M->p.closure == ORC_CLOSURE_SMAG) {
    double nu = smagorinsky_nu(M, i, j, k);
    return which == 0 ? nu : nu / M->p.Pr;
  }
  if (M->p.closure == ORC_CLOSURE_AMD) {
    return which == 0 ? amd_nu(M, i, j, k) : amd_kappa(M, M->c[which - 1], i, j, k);
  }
  if (M->p.closure == ORC_CLOSURE_SCALAR) return which == 0 ? M->p.nu : M->p.kappa;
  return 0.0;
}

static void compute_diffusivities(orc_model* M) {
  if (M->p.closure != ORC_CLOSURE_SMAG && M->p.closure != ORC_CLOSURE_AMD) { M->have_diff = 0; return; }
  int Nx = M->Nx, Ny = M->Ny, Nz = M->Nz;
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < Nz; ++k)
    for (int j = 0; j < Ny; ++j)
      for (int i = 0; i < Nx; ++i) {
        size_t id = ID(M, i, j, k);
        M->nue[id] = orc_diffusivity_at(M, 0, i, j, k);
        for (int n = 0; n < M->nt; ++n) M->kape[n][id] = orc_diffusivity_at(M, 1 + n, i, j, k);
      }
  M->have_diff = 1;
}

/* diffusivity lookups (from the per-stage arrays when present, else computed) */
static inline double NU(const orc_model* M, int i, int j, int k) {
  return M->have_diff ? A3(M, M->nue, i, j, k) : orc_diffusivity_at((orc_model*)M, 0, i, j, k);
}
static inline double KAP(const orc_model* M, int n, int i, int j, int k) {
  if (M->p.closure == ORC_CLOSURE_SMAG) return NU(M, i, j, k) / M->p.Pr;
  return M->have_diff ? A3(M, M->kape[n], i, j, k) : orc_diffusivity_at((orc_model*)M, 1 + n, i, j, k);
}
static inline int stress_closure(const orc_model* M) { return M->p.closure == ORC_CLOSURE_SMAG || M->p.closure == ORC_CLOSURE_AMD; }

/* ------------------------------------------------------------------ */
/* Fluxes.  Each F*_q(i,j,k) is the total (advective + closure) flux of q
 * through the left (x), south (y) or bottom (z) face of control volume
 * (i,j,k) of q, so that G_q = -(F(i+1)-F(i))/dx - ... (Eq. flux-divergence). */

/* u at fcc: x-faces are centres i-1; y-faces are ffc (i,j); z-faces are fcf (i,k) */
static double Fx_u(const orc_model* M, int i, int j, int k) {
  double U = cen_x(M, M->u, i, j, k);
  double F = U * weno_x(M, M->u, i, j, k, U);
  if (M->p.closure == ORC_CLOSURE_SCALAR) F += -M->p.nu * (A3(M, M->u, i, j, k) - A3(M, M->u, i - 1, j, k)) / M->dx;
  else if (stress_closure(M)) F += -2.0 * NU(M, i - 1, j, k) * dudx_ccc(M, i - 1, j, k);
  return F;
}
static double nu_ffc(const orc_model* M, int i, int j, int k) {
  return 0.25 * (NU(M, i - 1, j - 1, k) + NU(M, i, j - 1, k) + NU(M, i - 1, j, k) + NU(M, i, j, k));
}
static double nu_fcf(const orc_model* M, int i, int j, int k) {
  return 0.25 * (NU(M, i - 1, j, k - 1) + NU(M, i, j, k - 1) + NU(M, i - 1, j, k) + NU(M, i, j, k));
}
static double nu_cff(const orc_model* M, int i, int j, int k) {
  return 0.25 * (NU(M, i, j - 1, k - 1) + NU(M, i, j, k - 1) + NU(M, i, j - 1, k) + NU(M, i, j, k));
}
static double Fy_u(const orc_model* M, int i, int j, int k) {
  double V = cen_x(M, M->v, i, j, k);
  double F = V * weno_y(M, M->u, i, j, k, V);
  if (M->p.closure == ORC_CLOSURE_SCALAR) F += -M->p.nu * dudy_ffc(M, i, j, k);
  else if (stress_closure(M)) F += -2.0 * nu_ffc(M, i, j, k) * S12_ffc(M, i, j, k);
  return F;
}
static double Fz_u(const orc_model* M, int i, int j, int k) {
  if (k == 0) return M->p.bottom_flux[0];
  if (k == M->Nz) return M->p.top_flux[0];
  double W = cen_x(M, M->w, i, j, k);
  double F = W * weno_z(M, M->u, i, j, k, M->Nz - 1, W);
  if (M->p.closure == ORC_CLOSURE_SCALAR) F += -M->p.nu * dudz_fcf(M, i, j, k);
  else if (stress_closure(M)) F += -2.0 * nu_fcf(M, i, j, k) * S13_fcf(M, i, j, k);
  return F;
}

/* v at cfc: x-faces ffc (i,j); y-faces are centres j-1; z-faces cff (j,k) */
static double Fx_v(const orc_model* M, int i, int j, int k) {
  double U = cen_y(M, M->u, i, j, k);
  double F = U * weno_x(M, M->v, i, j, k, U);
  if (M->p.closure == ORC_CLOSURE_SCALAR) F += -M->p.nu * dvdx_ffc(M, i, j, k);
  else if (stress_closure(M)) F += -2.0 * nu_ffc(M, i, j, k) * S12_ffc(M, i, j, k);
  return F;
}
static double Fy_v(const orc_model* M, int i, int j, int k) {
  double V = cen_y(M, M->v, i, j, k);
  double F = V * weno_y(M, M->v, i, j, k, V);
  if (M->p.closure == ORC_CLOSURE_SCALAR) F += -M->p.nu * (A3(M, M->v, i, j, k) - A3(M, M->v, i, j - 1, k)) / M->dy;
  else if (stress_closure(M)) F += -2.0 * NU(M, i, j - 1, k) * dvdy_ccc(M, i, j - 1, k);
  return F;
}
static double Fz_v(const orc_model* M, int i, int j, int k) {
  if (k == 0) return M->p.bottom_flux[1];
  if (k == M->Nz) return M->p.top_flux[1];
  double W = cen_y(M, M->w, i, j, k);
  double F = W * weno_z(M, M->v, i, j, k, M->Nz - 1, W);
  if (M->p.closure == ORC_CLOSURE_SCALAR) F += -M->p.nu * dvdz_cff(M, i, j, k);
  else if (stress_closure(M)) F += -2.0 * nu_cff(M, i, j, k) * S23_cff(M, i, j, k);
  return F;
}

/* w at ccf (interior faces 1..Nz-1): x-faces fcf (i,k); y-faces cff (j,k);
 * z-faces are centres m-1 for interface m = 1..Nz */
static double Fx_w(const orc_model* M, int i, int j, int k) {
  double U = cen_z(M, M->u, i, j, k, M->Nz - 1);
  double F = U * weno_x(M, M->w, i, j, k, U);
  if (M->p.closure == ORC_CLOSURE_SCALAR) F += -M->p.nu * dwdx_fcf(M, i, j, k);
  else if (stress_closure(M)) F += -2.0 * nu_fcf(M, i, j, k) * S13_fcf(M, i, j, k);
  return F;
}
static double Fy_w(const orc_model* M, int i, int j, int k) {
  double V = cen_z(M, M->v, i, j, k, M->Nz - 1);
  double F = V * weno_y(M, M->w, i, j, k, V);
  if (M->p.closure == ORC_CLOSURE_SCALAR) F += -M->p.nu * dwdy_cff(M, i, j, k);
  else if (stress_closure(M)) F += -2.0 * nu_cff(M, i, j, k) * S23_cff(M, i, j, k);
  return F;
}
static double Fz_w(const orc_model* M, int i, int j, int m) {
  double W = cen_z(M, M->w, i, j, m, M->Nz);
  double F = W * weno_z(M, M->w, i, j, m, M->Nz, W);
  if (M->p.closure == ORC_CLOSURE_SCALAR) F += -M->p.nu * (A3(M, M->w, i, j, m) - A3(M, M->w, i, j, m - 1)) / M->dzc[m - 1];
  else if (stress_closure(M)) F += -2.0 * NU(M, i, j, m - 1) * dwdz_ccc(M, i, j, m - 1);
  return F;
}

/* tracers at ccc: faces fcc (i), cfc (j), ccf (k) */
static double Fx_c(const orc_model* M, int n, int i, int j, int k) {
  const double* c = M->c[n];
  double U = A3(M, M->u, i, j, k);
  double F = U * weno_x(M, c, i, j, k, U);
  double dc = (A3(M, c, i, j, k) - A3(M, c, i - 1, j, k)) / M->dx;
  if (M->p.closure == ORC_CLOSURE_SCALAR) F += -M->p.kappa * dc;
  else if (stress_closure(M)) F += -0.5 * (KAP(M, n, i - 1, j, k) + KAP(M, n, i, j, k)) * dc;
  return F;
}
static double Fy_c(const orc_model* M, int n, int i, int j, int k) {
  const double* c = M->c[n];
  double V = A3(M, M->v, i, j, k);
  double F = V * weno_y(M, c, i, j, k, V);
  double dc = (A3(M, c, i, j, k) - A3(M, c, i, j - 1, k)) / M->dy;
  if (M->p.closure == ORC_CLOSURE_SCALAR) F += -M->p.kappa * dc;
  else if (stress_closure(M)) F += -0.5 * (KAP(M, n, i, j - 1, k) + KAP(M, n, i, j, k)) * dc;
  return F;
}
static double Fz_c(const orc_model* M, int n, int i, int j, int k) {
  if (k == 0) return M->p.bottom_flux[2 + n];
  if (k == M->Nz) return M->p.top_flux[2 + n];
  const double* c = M->c[n];
  double W = A3(M, M->w, i, j, k);
  double F = W * weno_z(M, c, i, j, k, M->Nz - 1, W);
  double dc = dcdz_ccf(M, c, i, j, k);
  if (M->p.closure == ORC_CLOSURE_SCALAR) F += -M->p.kappa * dc;
  else if (stress_closure(M)) F += -0.5 * (KAP(M, n, i, j, k - 1) + KAP(M, n, i, j, k)) * dc;
  return F;
}

/* ------------------------------------------------------------------ */
/* tendencies (Eq. nonhydrotatic-momentum-equations with p excluded,     */
/* Eq. nonhydrostatic-tracer-equation)                                 */
static double G_u(const orc_model* M, int i, int j, int k) {
  double G = -(Fx_u(M, i + 1, j, k) - Fx_u(M, i, j, k)) / M->dx
             - (Fy_u(M, i, j + 1, k) - Fy_u(M, i, j, k)) / M->dy
             - (Fz_u(M, i, j, k + 1) - Fz_u(M, i, j, k)) / M->dzc[k];
  /* -f z x u: +f v, with v averaged onto the u point */
  double vbar = 0.25 * (A3(M, M->v, i - 1, j, k) + A3(M, M->v, i, j, k) + A3(M, M->v, i - 1, j + 1, k) + A3(M, M->v, i, j + 1, k));
  return G + M->p.f * vbar;
}
static double G_v(const orc_model* M, int i, int j, int k) {
  double G = -(Fx_v(M, i + 1, j, k) - Fx_v(M, i, j, k)) / M->dx
             - (Fy_v(M, i, j + 1, k) - Fy_v(M, i, j, k)) / M->dy
             - (Fz_v(M, i, j, k + 1) - Fz_v(M, i, j, k)) / M->dzc[k];
  double ubar = 0.25 * (A3(M, M->u, i, j - 1, k) + A3(M, M->u, i + 1, j - 1, k) + A3(M, M->u, i, j, k) + A3(M, M->u, i + 1, j, k));
  return G - M->p.f * ubar;
}
static double G_w(const orc_model* M, int i, int j, int k) {
  if (k <= 0 || k >= M->Nz) return 0.0;
  double G = -(Fx_w(M, i + 1, j, k) - Fx_w(M, i, j, k)) / M->dx
             - (Fy_w(M, i, j + 1, k) - Fy_w(M, i, j, k)) / M->dy
             - (Fz_w(M, i, j, k + 1) - Fz_w(M, i, j, k)) / M->dzf[k];
  /* buoyancy -b g_hat = +b z_hat, b averaged onto the w point */
  return G + 0.5 * (buoyancy(M, i, j, k - 1) + buoyancy(M, i, j, k));
}
static double G_c(const orc_model* M, int n, int i, int j, int k) {
  return -(Fx_c(M, n, i + 1, j, k) - Fx_c(M, n, i, j, k)) / M->dx
         - (Fy_c(M, n, i, j + 1, k) - Fy_c(M, n, i, j, k)) / M->dy
         - (Fz_c(M, n, i, j, k + 1) - Fz_c(M, n, i, j, k)) / M->dzc[k];
}

double orc_tendency_at(orc_model* M, int field, int i, int j, int k) {
  M->have_diff = 0;    /* pointwise: diffusivities recomputed from the state */
  if (field == ORC_U) return G_u(M, i, j, k);
  if (field == ORC_V) return G_v(M, i, j, k);
  if (field == ORC_W) return G_w(M, i, j, k);
  return G_c(M, field - ORC_C0, i, j, k);
}

static void add_face_flux_divergence(orc_model* M, double* Gu, double* Gv, double* Gb);
static void add_vertical_diffusion(orc_model* M, double* Gu, double* Gv, double* Gw, double** Gc);
static void implicit_vertical_step(orc_model* M, double dtau);

static void all_tendencies(orc_model* M, double* Gu, double* Gv, double* Gw, double** Gc) {
  compute_diffusivities(M);
  int Nx = M->Nx, Ny = M->Ny, Nz = M->Nz;
#pragma omp parallel for collapse(2) schedule(dynamic, 1)
  for (int k = 0; k < Nz; ++k)
    for (int j = 0; j < Ny; ++j)
      for (int i = 0; i < Nx; ++i) {
        size_t id = ID(M, i, j, k);
        Gu[id] = G_u(M, i, j, k);
        Gv[id] = G_v(M, i, j, k);
        Gw[id] = G_w(M, i, j, k);
        for (int n = 0; n < M->nt; ++n) Gc[n][id] = G_c(M, n, i, j, k);
      }
  size_t plane = (size_t)Nx * Ny;
  memset(Gw + (size_t)Nz * plane, 0, plane * sizeof(double));
  if (M->flux_fn) add_face_flux_divergence(M, Gu, Gv, Gc[0]);
  if (!M->p.vertical_implicit && (M->nuz || M->kapz)) add_vertical_diffusion(M, Gu, Gv, Gw, Gc);
}

void orc_tendencies(orc_model* M, double* Gu, double* Gv, double* Gw, double* Gc) {
  double* gc[ORC_MAX_TRACERS];
  size_t N = (size_t)M->Nx * M->Ny * M->Nz;
  for (int n = 0; n < M->nt; ++n) gc[n] = Gc + n * N;
  all_tendencies(M, Gu, Gv, Gw, gc);
  M->have_diff = 0;
}

/* ------------------------------------------------------------------ */
/* FFT: recursive mixed radix on the smallest prime factor (plain DFT    */
/* combination), any n.                                                */
static void fft_rec(double* re, double* im, int n, int sign, double* scratch) {
  if (n <= 1) return;
  int p = 2;
  while (n % p) ++p;
  int m = n / p;
  double* sre = scratch;            /* p sub-sequences, each m long */
  double* sim = scratch + n;
  double* deeper = scratch + 2 * n;
  for (int r = 0; r < p; ++r)
    for (int t = 0; t < m; ++t) {
      sre[r * m + t] = re[t * p + r];
      sim[r * m + t] = im[t * p + r];
    }
  for (int r = 0; r < p; ++r) fft_rec(sre + r * m, sim + r * m, m, sign, deeper);
  for (int kk = 0; kk < n; ++kk) {
    double ar = 0.0, ai = 0.0;
    for (int r = 0; r < p; ++r) {
      long ang = ((long)r * kk) % n;
      double th = sign * 2.0 * M_PI * (double)ang / (double)n;
      double c = cos(th), s = sin(th);
      double xr = sre[r * m + kk % m], xi = sim[r * m + kk % m];
      ar += c * xr - s * xi;
      ai += c * xi + s * xr;
    }
    re[kk] = ar;
    im[kk] = ai;
  }
}

void orc_fft(double* re, double* im, int n, int sign) {
  double* scratch = (double*)malloc(sizeof(double) * 4 * (size_t)n + 64);
  fft_rec(re, im, n, sign, scratch);
  free(scratch);
}

/* ------------------------------------------------------------------ */
/* Poisson: lap p = rhs.  Horizontal eigenfunction expansion by FFT,     */
/* tridiagonal (Thomas) in z, Neumann walls, zero volume mean.          */
void orc_poisson(orc_model* M, const double* rhs, double* pout) {
  int Nx = M->Nx, Ny = M->Ny, Nz = M->Nz;
  size_t plane = (size_t)Nx * Ny, N = plane * Nz;
  double* Xr = (double*)malloc(sizeof(double) * N);
  double* Xi = (double*)malloc(sizeof(double) * N);
  memcpy(Xr, rhs, sizeof(double) * N);
  memset(Xi, 0, sizeof(double) * N);
  int L = Nx > Ny ? Nx : Ny;
  /* forward 2D FFT of each plane */
#pragma omp parallel
  {
    double* lr = (double*)malloc(sizeof(double) * L);
    double* li = (double*)malloc(sizeof(double) * L);
    double* scr = (double*)malloc(sizeof(double) * 4 * L + 64);
#pragma omp for collapse(2)
    for (int k = 0; k < Nz; ++k)
      for (int j = 0; j < Ny; ++j) {
        size_t o = k * plane + (size_t)j * Nx;
        for (int i = 0; i < Nx; ++i) { lr[i] = Xr[o + i]; li[i] = Xi[o + i]; }
        fft_rec(lr, li, Nx, -1, scr);
        for (int i = 0; i < Nx; ++i) { Xr[o + i] = lr[i]; Xi[o + i] = li[i]; }
      }
#pragma omp for collapse(2)
    for (int k = 0; k < Nz; ++k)
      for (int i = 0; i < Nx; ++i) {
        size_t o = k * plane + i;
        for (int j = 0; j < Ny; ++j) { lr[j] = Xr[o + (size_t)j * Nx]; li[j] = Xi[o + (size_t)j * Nx]; }
        fft_rec(lr, li, Ny, -1, scr);
        for (int j = 0; j < Ny; ++j) { Xr[o + (size_t)j * Nx] = lr[j]; Xi[o + (size_t)j * Nx] = li[j]; }
      }
    free(lr); free(li); free(scr);
  }
  /* tridiagonal solve per horizontal wavenumber */
#pragma omp parallel
  {
    double* cp = (double*)malloc(sizeof(double) * Nz);
    double* dr = (double*)malloc(sizeof(double) * Nz);
    double* di = (double*)malloc(sizeof(double) * Nz);
#pragma omp for collapse(2)
    for (int ky = 0; ky < Ny; ++ky)
      for (int kx = 0; kx < Nx; ++kx) {
        double sx = 2.0 * sin(M_PI * kx / Nx) / M->dx, sy = 2.0 * sin(M_PI * ky / Ny) / M->dy;
        double lam = -(sx * sx) - (sy * sy);
        int gauge = (kx == 0 && ky == 0);
        double prev_c = 0.0, prev_dr = 0.0, prev_di = 0.0;
        for (int k = 0; k < Nz; ++k) {
          double a = (k > 0) ? 1.0 / (M->dzc[k] * M->dzf[k]) : 0.0;
          double c = (k < Nz - 1) ? 1.0 / (M->dzc[k] * M->dzf[k + 1]) : 0.0;
          double b = -(a + c) + lam;
          size_t o = (size_t)k * plane + (size_t)ky * Nx + kx;
          double rr = Xr[o], ri = Xi[o];
          if (gauge && k == 0) { a = 0.0; b = 1.0; c = 0.0; rr = 0.0; ri = 0.0; }
          double den = b - a * prev_c;
          cp[k] = c / den;
          dr[k] = (rr - a * prev_dr) / den;
          di[k] = (ri - a * prev_di) / den;
          prev_c = cp[k]; prev_dr = dr[k]; prev_di = di[k];
        }
        for (int k = Nz - 2; k >= 0; --k) {
          dr[k] -= cp[k] * dr[k + 1];
          di[k] -= cp[k] * di[k + 1];
        }
        if (gauge) {
          double sr = 0.0, si = 0.0, h = 0.0;
          for (int k = 0; k < Nz; ++k) { sr += M->dzc[k] * dr[k]; si += M->dzc[k] * di[k]; h += M->dzc[k]; }
          for (int k = 0; k < Nz; ++k) { dr[k] -= sr / h; di[k] -= si / h; }
        }
        for (int k = 0; k < Nz; ++k) {
          size_t o = (size_t)k * plane + (size_t)ky * Nx + kx;
          Xr[o] = dr[k]; Xi[o] = di[k];
        }
      }
    free(cp); free(dr); free(di);
  }
  /* inverse 2D FFT, normalise */
#pragma omp parallel
  {
    double* lr = (double*)malloc(sizeof(double) * L);
    double* li = (double*)malloc(sizeof(double) * L);
    double* scr = (double*)malloc(sizeof(double) * 4 * L + 64);
#pragma omp for collapse(2)
    for (int k = 0; k < Nz; ++k)
      for (int i = 0; i < Nx; ++i) {
        size_t o = k * plane + i;
        for (int j = 0; j < Ny; ++j) { lr[j] = Xr[o + (size_t)j * Nx]; li[j] = Xi[o + (size_t)j * Nx]; }
        fft_rec(lr, li, Ny, +1, scr);
        for (int j = 0; j < Ny; ++j) { Xr[o + (size_t)j * Nx] = lr[j]; Xi[o + (size_t)j * Nx] = li[j]; }
      }
#pragma omp for collapse(2)
    for (int k = 0; k < Nz; ++k)
      for (int j = 0; j < Ny; ++j) {
        size_t o = k * plane + (size_t)j * Nx;
        for (int i = 0; i < Nx; ++i) { lr[i] = Xr[o + i]; li[i] = Xi[o + i]; }
        fft_rec(lr, li, Nx, +1, scr);
        for (int i = 0; i < Nx; ++i) pout[o + i] = lr[i] / (double)plane;
      }
    free(lr); free(li); free(scr);
  }
  free(Xr);
  free(Xi);
}

/* ------------------------------------------------------------------ */
void orc_divergence(const orc_model* M, double* out) {
  int Nx = M->Nx, Ny = M->Ny, Nz = M->Nz;
#pragma omp parallel for collapse(2)
  for (int k = 0; k < Nz; ++k)
    for (int j = 0; j < Ny; ++j)
      for (int i = 0; i < Nx; ++i)
        out[ID(M, i, j, k)] = dudx_ccc(M, i, j, k) + dvdy_ccc(M, i, j, k) + dwdz_ccc(M, i, j, k);
}

/* Horizontal means and vertical fluxes for coarse-graining (the fine LES as training data):
 * the fluxes are the horizontal means of the model's own vertical face fluxes (advective WENO
 * flux + closure flux; prescribed fluxes at the walls). */
void orc_profiles(orc_model* M, double* out) {
  int Nx = M->Nx, Ny = M->Ny, Nz = M->Nz;
  double inv = 1.0 / ((double)Nx * Ny);
  compute_diffusivities(M);
  for (int k = 0; k < Nz; ++k) {
    double sb = 0, su = 0, sv = 0;
    for (int j = 0; j < Ny; ++j)
      for (int i = 0; i < Nx; ++i) { sb += buoyancy(M, i, j, k); su += A3(M, M->u, i, j, k); sv += A3(M, M->v, i, j, k); }
    out[k] = sb * inv; out[Nz + k] = su * inv; out[2 * Nz + k] = sv * inv;
  }
  double* F = out + 3 * Nz;
  for (int k = 0; k <= Nz; ++k) {
    double fb = 0, fu = 0, fv = 0;
    for (int j = 0; j < Ny; ++j)
      for (int i = 0; i < Nx; ++i) {
        fu += Fz_u(M, i, j, k);
        fv += Fz_v(M, i, j, k);
        if (M->p.eos == ORC_EOS_LINEAR_TS)
          fb += M->p.g * (M->p.alpha * Fz_c(M, 0, i, j, k) - M->p.beta * Fz_c(M, 1, i, j, k));
        else
          fb += Fz_c(M, 0, i, j, k);
      }
    F[k] = fb * inv; F[(Nz + 1) + k] = fu * inv; F[2 * (Nz + 1) + k] = fv * inv;
  }
  M->have_diff = 0;
}

void orc_project(orc_model* M, double dts) {
  int Nx = M->Nx, Ny = M->Ny, Nz = M->Nz;
  size_t N = (size_t)Nx * Ny * Nz;
  double* rhs = M->work;
  orc_divergence(M, rhs);
  for (size_t n = 0; n < N; ++n) rhs[n] /= dts;
  orc_poisson(M, rhs, M->pr);
  /* u^{m+1} = u~ - dt grad p on every non-wall face (Eq. pressure-correction) */
#pragma omp parallel for collapse(2)
  for (int k = 0; k < Nz; ++k)
    for (int j = 0; j < Ny; ++j)
      for (int i = 0; i < Nx; ++i) {
        size_t id = ID(M, i, j, k);
        M->u[id] -= dts * (A3(M, M->pr, i, j, k) - A3(M, M->pr, i - 1, j, k)) / M->dx;
        M->v[id] -= dts * (A3(M, M->pr, i, j, k) - A3(M, M->pr, i, j - 1, k)) / M->dy;
        if (k > 0) M->w[id] -= dts * (A3(M, M->pr, i, j, k) - A3(M, M->pr, i, j, k - 1)) / M->dzf[k];
      }
}

/* ------------------------------------------------------------------ */
static const double RK_GAMMA[3] = {8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0};
static const double RK_ZETA[3] = {0.0, 17.0 / 60.0, 5.0 / 12.0};

/* One stage: c <- c + dt (g H - z G), G <- H, the semi-implicit vertical diffusion over dtau, the projection
 * over dtau (Eq. rk3 or Eq. qab2 with Eqs. tracer-time-discretization, predictor-velocity). */
/* The stepper's tendencies follow Eq. pressure-decomposition: b leaves the w equation and the
 * hydrostatic pressure anomaly p_hy (d p_hy/dz = b, discretely (p_hy(k) - p_hy(k-1))/dz_f(k) =
 * (b(k-1) + b(k))/2 with p_hy = 0 in the bottom cell of each column) enters u and v as -grad_h p_hy.
 * With explicit terms only this differs from keeping b in G_w by a discrete gradient, which the
 * projection removes; the semi-implicit vertical step acts on the split form, as Eq.
 * predictor-velocity states. */
static void hydrostatic_split(orc_model* M, double* Hu, double* Hv, double* Hw) {
  int Nx = M->Nx, Ny = M->Ny, Nz = M->Nz;
  double* ph = M->work;
  for (int j = 0; j < Ny; ++j)
    for (int i = 0; i < Nx; ++i) {
      ph[ID(M, i, j, 0)] = 0.0;
      for (int k = 1; k < Nz; ++k)
        ph[ID(M, i, j, k)] = ph[ID(M, i, j, k - 1)] + M->dzf[k] * 0.5 * (buoyancy(M, i, j, k - 1) + buoyancy(M, i, j, k));
    }
#pragma omp parallel for collapse(2)
  for (int k = 0; k < Nz; ++k)
    for (int j = 0; j < Ny; ++j)
      for (int i = 0; i < Nx; ++i) {
        size_t id = ID(M, i, j, k);
        Hu[id] -= (A3(M, ph, i, j, k) - A3(M, ph, i - 1, j, k)) / M->dx;
        Hv[id] -= (A3(M, ph, i, j, k) - A3(M, ph, i, j - 1, k)) / M->dy;
        if (k > 0) Hw[id] -= 0.5 * (buoyancy(M, i, j, k - 1) + buoyancy(M, i, j, k));
      }
}

static void learned_profiles(orc_model* M);

static void stage(orc_model* M, double dt, double g, double z, double dtau) {
  size_t plane = (size_t)M->Nx * M->Ny, N = plane * M->Nz;
  if (M->diff_fn) learned_profiles(M);          /* from the stage's initial state */
  all_tendencies(M, M->Hu, M->Hv, M->Hw, M->Hc);
  hydrostatic_split(M, M->Hu, M->Hv, M->Hw);
#pragma omp parallel for schedule(static)
  for (size_t n = 0; n < N; ++n) {
    M->u[n] += dt * (g * M->Hu[n] - z * M->Gu[n]);
    M->v[n] += dt * (g * M->Hv[n] - z * M->Gv[n]);
    if (n >= plane) M->w[n] += dt * (g * M->Hw[n] - z * M->Gw[n]);
    for (int t = 0; t < M->nt; ++t) M->c[t][n] += dt * (g * M->Hc[t][n] - z * M->Gc[t][n]);
    M->Gu[n] = M->Hu[n]; M->Gv[n] = M->Hv[n]; M->Gw[n] = M->Hw[n];
    for (int t = 0; t < M->nt; ++t) M->Gc[t][n] = M->Hc[t][n];
  }
  M->have_diff = 0;
  if (M->p.vertical_implicit && (M->nuz || M->kapz)) implicit_vertical_step(M, dtau);
  orc_project(M, dtau);
}

void orc_time_step(orc_model* M, double dt, int nsteps) {
  for (int step = 0; step < nsteps; ++step) {
    if (M->p.timestepper == ORC_QAB2) {
      /* Eq. qab2: (3/2 + chi) G^m - (1/2 + chi) G^{m-1}; the first step is forward Euler (chi = -1/2) */
      const double chi = M->ab_started ? M->p.chi : -0.5;
      stage(M, dt, 1.5 + chi, 0.5 + chi, dt);
      M->ab_started = 1;
      continue;
    }
    for (int st = 0; st < 3; ++st) {
      double g = RK_GAMMA[st], z = RK_ZETA[st];
      stage(M, dt, g, z, (g - z) * dt);
    }
  }
}

/* ------------------------------------------------------------------ */
void orc_diagnostics(const orc_model* M, double dt, double* out) {
  int Nx = M->Nx, Ny = M->Ny, Nz = M->Nz, nt = M->nt;
  double sc[ORC_MAX_TRACERS] = {0}, su = 0, sv = 0, sw = 0, maxdiv = 0, cfl = 0, bad = 0;
  double A = M->dx * M->dy;
  for (int k = 0; k < Nz; ++k)
    for (int j = 0; j < Ny; ++j)
      for (int i = 0; i < Nx; ++i) {
        size_t id = ID(M, i, j, k);
        double V = A * M->dzc[k];
        for (int n = 0; n < nt; ++n) { sc[n] += V * M->c[n][id]; if (!isfinite(M->c[n][id])) bad += 1; }
        su += V * M->u[id];
        sv += V * M->v[id];
        double d = fabs(dudx_ccc(M, i, j, k) + dvdy_ccc(M, i, j, k) + dwdz_ccc(M, i, j, k));
        if (d > maxdiv) maxdiv = d;
        double cu = fabs(M->u[id]) / M->dx, cv = fabs(M->v[id]) / M->dy;
        if (cu > cfl) cfl = cu;
        if (cv > cfl) cfl = cv;
        if (!isfinite(M->u[id]) || !isfinite(M->v[id]) || !isfinite(M->w[id])) bad += 1;
        if (k > 0) {
          sw += A * M->dzf[k] * M->w[id];
          double cw = fabs(M->w[id]) / M->dzf[k];
          if (cw > cfl) cfl = cw;
        }
      }
  for (int n = 0; n < nt; ++n) out[n] = sc[n];
  out[nt] = su; out[nt + 1] = sv; out[nt + 2] = sw; out[nt + 3] = maxdiv; out[nt + 4] = cfl * dt; out[nt + 5] = bad;
}

/* ------------------------------------------------------------------ */
void orc_regrid(const double* zf_in, int nin, const double* in, const double* zf_out, int nout, double* out) {
  for (int j = 0; j < nout; ++j) {
    double lo = zf_out[j], hi = zf_out[j + 1], acc = 0.0;
    for (int i = 0; i < nin; ++i) {
      double a = zf_in[i] > lo ? zf_in[i] : lo;
      double b = zf_in[i + 1] < hi ? zf_in[i + 1] : hi;
      if (b > a) acc += in[i] * (b - a);
    }
    out[j] = acc / (hi - lo);
  }
}

/* ------------------------------------------------------------------ */
void orc_grid_metrics(const orc_model* M, double* zc, double* dzc, double* dzf) {
  memcpy(zc, M->zc, sizeof(double) * M->Nz);
  memcpy(dzc, M->dzc, sizeof(double) * M->Nz);
  memcpy(dzf, M->dzf, sizeof(double) * (M->Nz + 1));
}

size_t orc_field_len(const orc_model* M, int field) {
  size_t plane = (size_t)M->Nx * M->Ny;
  int f = field >= ORC_G ? field - ORC_G : field;
  return plane * (size_t)(f == ORC_W ? M->Nz + 1 : M->Nz);
}

static double* field_ptr(const orc_model* M, int field) {
  if (field == ORC_U) return M->u;
  if (field == ORC_V) return M->v;
  if (field == ORC_W) return M->w;
  if (field == ORC_P) return M->pr;
  if (field >= ORC_C0 && field < ORC_C0 + M->nt) return M->c[field - ORC_C0];
  if (field == ORC_G + ORC_U) return M->Gu;
  if (field == ORC_G + ORC_V) return M->Gv;
  if (field == ORC_G + ORC_W) return M->Gw;
  if (field >= ORC_G + ORC_C0 && field < ORC_G + ORC_C0 + M->nt) return M->Gc[field - ORC_G - ORC_C0];
  return NULL;
}

void orc_set(orc_model* M, int field, const double* src) {
  double* d = field_ptr(M, field);
  if (!d) return;
  M->ab_started = (field >= ORC_G) ? 1 : 0;   /* QAB2: a restored G^{m-1} continues the run */
  memcpy(d, src, sizeof(double) * orc_field_len(M, field));
  if (field == ORC_W) {   /* impenetrable walls */
    size_t plane = (size_t)M->Nx * M->Ny;
    memset(M->w, 0, plane * sizeof(double));
    memset(M->w + (size_t)M->Nz * plane, 0, plane * sizeof(double));
  }
}

void orc_get(const orc_model* M, int field, double* dst) {
  double* s = field_ptr(M, field);
  if (!s) return;
  memcpy(dst, s, sizeof(double) * orc_field_len(M, field));
}

orc_model* orc_create(const orc_params* p) {
  if (p->Nx < 1 || p->Ny < 1 || p->Nz < 1) return NULL;
  if ((p->nu_z || p->kappa_z) && p->Nz > 512) return NULL;       /* column buffers of the vertical solver */
  if (p->weno_order < 1 || p->weno_order > 2 * ORC_RMAX - 1 || (p->weno_order % 2) == 0) return NULL;
  if (p->n_tracers < 0 || p->n_tracers > ORC_MAX_TRACERS) return NULL;
  if (p->eos == ORC_EOS_LINEAR_TS && p->n_tracers < 2) return NULL;
  if (p->eos == ORC_EOS_BUOYANCY_TRACER && p->n_tracers < 1) return NULL;
  orc_model* M = (orc_model*)calloc(1, sizeof(orc_model));
  M->p = *p;
  M->Nx = p->Nx; M->Ny = p->Ny; M->Nz = p->Nz; M->nt = p->n_tracers;
  M->R = (p->weno_order + 1) / 2;
  M->P = M->R - 1 > 0 ? M->R - 1 : 1;       /* centered order N-1 (>= 2) for advecting velocities */
  M->dx = p->Lx / p->Nx; M->dy = p->Ly / p->Ny;
  int Nz = p->Nz;
  M->zf = (double*)malloc(sizeof(double) * (Nz + 1));
  M->zc = (double*)malloc(sizeof(double) * Nz);
  M->dzc = (double*)malloc(sizeof(double) * Nz);
  M->dzf = (double*)calloc(Nz + 1, sizeof(double));
  memcpy(M->zf, p->zf, sizeof(double) * (Nz + 1));
  M->p.zf = M->zf;
  for (int k = 0; k < Nz; ++k) { M->zc[k] = 0.5 * (M->zf[k] + M->zf[k + 1]); M->dzc[k] = M->zf[k + 1] - M->zf[k]; }
  for (int k = 1; k < Nz; ++k) M->dzf[k] = M->zc[k] - M->zc[k - 1];
  M->dzf[0] = M->dzc[0]; M->dzf[Nz] = M->dzc[Nz - 1];   /* unused: wall faces carry no gradient */
  size_t plane = (size_t)p->Nx * p->Ny, N = plane * Nz, NW = plane * (Nz + 1);
  M->u = (double*)calloc(N, sizeof(double)); M->v = (double*)calloc(N, sizeof(double)); M->w = (double*)calloc(NW, sizeof(double));
  M->Gu = (double*)calloc(N, sizeof(double)); M->Gv = (double*)calloc(N, sizeof(double)); M->Gw = (double*)calloc(NW, sizeof(double));
  M->Hu = (double*)calloc(N, sizeof(double)); M->Hv = (double*)calloc(N, sizeof(double)); M->Hw = (double*)calloc(NW, sizeof(double));
  M->pr = (double*)calloc(N, sizeof(double)); M->work = (double*)calloc(N, sizeof(double));
  M->nue = (double*)calloc(N, sizeof(double));
  for (int n = 0; n < M->nt; ++n) {
    M->c[n] = (double*)calloc(N, sizeof(double));
    M->Gc[n] = (double*)calloc(N, sizeof(double));
    M->Hc[n] = (double*)calloc(N, sizeof(double));
    M->kape[n] = (double*)calloc(N, sizeof(double));
  }
  if (p->nu_z) { M->nuz = (double*)malloc(sizeof(double) * (Nz + 1)); memcpy(M->nuz, p->nu_z, sizeof(double) * (Nz + 1)); }
  if (p->kappa_z) { M->kapz = (double*)malloc(sizeof(double) * (Nz + 1)); memcpy(M->kapz, p->kappa_z, sizeof(double) * (Nz + 1)); }
  M->p.nu_z = M->nuz; M->p.kappa_z = M->kapz;
#ifdef _OPENMP
  if (p->nthreads > 0) omp_set_num_threads(p->nthreads);
#endif
  return M;
}

void orc_destroy(orc_model* M) {
  if (!M) return;
  free(M->zf); free(M->zc); free(M->dzc); free(M->dzf);
  free(M->u); free(M->v); free(M->w); free(M->Gu); free(M->Gv); free(M->Gw);
  free(M->Hu); free(M->Hv); free(M->Hw); free(M->pr); free(M->work); free(M->nue); free(M->Fcol); free(M->nuz); free(M->kapz);
  for (int n = 0; n < M->nt; ++n) { free(M->c[n]); free(M->Gc[n]); free(M->Hc[n]); free(M->kape[n]); }
  free(M);
}

/* ================================================================== */
/* Learned column closure: features, closure fluxes, coarse-graining   */
/* and the face-flux hook.  Column quantities q = 0: b, 1: ubar (u at   */
/* the cell centre), 2: vbar; fluxes are upward through the w-faces of  */
/* the cell-centre columns.                                            */
static double ubar_c(const orc_model* M, int i, int j, int k) { return 0.5 * (A3(M, M->u, i, j, k) + A3(M, M->u, i + 1, j, k)); }
static double vbar_c(const orc_model* M, int i, int j, int k) { return 0.5 * (A3(M, M->v, i, j, k) + A3(M, M->v, i, j + 1, k)); }
static double colq(const orc_model* M, int q, int i, int j, int k) {
  return q == 0 ? buoyancy(M, i, j, k) : (q == 1 ? ubar_c(M, i, j, k) : vbar_c(M, i, j, k));
}
/* d q / dz across face k; zero outside the interior faces 1..Nz-1 */
static double colgrad(const orc_model* M, int q, int i, int j, int k) {
  if (k <= 0 || k >= M->Nz) return 0.0;
  return (colq(M, q, i, j, k) - colq(M, q, i, j, k - 1)) / M->dzf[k];
}

void orc_closure_features(orc_model* M, double N2_background, double* X) {
  int Nx = M->Nx, Ny = M->Ny, Nz = M->Nz;
  size_t plane = (size_t)Nx * Ny;
  double* h = (double*)calloc(plane, sizeof(double));
  if (N2_background > 0.0)
    for (int j = 0; j < Ny; ++j)
      for (int i = 0; i < Nx; ++i) {
        double acc = 0.0;
        for (int k = 1; k < Nz; ++k) {
          double deficit = 1.0 - colgrad(M, 0, i, j, k) / N2_background;
          if (deficit > 0.0) acc += deficit * M->dzf[k];
        }
        h[(size_t)j * Nx + i] = acc;
      }
#pragma omp parallel for collapse(2)
  for (int k = 0; k <= Nz; ++k)
    for (int j = 0; j < Ny; ++j)
      for (int i = 0; i < Nx; ++i) {
        double* x = X + (((size_t)k * Ny + j) * Nx + i) * ORC_NF;
        for (int n = 0; n < ORC_NF; ++n) x[n] = 0.0;
        for (int m = -2; m <= 2; ++m) {
          x[0 + m + 2] = colgrad(M, 0, i, j, k + m);
          x[5 + m + 2] = colgrad(M, 1, i, j, k + m);
          x[10 + m + 2] = colgrad(M, 2, i, j, k + m);
        }
        x[15] = M->p.top_flux[2];
        x[16] = M->p.f;
        x[17] = N2_background;
        x[18] = M->zf[Nz] - M->zf[k];
        x[19] = h[(size_t)j * Nx + i];
      }
  free(h);
}

/* closure (SGS) vertical flux of b, ubar, vbar at face k of column (i,j), 0 at the walls */
static double col_sgs_flux(const orc_model* M, int q, int i, int j, int k) {
  if (k <= 0 || k >= M->Nz) return 0.0;
  if (q == 0) {
    if (M->p.eos == ORC_EOS_LINEAR_TS) {
      double fT = -0.5 * (KAP(M, 0, i, j, k - 1) + KAP(M, 0, i, j, k)) * dcdz_ccf(M, M->c[0], i, j, k);
      double fS = -0.5 * (KAP(M, 1, i, j, k - 1) + KAP(M, 1, i, j, k)) * dcdz_ccf(M, M->c[1], i, j, k);
      if (M->p.closure == ORC_CLOSURE_SCALAR) { fT = -M->p.kappa * dcdz_ccf(M, M->c[0], i, j, k); fS = -M->p.kappa * dcdz_ccf(M, M->c[1], i, j, k); }
      if (M->p.closure == ORC_CLOSURE_NONE) return 0.0;
      return M->p.g * (M->p.alpha * fT - M->p.beta * fS);
    }
    if (M->p.closure == ORC_CLOSURE_SCALAR) return -M->p.kappa * colgrad(M, 0, i, j, k);
    if (M->p.closure == ORC_CLOSURE_NONE) return 0.0;
    return -0.5 * (KAP(M, 0, i, j, k - 1) + KAP(M, 0, i, j, k)) * colgrad(M, 0, i, j, k);
  }
  if (M->p.closure == ORC_CLOSURE_SCALAR) return -M->p.nu * colgrad(M, q, i, j, k);
  if (M->p.closure == ORC_CLOSURE_NONE) return 0.0;
  return -0.5 * (NU(M, i, j, k - 1) + NU(M, i, j, k)) * colgrad(M, q, i, j, k);
}

void orc_column_sgs_flux(orc_model* M, double* F) {
  int Nx = M->Nx, Ny = M->Ny, Nz = M->Nz;
  size_t plane = (size_t)Nx * Ny, NW = plane * (Nz + 1);
  compute_diffusivities(M);
#pragma omp parallel for collapse(2)
  for (int k = 0; k <= Nz; ++k)
    for (int j = 0; j < Ny; ++j)
      for (int i = 0; i < Nx; ++i)
        for (int q = 0; q < 3; ++q) F[q * NW + ((size_t)k * Ny + j) * Nx + i] = col_sgs_flux(M, q, i, j, k);
  M->have_diff = 0;
}

void orc_coarse_grain(orc_model* M, int cx, int cy, double* out) {
  int Nx = M->Nx, Ny = M->Ny, Nz = M->Nz;
  int rx = Nx / cx, ry = Ny / cy;
  size_t cp = (size_t)cx * cy;
  double* uc = out;
  double* vc = uc + (size_t)Nz * cp;
  double* wc = vc + (size_t)Nz * cp;
  double* bc = wc + (size_t)(Nz + 1) * cp;
  double* tau = bc + (size_t)Nz * cp;
  compute_diffusivities(M);
  double inv = 1.0 / ((double)rx * ry);
#pragma omp parallel for collapse(2)
  for (int k = 0; k <= Nz; ++k)
    for (int J = 0; J < cy; ++J)
      for (int I = 0; I < cx; ++I) {
        size_t cid = ((size_t)k * cy + J) * cx + I;
        double su = 0, sv = 0, sw = 0, sb = 0;
        double swq[3] = {0, 0, 0}, sq[3] = {0, 0, 0}, ssgs[3] = {0, 0, 0};
        for (int jj = 0; jj < ry; ++jj)
          for (int ii = 0; ii < rx; ++ii) {
            int i = I * rx + ii, j = J * ry + jj;
            double w = A3(M, M->w, i, j, k);
            sw += w;
            if (k < Nz) {
              sb += buoyancy(M, i, j, k);
              if (ii == 0) su += A3(M, M->u, i, j, k);      /* the coarse x-face coincides with fine face I*rx */
              if (jj == 0) sv += A3(M, M->v, i, j, k);
            }
            if (k > 0 && k < Nz)
              for (int q = 0; q < 3; ++q) {
                double qf = 0.5 * (colq(M, q, i, j, k - 1) + colq(M, q, i, j, k));
                swq[q] += w * qf;
                sq[q] += qf;
                ssgs[q] += col_sgs_flux(M, q, i, j, k);
              }
          }
        wc[cid] = sw * inv;
        if (k < Nz) {
          bc[cid] = sb * inv;
          uc[cid] = su / ry;
          vc[cid] = sv / rx;
        }
        for (int q = 0; q < 3; ++q) {
          double t = 0.0;
          if (k > 0 && k < Nz) t = swq[q] * inv - (sw * inv) * (sq[q] * inv) + ssgs[q] * inv;
          tau[(size_t)q * (Nz + 1) * cp + cid] = t;
        }
      }
  M->have_diff = 0;
}

void orc_set_face_flux(orc_model* M, orc_face_flux_fn fn, void* ctx) {
  M->flux_fn = fn;
  M->flux_ctx = ctx;
  if (fn && !M->Fcol) M->Fcol = (double*)calloc((size_t)3 * (M->Nz + 1) * M->Nx * M->Ny, sizeof(double));
}

void orc_set_face_diffusivity(orc_model* M, orc_face_flux_fn fn, void* ctx) {
  M->diff_fn = fn;
  M->diff_ctx = ctx;
  if (!fn) return;
  if (!M->Fcol) M->Fcol = (double*)calloc((size_t)3 * (M->Nz + 1) * M->Nx * M->Ny, sizeof(double));
  if (!M->nuz) M->nuz = (double*)calloc((size_t)M->Nz + 1, sizeof(double));
  if (!M->kapz) M->kapz = (double*)calloc((size_t)M->Nz + 1, sizeof(double));
  M->p.nu_z = M->nuz; M->p.kappa_z = M->kapz;
  M->p.vertical_implicit = 1;
}

/* kappa_z, nu_z <- the horizontal means of the hook's diffusivities at the interior faces. */
static void learned_profiles(orc_model* M) {
  int Nx = M->Nx, Ny = M->Ny, Nz = M->Nz;
  size_t plane = (size_t)Nx * Ny, NW = plane * (Nz + 1);
  M->diff_fn(M->diff_ctx, M, M->Fcol);
  for (int k = 0; k <= Nz; ++k) {
    double s0 = 0.0, s1 = 0.0;
    if (k > 0 && k < Nz)
      for (size_t c = 0; c < plane; ++c) { s0 += M->Fcol[(size_t)k * plane + c]; s1 += M->Fcol[NW + (size_t)k * plane + c]; }
    M->kapz[k] = s0 / (double)plane;
    M->nuz[k] = s1 / (double)plane;
  }
}

/* G_b -= dF_b/dz at centres; G_u, G_v -= dF/dz of the face flux averaged onto the u and v columns.
 * The flux through the wall faces (k = 0, Nz) is taken as zero whatever the hook wrote. */
static void add_face_flux_divergence(orc_model* M, double* Gu, double* Gv, double* Gb) {
  int Nx = M->Nx, Ny = M->Ny, Nz = M->Nz;
  size_t plane = (size_t)Nx * Ny, NW = plane * (Nz + 1);
  M->flux_fn(M->flux_ctx, M, M->Fcol);
  double* F = M->Fcol;
  for (int q = 0; q < 3; ++q) {
    memset(F + q * NW, 0, plane * sizeof(double));
    memset(F + q * NW + (size_t)Nz * plane, 0, plane * sizeof(double));
  }
  const double *Fb = F, *Fu = F + NW, *Fv = F + 2 * NW;
#pragma omp parallel for collapse(2)
  for (int k = 0; k < Nz; ++k)
    for (int j = 0; j < Ny; ++j)
      for (int i = 0; i < Nx; ++i) {
        size_t id = ID(M, i, j, k);
        double r = 1.0 / M->dzc[k];
        Gb[id] -= (A3(M, Fb, i, j, k + 1) - A3(M, Fb, i, j, k)) * r;
        double fu1 = 0.5 * (A3(M, Fu, i - 1, j, k + 1) + A3(M, Fu, i, j, k + 1));
        double fu0 = 0.5 * (A3(M, Fu, i - 1, j, k) + A3(M, Fu, i, j, k));
        Gu[id] -= (fu1 - fu0) * r;
        double fv1 = 0.5 * (A3(M, Fv, i, j - 1, k + 1) + A3(M, Fv, i, j, k + 1));
        double fv0 = 0.5 * (A3(M, Fv, i, j - 1, k) + A3(M, Fv, i, j, k));
        Gv[id] -= (fv1 - fv0) * r;
      }
}

/* ================================================================== */
/* Vertical diffusion with a z-profile of diffusivity (explicit term   */
/* or the semi-implicit step), Eqs. tracer-with-tendency,               */
/* tracer-time-discretization, predictor-velocity.                      */
void orc_vertical_diffusion(const orc_model* M, int stag, const double* kf, const double* q, double* out) {
  int Nz = M->Nz;
  if (stag == 0) {
    for (int k = 0; k < Nz; ++k) {
      double Fb = (k == 0) ? 0.0 : -kf[k] * (q[k] - q[k - 1]) / M->dzf[k];
      double Ft = (k == Nz - 1) ? 0.0 : -kf[k + 1] * (q[k + 1] - q[k]) / M->dzf[k + 1];
      out[k] = -(Ft - Fb) / M->dzc[k];
    }
  } else {
    out[0] = 0.0; out[Nz] = 0.0;
    for (int k = 1; k < Nz; ++k) {
      double kb = 0.5 * (kf[k - 1] + kf[k]), kt = 0.5 * (kf[k] + kf[k + 1]);
      double Fb = -kb * (q[k] - q[k - 1]) / M->dzc[k - 1];
      double Ft = -kt * (q[k + 1] - q[k]) / M->dzc[k];
      out[k] = -(Ft - Fb) / M->dzf[k];
    }
  }
}

/* (I - dtau D) q = rhs by the Thomas algorithm; for face-staggered q the walls stay 0. */
void orc_vertical_implicit_solve(const orc_model* M, int stag, const double* kf, double dtau, const double* rhs, double* q) {
  int Nz = M->Nz;
  int n0 = (stag == 0) ? 0 : 1, n1 = (stag == 0) ? Nz - 1 : Nz - 1;   /* unknowns n0..n1 */
  int n = n1 - n0 + 1;
  double* a = (double*)calloc(n, sizeof(double));
  double* b = (double*)calloc(n, sizeof(double));
  double* c = (double*)calloc(n, sizeof(double));
  double* d = (double*)calloc(n, sizeof(double));
  for (int r = 0; r < n; ++r) {
    int k = n0 + r;
    double lo = 0.0, hi = 0.0, h;
    if (stag == 0) {
      h = M->dzc[k];
      if (k > 0) lo = kf[k] / M->dzf[k];
      if (k < Nz - 1) hi = kf[k + 1] / M->dzf[k + 1];
    } else {
      h = M->dzf[k];
      lo = 0.5 * (kf[k - 1] + kf[k]) / M->dzc[k - 1];
      hi = 0.5 * (kf[k] + kf[k + 1]) / M->dzc[k];
    }
    /* row: -dtau lo/h q_{k-1} + (1 + dtau (lo + hi)/h) q_k - dtau hi/h q_{k+1} = rhs_k */
    a[r] = (r > 0) ? -dtau * lo / h : 0.0;
    c[r] = (r < n - 1) ? -dtau * hi / h : 0.0;
    b[r] = 1.0 + dtau * (lo + hi) / h;
    d[r] = rhs[k];
  }
  for (int r = 1; r < n; ++r) {
    double w = a[r] / b[r - 1];
    b[r] -= w * c[r - 1];
    d[r] -= w * d[r - 1];
  }
  double* x = (double*)calloc(n, sizeof(double));
  x[n - 1] = d[n - 1] / b[n - 1];
  for (int r = n - 2; r >= 0; --r) x[r] = (d[r] - c[r] * x[r + 1]) / b[r];
  if (stag == 1) { q[0] = 0.0; q[Nz] = 0.0; }
  for (int r = 0; r < n; ++r) q[n0 + r] = x[r];
  free(a); free(b); free(c); free(d); free(x);
}

/* Gather a column (stride plane), apply f, scatter back. */
static void column_apply_explicit(const orc_model* M, int stag, const double* kf, double* f, double* G) {
  int Nx = M->Nx, Ny = M->Ny, Nz = M->Nz, L = Nz + stag;
  size_t plane = (size_t)Nx * Ny;
#pragma omp parallel for collapse(2)
  for (int j = 0; j < Ny; ++j)
    for (int i = 0; i < Nx; ++i) {
      double q[512 + 2], o[512 + 2];
      size_t c0 = (size_t)j * Nx + i;
      for (int k = 0; k < L; ++k) q[k] = f[c0 + k * plane];
      orc_vertical_diffusion(M, stag, kf, q, o);
      for (int k = 0; k < L; ++k) G[c0 + k * plane] += o[k];
    }
}

static void add_vertical_diffusion(orc_model* M, double* Gu, double* Gv, double* Gw, double** Gc) {
  if (M->nuz) {
    column_apply_explicit(M, 0, M->nuz, M->u, Gu);
    column_apply_explicit(M, 0, M->nuz, M->v, Gv);
    column_apply_explicit(M, 1, M->nuz, M->w, Gw);
  }
  if (M->kapz)
    for (int t = 0; t < M->nt; ++t) column_apply_explicit(M, 0, M->kapz, M->c[t], Gc[t]);
}

static void column_solve(const orc_model* M, int stag, const double* kf, double dtau, double* f) {
  int Nx = M->Nx, Ny = M->Ny, Nz = M->Nz, L = Nz + stag;
  size_t plane = (size_t)Nx * Ny;
#pragma omp parallel for collapse(2)
  for (int j = 0; j < Ny; ++j)
    for (int i = 0; i < Nx; ++i) {
      double r[512 + 2], q[512 + 2];
      size_t c0 = (size_t)j * Nx + i;
      for (int k = 0; k < L; ++k) r[k] = f[c0 + k * plane];
      orc_vertical_implicit_solve(M, stag, kf, dtau, r, q);
      for (int k = 0; k < L; ++k) f[c0 + k * plane] = q[k];
    }
}

static void implicit_vertical_step(orc_model* M, double dtau) {
  if (M->nuz) {
    column_solve(M, 0, M->nuz, dtau, M->u);
    column_solve(M, 0, M->nuz, dtau, M->v);
    column_solve(M, 1, M->nuz, dtau, M->w);
  }
  if (M->kapz)
    for (int t = 0; t < M->nt; ++t) column_solve(M, 0, M->kapz, dtau, M->c[t]);
}
