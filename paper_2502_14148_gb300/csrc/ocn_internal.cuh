// Internal declarations shared by the translation units of the CUDA library.
// Nothing here is part of the public ABI (include/ocn.h).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/ocn.h"

namespace ocn {

constexpr int kMaxTracers = OCN_MAX_TRACERS;
constexpr int kMaxR = 5;          // WENO order up to 9
constexpr int kMaxFftPasses = 12;

// Reconstruction tables in the kernel's precision (uploaded to __constant__).
template <typename T>
struct WenoTables {
  T sub[kMaxR + 1][kMaxR][kMaxR];          // [r][s][n]: substencil s of WENO(2r-1), weight of cell -r+s+n
  T d[kMaxR + 1][kMaxR];                   // linear weights
  T beta[kMaxR + 1][kMaxR][kMaxR][kMaxR];  // symmetric smoothness forms
  T cen[kMaxR + 1][2 * kMaxR];             // centered order 2p: weight of cell -p+n
  // Difference form used by the kernels (d_m = t_{m+1} - t_m in the upwind frame, m = 0..2r-3):
  T gq[kMaxR + 1][kMaxR][kMaxR - 1];       // q_s - t_{r-1} = sum_a gq[r][s][a] d_{s+a}
  T dbeta[kMaxR + 1][kMaxR][kMaxR - 1][kMaxR - 1];  // beta_s = sum_ab dbeta[r][s][a][b] d_{s+a} d_{s+b}
};

// Host-side derivation of the tables (coeffs.cpp).
void derive_weno_tables(WenoTables<double>* out);
// Upload to the constant memory of every tendency translation unit.
cudaError_t upload_weno_tables(const WenoTables<double>& t);
cudaError_t upload_tables_f64(const WenoTables<double>& t);
cudaError_t upload_tables_f64_batch(const WenoTables<double>& t);

// Fields of one prognostic state.
template <typename T>
struct StatePtrs {
  T* u;
  T* v;
  T* w;
  T* c[kMaxTracers];
};

// Bounds-checked builds (every translation unit compiled with -DOCN_BOUNDS_CHECK=1: the library
// variant libocn_checked.so, for tests).  The tendency kernel, the projection FFTs and the
// tridiagonal solve check their indices; one outside its array sets a bit of the model's status
// word (the code below) and is replaced by 0, so the access stays inside the array and nothing
// traps.  In the normal build a check is the index itself and costs nothing.
enum : unsigned {
  kOobPlane = 1u,        // a thread's stencil window or a ring point outside the staged plane
  kOobGather = 2u,       // a staged plane's source element or level outside its field
  kOobFlux = 4u,         // a face-flux slot outside the flux planes
  kOobGlobal = 8u,       // a state, tendency or eddy-viscosity element outside its field
  kOobFftShared = 16u,   // an FFT pass element outside its shared buffer
  kOobFftGlobal = 32u,   // a spectrum, velocity or pressure element outside its array
  kOobTridiag = 64u      // a tridiagonal unknown or factor outside the spectrum
};
#ifndef OCN_BOUNDS_CHECK
#define OCN_BOUNDS_CHECK 0
#endif
#ifdef __CUDACC__
__device__ __forceinline__ long long oob_index(long long i, long long n, unsigned* st, unsigned code) {
  if (i < 0 || i >= n) {
    if (st) atomicOr(st, code);
    return 0;
  }
  return i;
}
#endif
#if OCN_BOUNDS_CHECK
#define OCN_CHK(i, n, st, code) ((decltype((i) + 0))::ocn::oob_index((long long)(i), (long long)(n), (st), (code)))
#else
#define OCN_CHK(i, n, st, code) (i)
#endif

template <typename T>
struct TendencyArgs {
  StatePtrs<T> cur;       // state at the start of the substage (read)
  StatePtrs<T> nxt;       // new state (u~, tracers at m+1) (written)
  StatePtrs<T> G;         // G^{m-1} (read when zeta != 0), overwritten with G^m
  const T* nu;            // eddy viscosity at centres (closure SMAG/AMD)
  const T* kap[kMaxTracers];  // AMD tracer diffusivities
  const T* rdzc;          // 1/dz_c[k], k < Nz
  const T* rdzf;          // 1/dz_f[k], 1 <= k < Nz (entries 0, Nz unused)
  const T* dzf;           // dz_f[k]
  int Nx, Ny, Nz, nt;
  T rdx, rdy;
  const T* cref[kMaxTracers];  // per-level reference profiles: tracer n is stored as c - cref[n][k] (or null)
  int closure;
  T nu0, kappa0;          // scalar diffusivity
  T inv_Pr;
  T f;
  int eos;
  T g_alpha, g_beta, T0, S0;
  T top[2 + kMaxTracers], bot[2 + kMaxTracers];
  T dt_gamma, dt_zeta;    // RK coefficients times dt
  int mode;               // 0: RK update + G;  1: G only
  int variant;            // tile variant of the FP32 kernel (0: 32x8 one CTA/SM, 1: 32x8 two, 2: 32x16, 3: 32x4 three,
                          // 4: 32x14, 5: 32x12, 6: 16x16 two CTAs/SM for grids under 32 columns wide)
  // FP32 Smagorinsky-Lilly and AMD kernels compute the eddy diffusivities of the stage state
  // themselves (in the same z march, from the staged planes) and write nu_e here for other readers;
  // nu and kap above are unused then.
  T* nu_out;
  const T* dzc;           // dz_c[k]
  T dx, dy, Cs, Cb, C_amd;  // grid spacing, Smagorinsky, stratification and AMD constants
  unsigned* oob;          // status word of the bounds-checked build (or null)
};

template <typename T>
struct ClosureArgs {
  StatePtrs<T> cur;
  const T* cref[kMaxTracers];  // per-level tracer reference profiles (or null)
  T* nu;
  T* kap[kMaxTracers];
  const T* dzc;
  const T* rdzc;
  const T* rdzf;
  int Nx, Ny, Nz, nt;
  T dx, dy, rdx, rdy;
  int closure;
  T Cs, Cb, inv_Pr, C_amd;
  int eos;
  T g_alpha, g_beta, T0, S0;
};

// FFT plan for one line length (the half length for the real transform in x).
struct FftPlan {
  int n;                       // line length
  int npass;
  int radix[kMaxFftPasses];
};

template <typename T>
struct PoissonArgs {
  T* u; T* v; T* w;            // velocity to project (in place)
  T* p;                        // pressure out
  T* spec;                     // complex [Nz][Ny][Sp] interleaved (re, im); kx = 0 .. Nx/2 used
  T* cpiv;                     // Thomas pivots c' [Nz][Ny][Sp]
  T* pinv;                     // 1 / Thomas diagonal [Nz][Ny][Sp] when stored (else null: computed per solve)
  const T* rdzc; const T* rdzf; const T* dzc;
  const T* lamx;               // [Nx/2+1]
  const T* lamy;               // [Ny]
  const T* twx;                // e^{-2 pi i t/Nx}, t < Nx (complex interleaved)
  const T* twy;                // e^{-2 pi i t/Ny}, t < Ny
  int Nx, Ny, Nz, Mx;          // Mx = Nx/2
  int Sp;                      // row stride of the spectrum and pivots (>= Mx + 1)
  T rdx, rdy;
  T inv_dt;                    // 1 / (stage dt)
  T dt;                        // stage dt
  T scale;                     // 1 / (Mx * Ny) for the inverse transforms
  T Htot;                      // total depth (for the gauge mean)
  int fp64_pivots;
  FftPlan px, py;
  unsigned* oob;               // status word of the bounds-checked build (or null)
};

// Row stride of a model's spectrum: Nx/2 + 1 rounded up to a multiple of 8 complex values, so
// that every row, and every tile of 4 or 8 kx columns that the y transform moves, starts on a
// 32-byte sector (an odd stride would split most of the y transform's 32-byte row pieces over two
// sectors).
inline int spec_row_stride(int Mx) { return (Mx + 1 + 7) / 8 * 8; }

template <typename T>
struct DiagArgs {
  StatePtrs<T> cur;
  const T* dzc; const T* dzf; const T* rdzc; const T* rdzf;
  int Nx, Ny, Nz, nt;
  T dx, dy, rdx, rdy;
  double* partial;             // [nblocks][nvals]
  double* out;                 // [nvals]
  int nblocks;
};

// Optional per-launch hook (kernel timing): called around every kernel launch.
struct LaunchHook {
  void (*before)(void* ctx, int kclass) = nullptr;
  void (*after)(void* ctx, int kclass) = nullptr;
  void* ctx = nullptr;
  void pre(int k) const { if (before) before(ctx, k); }
  void post(int k) const { if (after) after(ctx, k); }
};

// Launchers (return the launch error; kernels are enqueued on `s`).
template <typename T> cudaError_t launch_closure(const ClosureArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_tendency(const TendencyArgs<T>& a, int weno_r, cudaStream_t s);
template <> cudaError_t launch_tendency<float>(const TendencyArgs<float>& a, int weno_r, cudaStream_t s);
template <> cudaError_t launch_tendency<double>(const TendencyArgs<double>& a, int weno_r, cudaStream_t s);
cudaError_t launch_tendency_f32_r5(const TendencyArgs<float>& a, cudaStream_t s);
cudaError_t launch_tendency_f32_r3(const TendencyArgs<float>& a, cudaStream_t s);
constexpr int kTendencyVariants = 7;
template <typename T> cudaError_t launch_projection(const PoissonArgs<T>& a, cudaStream_t s, int* nlaunch,
                                                    const LaunchHook& hook = LaunchHook());
template <typename T> cudaError_t launch_diagnostics(const DiagArgs<T>& a, cudaStream_t s);
// Factor the projection's tridiagonal systems once (they depend only on the grid): fills a.cpiv
// and a.pinv, the pivots computed in FP64 when a.fp64_pivots.
template <typename T> cudaError_t launch_tridiag_factor(const PoissonArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_fill(T* p, size_t n, T v, cudaStream_t s);
template <typename T> cudaError_t launch_shift(T* p, size_t n, T v, cudaStream_t s);
// Per-level horizontal means (FP64) used by the coarse-graining profiles:
// out[0..Nz) <G_u>, [Nz..2Nz) <G_v>, [2Nz..3Nz) <G_c0>, [3Nz..4Nz) <G_c1>, [4Nz..5Nz) <u>, [5Nz..6Nz) <v>,
// [6Nz..7Nz) <b> (tracers stored about reference profiles; b from the EOS).
template <typename T>
struct ProfileArgs {
  const T* Gu; const T* Gv; const T* Gc0; const T* Gc1;
  const T* u; const T* v; const T* c0; const T* c1;
  const T* cref0; const T* cref1;
  size_t plane;
  int Nz, eos;
  double g_alpha, g_beta, T0, S0;
  double* out;
};
template <typename T> cudaError_t launch_profile_means(const ProfileArgs<T>& a, cudaStream_t s);
// Per-level horizontal means of a [Nz][plane] field (FP64 accumulation) into ref[Nz],
// and p[k][.] += sign * ref[k].
template <typename T> cudaError_t launch_level_mean(const T* p, size_t plane, int Nz, T* ref, cudaStream_t s);
template <typename T> cudaError_t launch_level_shift(T* p, size_t plane, int Nz, const T* ref, T sign, cudaStream_t s);
template <typename T> cudaError_t launch_level_add(T* dst, const T* src, size_t plane, int Nz, const T* ref, cudaStream_t s);
int diag_blocks();
// Raise a kernel's dynamic shared memory limit to at least `bytes` on the current device (never
// lowers it: graphs captured earlier may launch the kernel with more).
cudaError_t raise_smem_limit(const void* fn, size_t bytes);
template <typename F>
cudaError_t raise_smem_limit(F* fn, size_t bytes) { return raise_smem_limit(reinterpret_cast<const void*>(fn), bytes); }
// Records the text returned by ocn_last_error() on this thread and returns s.
ocn_status set_last_error(ocn_status s, const char* msg);

// Vertical diffusion with diffusivity profiles at the w-faces (vertical.cu): fields f = 0 u, 1 v,
// 2 w, 3 + n tracer n; bit f of `fields` selects them.  Explicit: G += D(qin), mode 0 also
// qout += dt_gamma D(qin).  Implicit: qout <- (I - dtau D)^{-1} qout in place.
template <typename T>
struct VDiffArgs {
  const T* qin[3 + kMaxTracers];
  T* qout[3 + kMaxTracers];
  T* G[3 + kMaxTracers];
  const T* cref[kMaxTracers];
  const T* nuz; const T* kapz;             // [Nz+1]
  const T* dzc; const T* dzf;              // dz_c [Nz], dz_f [Nz+1] (interior faces 1..Nz-1)
  int Nx, Ny, Nz, nt;
  int fields;
  int mode;
  T dt_gamma, dtau;
  // work space of the segmented implicit solve ((3 + nt) (4 Nz + 16) values, written by its factor
  // kernel and read by its solve kernel of the same call; nothing is kept between calls) and its
  // capacity in elements; 0 selects the one-thread-per-column solve
  T* tab;
  size_t tab_cap;
  int seg;                                 // rows per segment of the segmented solve (set by the launcher)
};
// Enqueues the vertical diffusion kernels; *nlaunch (if not null) is increased by the number of
// kernels launched or recorded.
template <typename T>
cudaError_t launch_vertical_diffusion(const VDiffArgs<T>& a, bool implicit, cudaStream_t s, int* nlaunch);

// Tensor-core GEMM of the learned column closure (mlp.cu):  D = A . B^T with A [M][K] and
// B [N][K] BF16 (K contiguous, lda/ldb multiples of 8 elements, 16-byte aligned bases),
// FP32 accumulation, 16 <= N <= 256 (multiple of 16), K a multiple of 8.  Split-K over
// gridDim.y: split y covers K range [y*kchunk, (y+1)*kchunk) (kchunk a multiple of 64).
// Epilogue (row r, column c, x = accumulated value):
//   mode 0: D[(y*M + r)*ldd + c] = x                        (split-K partials)
//   mode 1: z = x + bias[c]; D[r*ldd+c] = z (if D); H[r*ldh+c] = bf16(gelu(z));
//           HT[c*ldht+r] = bf16(gelu(z)) (if HT)
//   mode 2: D[r*ldd+c] = x + bias[c]
//   mode 3: g = x * gelu'(Z[r*ldz+c]); D[r*ldd+c] = g (if D); H, HT as mode 1 with g
// status (if not null) is set to 1 when a bounded wait for the tensor cores gave up.
struct GemmArgs {
  const void* A; int lda;
  const void* B; int ldb;
  int M, N, K, kchunk;
  int mode;
  float* D; int ldd;
  const float* bias;
  void* H; int ldh;
  void* HT; int ldht;
  const float* Z; int ldz;
  int* status;
  int no_issue;                    // test of the timeout path: stage, but issue no MMA and no commit
};
cudaError_t launch_gemm_tc(const GemmArgs& a, int nsplit, cudaStream_t s);

// ---- learned column closure (column.cu, mlp.cu); FP32 buoyancy-tracer models.
// Column quantities: b (stored anomaly + reference profile), ubar = (u_i + u_{i+1})/2,
// vbar = (v_j + v_{j+1})/2 at centres; fluxes live on the w-faces of the centre columns,
// arrays [3][Nz+1][Ny][Nx] (b, ubar, vbar).
constexpr int kColumnFeatures = 32;       // padded feature vector (20 used)
struct ColumnArgs {
  const float* b; const float* cref;      // tracer 0 anomaly and its reference profile (or null)
  const float* u; const float* v; const float* w;
  const float* rdzf;                      // [Nz+1], 0 at the walls
  const float* rdzc;                      // [Nz]
  const float* dzf;                       // [Nz+1]
  const float* depth;                     // [Nz+1]: zf[Nz] - zf[k]
  const float* nu; const float* kap;      // eddy viscosity / tracer-0 diffusivity at centres (or null)
  int closure; float nu0, kappa0, inv_Pr;
  int Nx, Ny, Nz;
  float Jb, f, N2bg;                      // surface buoyancy flux, Coriolis, background N^2
  float* h;                               // [Ny][Nx] mixed-layer depth estimate
};
cudaError_t launch_column_h(const ColumnArgs& a, cudaStream_t s);
cudaError_t launch_closure_features(const ColumnArgs& a, float* X, cudaStream_t s);
cudaError_t launch_column_sgs_flux(const ColumnArgs& a, float* F, cudaStream_t s);
cudaError_t launch_coarse_grain(const ColumnArgs& a, int cx, int cy, double* out, cudaStream_t s);
// G += dG and (mode 0) nxt += dt_gamma dG for dG = -dF/dz of the face fluxes (u, v: averaged onto their columns)
struct FaceFluxArgs {
  const float* F;
  float* Gu; float* Gv; float* Gb;
  float* nu_; float* nv; float* nb;
  const float* rdzc;
  int Nx, Ny, Nz, mode;
  float dt_gamma;
};
cudaError_t launch_apply_face_flux(const FaceFluxArgs& a, cudaStream_t s);
struct MlpClosureArgs {
  ColumnArgs col;
  const void* W[4]; const float* bias[4];  // BF16 weights [n_out][n_in], FP32 biases (32-128-128-128-16)
  float mu[kColumnFeatures], inv_sigma[kColumnFeatures];
  int relu;                                // 1: outputs are diffusivities, max(0, scale * y)
  float scale[3];
  float* F;                                // [3][Nz+1][Ny][Nx]
  int* status;                             // set to 1 if a bounded wait gave up
};
cudaError_t launch_mlp_closure(const MlpClosureArgs& a, cudaStream_t s);
// Horizontal means of face quantities 0 and 1 of F ([3][Nz+1][Ny][Nx]) per face, into p0 and p1
// ([Nz+1]; 0 at the walls): the learned diffusivities' column-mean profiles.
struct FaceMeanArgs {
  const float* F;
  float* p0; float* p1;
  int Nx, Ny, Nz;
};
cudaError_t launch_face_mean(const FaceMeanArgs& a, cudaStream_t s);
// Layer pointers of a network (mlp.cu): returns false unless its shape is 32-128-128-128-16.
bool mlp_closure_layers(const ocn_mlp* n, const void** W, const float** bias);

}  // namespace ocn
