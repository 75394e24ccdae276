/*
 * ocn.h -- C ABI of the GB300 (sm_103a) nonhydrostatic Boussinesq RK3 substep.
 *
 * The library advances the incompressible Boussinesq equations on a staggered
 * C-grid (arXiv 2502.14148):
 *   momentum   Sec. 3.1.1, Eq. nonhydrotatic-momentum-equations, in flux form
 *              (Eq. flux-form-advection), without Stokes drift, background
 *              fields or user forcing;
 *   tracers    Sec. 3.1.2, Eq. nonhydrostatic-tracer-equation (advection +
 *              closure + boundary fluxes);
 *   time       low-storage RK3, Appendix A.1 Eq. rk3;
 *   pressure   fractional step, Appendix A.2, Eqs. predictor-velocity,
 *              pressure-correction and pressure-poisson, solved by an FFT in
 *              x and y and a tridiagonal solve in z (the eigenfunction
 *              expansion of the discrete Laplacian described there);
 *   space      finite volumes, Appendix B: Eq. flux-divergence, WENO
 *              reconstruction (Eq. fifth-order-weno generalised to order
 *              2r-1 with WENO-Z weights), centered advecting velocities for
 *              momentum (Sec. B.2.1).
 *
 * Grid: x and y periodic and uniform, z bounded (impenetrable, free-slip,
 * no-flux walls unless a boundary flux is given) with arbitrary ascending face
 * heights.  Face index i is left of cell index i (Appendix B.1).
 *
 * Layout of every field in device or host memory: x fastest, then y, then z.
 *   u (Face,Center,Center), v (Center,Face,Center), tracers, p: [Nz][Ny][Nx]
 *   w (Center,Center,Face): [Nz+1][Ny][Nx]; w[0] and w[Nz] (the walls) are 0.
 * Element type: float when the model precision is 32, double when it is 64.
 *
 * Ownership: the library never allocates device memory.  The caller obtains
 * the size of the model's device arena with ocn_model_arena_bytes(), allocates
 * it (for example as a PyTorch tensor), and binds it with
 * ocn_model_bind_arena() before any other call that touches fields.  The
 * arena must stay valid until ocn_model_destroy(); the library never frees it.
 * Host buffers passed to ocn_set_field/ocn_get_field are read or written
 * during the call only (pinned host memory gives the fastest copies).
 *
 * Streams: all work of a model is issued on the cudaStream_t given at
 * creation (NULL selects the legacy default stream; graph capture of the time
 * step then stays off).  Calls return after enqueueing, except
 * ocn_set_field from host memory (which waits for its copy), ocn_get_field to
 * host memory (which waits for the data) and ocn_diagnostics, which
 * synchronises the stream.
 *
 * Errors: every call returns an ocn_status.  OCN_OK is 0; failures are
 * negative.  ocn_last_error() returns a thread-local description of the last
 * failure on the calling thread.  Nothing aborts, traps or exits.
 */
#ifndef OCN_H
#define OCN_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OCN_ABI_VERSION 2
#define OCN_MAX_TRACERS 4

typedef enum {
  OCN_OK = 0,
  OCN_ERR_ARG = -1,          /* invalid argument (null pointer, size mismatch, unknown id) */
  OCN_ERR_CUDA = -2,         /* a CUDA runtime call or kernel launch failed */
  OCN_ERR_OOM = -3,          /* host allocation failed */
  OCN_ERR_NONFINITE = -4,    /* diagnostics found a NaN or Inf */
  OCN_ERR_CFL = -5,          /* diagnostics found an advective CFL number above 1 */
  OCN_ERR_TIMEOUT = -6,      /* a bounded device-side wait gave up */
  OCN_ERR_UNSUPPORTED = -7,  /* valid but not built (e.g. a WENO order without a kernel) */
  OCN_ERR_STATE = -8         /* call order violated (e.g. arena not bound) */
} ocn_status;

enum { OCN_CLOSURE_NONE = 0, OCN_CLOSURE_SCALAR = 1, OCN_CLOSURE_SMAGORINSKY = 2, OCN_CLOSURE_AMD = 3 };
enum { OCN_EOS_BUOYANCY_TRACER = 0, OCN_EOS_LINEAR_TS = 1 };

/* Field ids for ocn_set_field / ocn_get_field. */
enum {
  OCN_FIELD_U = 0, OCN_FIELD_V = 1, OCN_FIELD_W = 2,
  OCN_FIELD_TRACER0 = 3,     /* tracer n is OCN_FIELD_TRACER0 + n */
  OCN_FIELD_P = 10,          /* pressure of the last projection, zero volume mean: after ocn_project the
                                kinematic pressure; after ocn_time_step the nonhydrostatic part p_nh of the
                                last substage (Eq. pressure-decomposition), scaled by 1/((gamma-zeta) dt) */
  OCN_FIELD_G = 20,          /* tendency G of field f is OCN_FIELD_G + f (G^{m-1} after a step) */
  OCN_FIELD_NU_E = 30,       /* eddy viscosity at cell centres (Smagorinsky-Lilly, AMD) */
  OCN_FIELD_TRACER_REF0 = 40, /* reference profile of tracer n ([Nz] values) is OCN_FIELD_TRACER_REF0 + n */
  OCN_FIELD_RAW = 0x100      /* OR'ed with a tracer id: the stored anomaly c - ref[k] itself */
};
/* Tracers are stored as anomalies about a per-level reference profile.  Setting
 * a tracer (without OCN_FIELD_RAW) makes its reference the horizontal mean of
 * each level and stores the anomaly; getting it returns anomaly + reference.
 * For a bitwise checkpoint, save u, v, w, every tracer with OCN_FIELD_RAW and
 * every OCN_FIELD_TRACER_REF0 + n; restore the same fields (setting a raw
 * tracer or a reference profile copies it as is). */

/* Grid (paper listing "RectilinearGrid(...)"): x in [0,Lx), y in [0,Ly) periodic,
 * uniform; z bounded with Nz+1 ascending face heights. */
typedef struct {
  int Nx, Ny, Nz;            /* Nx, Ny even and of the form 2^a 3^b, >= 4, Nx*Ny < 2^31; Nz >= 1 */
  double Lx, Ly;             /* > 0 */
  const double* z_faces;     /* Nz+1 strictly ascending heights; copied by ocn_grid_create */
} ocn_grid_desc;

/* Model (paper listing "NonhydrostaticModel(; grid, advection, closure, coriolis,
 * buoyancy, tracers, boundary_conditions)"). */
typedef struct {
  int precision;             /* 32 (FP32 state and tendencies) or 64 (FP64) */
  int weno_order;            /* 5 or 9; momentum advecting velocities use centered order weno_order-1 */
  int closure;               /* OCN_CLOSURE_* */
  double nu, kappa;          /* ScalarDiffusivity: constant viscosity and tracer diffusivity */
  double Cs, Cb, Pr;         /* Smagorinsky-Lilly: nu_e = (Cs D)^2 |S| sqrt(max(0, 1 - Cb N^2/(Pr |S|^2))), kappa_e = nu_e/Pr */
  double C_amd;              /* AMD Poincare constant (1/12 for second-order differences) */
  double f;                  /* FPlane Coriolis parameter */
  int n_tracers;             /* 1..OCN_MAX_TRACERS */
  int eos;                   /* OCN_EOS_BUOYANCY_TRACER: tracer 0 is b.  OCN_EOS_LINEAR_TS: tracers 0,1 are T,S */
  double g, alpha, beta, T0, S0;   /* linear EOS: b = g (alpha (T - T0) - beta (S - S0)) */
  double top_flux[2 + OCN_MAX_TRACERS];     /* upward flux of u, v, tracer 0.. through the top face */
  double bottom_flux[2 + OCN_MAX_TRACERS];  /* upward flux of u, v, tracer 0.. through the bottom face */
  int fp64_pivots;           /* tridiagonal pivots in FP64: 1 yes, 0 no, -1 when the z-grid is stretched */
} ocn_model_desc;

typedef struct ocn_grid ocn_grid;
typedef struct ocn_model ocn_model;

/* ABI version the library was built with (OCN_ABI_VERSION). */
int ocn_abi_version(void);

/* Thread-local text of the last failure ("" if none). Owned by the library. */
const char* ocn_last_error(void);

/* Create a grid from *desc.  *out receives a new handle (free with ocn_grid_destroy).
 * Errors: OCN_ERR_ARG for a null pointer, a size that is not even 2^a 3^b >= 4, a level of
 * 2^31 cells or more, non-positive lengths or non-ascending faces; OCN_ERR_OOM. */
ocn_status ocn_grid_create(const ocn_grid_desc* desc, ocn_grid** out);
void ocn_grid_destroy(ocn_grid* grid);

/* Create a model on a grid (the grid must outlive the model).  stream is a
 * cudaStream_t (NULL: legacy default stream).  Selects the CUDA device that is
 * current on the calling thread.
 * Errors: OCN_ERR_ARG (bad precision, tracer count, closure, eos),
 * OCN_ERR_UNSUPPORTED (weno_order other than 5 or 9), OCN_ERR_CUDA, OCN_ERR_OOM. */
ocn_status ocn_model_create(const ocn_grid* grid, const ocn_model_desc* desc, void* stream, ocn_model** out);
void ocn_model_destroy(ocn_model* model);

/* Bytes of device memory the model needs (state, tendencies, pressure,
 * diffusivities, spectral work space, metrics). */
ocn_status ocn_model_arena_bytes(const ocn_model* model, size_t* bytes);

/* Bind caller-owned device memory of at least ocn_model_arena_bytes() bytes,
 * 256-byte aligned.  Uploads the grid metrics and clears all fields to 0.
 * Errors: OCN_ERR_ARG (null, too small, misaligned), OCN_ERR_CUDA. */
ocn_status ocn_model_bind_arena(ocn_model* model, void* device_ptr, size_t bytes);

/* Copy a field in (set) or out (get).  nbytes must equal the field's size in
 * the model precision.  src/dst is device memory when *_is_device is 1, host
 * memory when it is 0 (the call waits for its copies) or OCN_HOST_ASYNC (below:
 * it does not).  Setting w forces w = 0 on the wall faces.  Setting a
 * field does not project the velocity (call ocn_project).
 * ocn_set_field from host memory returns once the host buffer has been copied;
 * the rest of its work (for a tracer, the new reference profile and the
 * anomaly) stays queued on the model stream.  ocn_get_field runs its copy (and,
 * for a tracer, the kernel that adds the reference profile back) on an
 * internal stream of the greatest priority, after the work queued on the model
 * stream and before the model stream's later work, so that it does not wait
 * behind the blocks of other work sharing the GPU; to host memory it returns
 * when the data has arrived.
 * Errors: OCN_ERR_ARG (also for *_is_device other than 0, 1, OCN_HOST_ASYNC),
 * OCN_ERR_STATE (no arena), OCN_ERR_CUDA. */
ocn_status ocn_set_field(ocn_model* model, int field, const void* src, size_t nbytes, int src_is_device);
ocn_status ocn_get_field(ocn_model* model, int field, void* dst, size_t nbytes, int dst_is_device);

/* *_is_device = OCN_HOST_ASYNC: host memory, and the call returns after
 * enqueueing instead of waiting for its copies.  The caller keeps the host
 * buffers valid (and, for a set, unchanged) until ocn_wait_transfers() has
 * returned; the model stream's later work is ordered after the copies as for the
 * waiting form.  Pinned host memory is needed for the copies to run
 * asynchronously.  This lets a caller overlap a model's copies with its own or
 * another model's steps and with copies in the other direction. */
#define OCN_HOST_ASYNC 2
/* Bounds checks (a test aid, not a step of the method): in the library variant
 * built with -DOCN_BOUNDS_CHECK=1 (libocn_checked.so: python -m
 * paper_2502_14148_gb300.build --checked), the tendency kernel, the projection
 * FFTs and the tridiagonal solve check their indices; an index outside its array
 * sets a bit of the model's status word (1 stencil window outside the staged
 * plane, 2 gather source, 4 face-flux slot, 8 state/tendency element, 16 FFT
 * shared buffer, 32 spectrum/velocity/pressure element, 64 tridiagonal unknown)
 * and is replaced by 0, so that nothing faults or traps.  Synchronises the model
 * stream, returns the word in *status and clears it; *checked (if not null) is 1
 * in the checked variant and 0 in the normal build (whose word stays 0).
 * Errors: OCN_ERR_ARG, OCN_ERR_STATE (no arena), OCN_ERR_CUDA. */
ocn_status ocn_bounds_status(ocn_model* model, unsigned* status, int* checked);

/* Wait until every host transfer issued on the model so far (the copies of
 * ocn_set_field(s) and everything of ocn_get_field(s)) has completed.
 * Errors: OCN_ERR_ARG, OCN_ERR_CUDA. */
ocn_status ocn_wait_transfers(ocn_model* model);

/* Several fields in one call: fields[i], srcs[i] / dsts[i] and nbytes[i] for
 * i < n, each as in ocn_set_field / ocn_get_field, applied in order.  All
 * copies of a set are issued first, back to back, and the call returns once
 * they are done (the follow-up work of tracers and of w stays queued on the
 * model stream), so no copy waits for another field's kernels.  A get forms the
 * full value of every requested tracer before the first copy, in the tracer's
 * slot of the model's other state buffer (which holds the previous stage state,
 * dead between steps and overwritten by the next one), then copies everything
 * and returns when all data has arrived (to host memory).  This is the host
 * transfer to use for a whole state: one wait per call instead of one per
 * field.  Errors: as for the single-field calls; nothing is enqueued when an
 * argument is invalid. */
ocn_status ocn_set_fields(ocn_model* model, int n, const int* fields, const void* const* srcs, const size_t* nbytes,
                          int src_is_device);
ocn_status ocn_get_fields(ocn_model* model, int n, const int* fields, void* const* dsts, const size_t* nbytes,
                          int dst_is_device);

/* Enforce incompressibility of the current velocity: solve the discrete
 * Poisson problem lap p = div u (Eq. pressure-poisson with dt = 1) and set
 * u -= grad p (Eq. pressure-correction).  Errors: OCN_ERR_STATE, OCN_ERR_CUDA. */
ocn_status ocn_project(ocn_model* model);

/* Advance nsteps full RK3 steps of size dt (three substages each; Appendix A.1
 * Eq. rk3 and Appendix A.2).  Each substage: eddy diffusivities, fused
 * tendency + RK update, then the pressure projection with step
 * (gamma_m - zeta_m) dt.  Buoyancy enters through the hydrostatic split of
 * Eq. pressure-decomposition: -grad_h p_hy in the horizontal momentum
 * equations, p_hy integrated up each column, the w equation without b (the
 * result equals the unsplit form up to rounding, since the two differ by a
 * discrete gradient that the projection removes).  Errors: OCN_ERR_ARG (nsteps < 0, dt not finite),
 * OCN_ERR_STATE, OCN_ERR_CUDA. */
ocn_status ocn_time_step(ocn_model* model, double dt, int nsteps);

/* Evaluate the tendencies G of every prognostic field at the current state
 * (no stepping; readable as OCN_FIELD_G + f), in the unsplit form: b
 * interpolated to the w faces appears in G_w.  Errors: OCN_ERR_STATE, OCN_ERR_CUDA. */
ocn_status ocn_compute_tendencies(ocn_model* model);

/* Diagnostics in FP64 (synchronises the stream).  out[0..n_tracers-1] = sum V c_n;
 * then sum V u, sum V v, sum V w, max |div u|, dt * max(|u|/dx, |v|/dy, |w|/dz),
 * count of non-finite values: nout must be >= n_tracers + 6.
 * Returns OCN_ERR_NONFINITE if any value is not finite and OCN_ERR_CFL if the
 * CFL number exceeds 1 (the values are written in both cases). */
ocn_status ocn_diagnostics(ocn_model* model, double dt, double* out, int nout);

/* Options.  OCN_OPT_GRAPHS: 1 (default) replays each time step from a CUDA
 * graph captured on first use per dt (at most 32 kept per model or ensemble: a
 * run with many distinct dt values starts the cache over); 0 launches kernels
 * directly.
 * OCN_OPT_SYNC_CHECK: 1 synchronises and checks for errors after every kernel.
 * OCN_OPT_KERNEL_TIMING: 1 launches directly and brackets every kernel with
 * CUDA events on the model stream (read with ocn_kernel_times); 0 (default) off. */
enum { OCN_OPT_GRAPHS = 1, OCN_OPT_SYNC_CHECK = 2, OCN_OPT_KERNEL_TIMING = 3, OCN_OPT_TENDENCY_VARIANT = 4 };
ocn_status ocn_set_option(ocn_model* model, int option, long long value);

/* Tile variants of the FP32 tendency kernel (OCN_OPT_TENDENCY_VARIANT): 0 = 32x8
 * columns per CTA, one CTA per SM; 1 = 32x8, two CTAs per SM; 2 = 32x16; 3 = 32x4,
 * three CTAs per SM; 4 = 32x14 (default); 5 = 32x12; 6 = 16x16, two CTAs per SM (for grids
 * under 32 columns wide).  All compute the same values. */
#define OCN_TENDENCY_VARIANTS 7

/* Autotuner: times every tendency variant on the model's current state (tendency
 * only: the state is not advanced; G is overwritten, so a QAB2 model restarts with
 * its Euler step), selects the fastest and
 * returns its index in *best and the milliseconds per launch of every variant in
 * ms[OCN_TENDENCY_VARIANTS] (either may be NULL).  Synchronises the stream.
 * Errors: OCN_ERR_STATE (no arena), OCN_ERR_CUDA. */
ocn_status ocn_autotune(ocn_model* model, int* best, double* ms);

/* Kernel classes reported by ocn_kernel_times. */
enum {
  OCN_K_CLOSURE = 0,     /* eddy diffusivities */
  OCN_K_TENDENCY = 1,    /* fused tendency + RK update */
  OCN_K_DIV_FFTX = 2,    /* divergence + real FFT in x */
  OCN_K_FFT_Y = 3,       /* complex FFT in y (forward and inverse) */
  OCN_K_TRIDIAG = 4,     /* tridiagonal solve in z */
  OCN_K_GAUGE = 5,       /* pressure gauge */
  OCN_K_IFFTX = 6,       /* inverse real FFT in x */
  OCN_K_CORRECT = 7,     /* velocity correction */
  OCN_K_COLUMN_CLOSURE = 8, /* learned column closure (features + network + flux divergence) */
  OCN_K_VERTICAL = 9,    /* vertical diffusion with diffusivity profiles (explicit or implicit) */
  OCN_K_COUNT = 10
};

/* Launch counts and summed device milliseconds per kernel class, accumulated
 * since OCN_OPT_KERNEL_TIMING was last set to 1; synchronises the stream.
 * counts and ms must hold OCN_K_COUNT entries.  Errors: OCN_ERR_ARG, OCN_ERR_CUDA. */
ocn_status ocn_kernel_times(ocn_model* model, int* counts, double* ms);

/* Number of kernel launches the last ocn_time_step issued per RK3 step. */
ocn_status ocn_launches_per_step(const ocn_model* model, int* launches);

/* Coarse-graining profiles (training data for column closures; horizontal means over the
 * periodic plane): out[0..Nz) <b>, [Nz..2Nz) <u>, [2Nz..3Nz) <v> at the levels, then the mean
 * upward flux of b, u and v through the faces 0..Nz (Nz+1 values each): the model's own face
 * flux (advective + closure; the prescribed fluxes at the walls), obtained exactly from the
 * mean budget of a tendency evaluation.  Overwrites G; the state is not advanced.  nout must be
 * >= 3*Nz + 3*(Nz+1).  Synchronises the stream.  Errors: OCN_ERR_ARG, OCN_ERR_STATE, OCN_ERR_CUDA. */
ocn_status ocn_profiles(ocn_model* model, double* out, int nout);

/* Conservative regridding of a column of cell averages between two ascending face lists
 * (finite-volume averaging, Sec. B listing "finite-volumes": integrals are preserved): out[j] is
 * the average over output cell j of the piecewise-constant input.  Host only.  Errors: OCN_ERR_ARG. */
ocn_status ocn_regrid(const double* zf_in, int nin, const double* in, const double* zf_out, int nout, double* out);

/* Ensembles: n independent members (own grids, forcings and sizes, one precision) stepped together.
 * Members share one device arena and the ensemble's stream; ocn_ensemble_member returns a borrowed
 * model handle (set/get/project/diagnostics/profiles; do not destroy it).  ocn_ensemble_time_step
 * advances every member by nsteps steps in one of three modes (OCN_OPT_ENSEMBLE_MODE):
 *  - OCN_ENSEMBLE_CONCURRENT (default): each step is one CUDA graph launch whose independent
 *    per-member branches of per-member kernels run concurrently;
 *  - OCN_ENSEMBLE_BATCHED: each step is one graph in which every kernel of the step is one launch
 *    over all members whose kernel sequences agree (same order, closure, tracers, stepper, tile
 *    variant; a learned closure with one shared network and feature normalisation).  Its blocks
 *    are the concatenation of the members' grids, each block taking its member's arguments from a
 *    device work list, so uneven sizes share a launch.  The members of such a group are split
 *    into OCN_OPT_ENSEMBLE_BRANCHES graph branches (1..64, default 4; balanced by cell count)
 *    whose launches overlap;
 *  - OCN_ENSEMBLE_SEQUENTIAL: members are stepped one after the other (the comparison baseline).
 * All modes give the same results bit for bit.  ocn_ensemble_autotune picks the tendency tile
 * variants in context: it times every member's tendency kernel launched together as in a step of
 * the ensemble's mode (batched launches, or each member on its own branch), first with one
 * variant for all FP32 members, then other variants per member shape (Nx, Ny, Nz, order,
 * closure, tracers), keeping a change only when the whole pass gets more than 2 % faster; call it
 * after choosing the mode.  variants[n] receives the choices (may be NULL).  Like ocn_autotune it
 * overwrites G (QAB2 members restart with their Euler step).  Errors as for the single-model
 * calls. */
typedef struct ocn_ensemble ocn_ensemble;
enum { OCN_OPT_ENSEMBLE_MODE = 5, OCN_OPT_ENSEMBLE_BRANCHES = 6 };
enum { OCN_ENSEMBLE_CONCURRENT = 0, OCN_ENSEMBLE_SEQUENTIAL = 1, OCN_ENSEMBLE_BATCHED = 2 };
ocn_status ocn_ensemble_create(int n, const ocn_grid_desc* grids, const ocn_model_desc* models, void* stream,
                               ocn_ensemble** out);
void ocn_ensemble_destroy(ocn_ensemble* ensemble);
ocn_status ocn_ensemble_arena_bytes(const ocn_ensemble* ensemble, size_t* bytes);
ocn_status ocn_ensemble_bind_arena(ocn_ensemble* ensemble, void* device_ptr, size_t bytes);
ocn_status ocn_ensemble_member(ocn_ensemble* ensemble, int i, ocn_model** member);
ocn_status ocn_ensemble_time_step(ocn_ensemble* ensemble, double dt, int nsteps);
ocn_status ocn_ensemble_set_option(ocn_ensemble* ensemble, int option, long long value);
ocn_status ocn_ensemble_autotune(ocn_ensemble* ensemble, int* variants);
ocn_status ocn_ensemble_launches_per_step(const ocn_ensemble* ensemble, int* launches);

/* No-allocation projection.  Some callers cannot call cudaMalloc: plug-ins
 * whose host application owns every device allocation through its own pool
 * allocator, and loops that must not allocate once they are running.  This
 * entry point gives them the projection of ocn_project -- lap p = div u with
 * Neumann walls and a zero-volume-mean gauge, then u -= grad p -- for a
 * velocity (u, v, w) and pressure p that the caller already holds, with every
 * other work array (spectrum, pivots, metrics, twiddles) inside a fixed device
 * array of about 6.3 MB that the library declares at file scope.  The paper has
 * no counterpart: it is a deployment variant of the projection, not a step of
 * the method.
 *   precision  32 (float arrays) or 64 (double arrays)
 *   Nx, Ny, Nz, Lx, Ly, z_faces   the grid, as in ocn_grid_desc (z_faces in host memory)
 *   u, v, w, p device arrays in the layouts above; u, v, w are corrected in place,
 *              p receives the pressure
 *   stream     cudaStream_t for all work (NULL: legacy default stream); the call
 *              returns after enqueueing
 *   error      if not NULL, receives a static description of a failure ("" on success)
 * Limits: Nx, Ny, Nz <= OCN_NOALLOC_MAX_N and (Nx/2+1)*Ny*Nz <= OCN_NOALLOC_MAX_MODES,
 * else OCN_ERR_ARG (so are the grid rules of ocn_grid_create).
 * The call allocates no device memory (no cudaMalloc, cudaFree or allocating
 * library routine).  The first call on each device looks up the device address
 * of the array and keeps it.  Every call uploads its grid tables from a host
 * array on the stream, so the call cannot be captured into a CUDA graph: a
 * stream that is being captured is refused with OCN_ERR_UNSUPPORTED before
 * anything is enqueued.
 * Every call on a device shares the one array and leaves its contents behind
 * (each call rewrites all it reads, so nothing needs clearing), so calls whose
 * work overlaps on the GPU, e.g. on two streams at once, race and must be
 * serialised by the caller.  Every device that loads the library holds the
 * array until the process exits. */
#define OCN_NOALLOC_MAX_N 4096
#define OCN_NOALLOC_MAX_MODES 262144
ocn_status ocn_project_noalloc(int precision, int Nx, int Ny, int Nz, double Lx, double Ly, const double* z_faces,
                               void* u, void* v, void* w, void* p, void* stream, const char** error);

/* Learned column closure: a multilayer perceptron trained and evaluated on the
 * 5th-generation tensor cores.  The paper motivates closures calibrated on LES
 * output (Sec. 3.2.3: CATKE is calibrated against a suite of LES; its outlook:
 * machine-learned parameterisations) but prints no network; this one is
 *   z_l = h_{l-1} W_l^T + b_l,  h_l = gelu(z_l) (exact erf form) for hidden layers,
 *   y = h_{L-1} W_L^T + b_L,
 * with the masked mean-square loss L = (1/2M) sum_m sum_j mask_j (y_mj - t_mj)^2
 * and Adam (Kingma & Ba 2015, bias-corrected).  Products run in BF16 with FP32
 * accumulation; master weights, biases, Adam moments and gradients are FP32.
 *   sizes      nlayers+1 widths (input, hidden..., output), each 16..256 and a multiple of 16
 *   max_batch  largest M of any later call (rows are padded to a multiple of 128 internally)
 *   stream     cudaStream_t for all work (NULL: legacy default stream)
 * Parameters are one flat FP32 array: for each layer W_l [n_out][n_in] (row-major) then
 * b_l [n_out]; ocn_mlp_num_params gives its length.  The caller allocates the device
 * arena (ocn_mlp_arena_bytes, 256-byte aligned) and binds it; binding zeroes it.
 * X [M][n_in], T and Y [M][n_out], mask [n_out] and grads (flat, the parameter layout)
 * are FP32 device arrays.  ocn_mlp_forward and ocn_mlp_adam return after enqueueing;
 * ocn_mlp_gradients, ocn_mlp_set_params/get_params (host side) and ocn_mlp_train_step
 * with a non-null loss synchronise the stream.  loss (host double) receives L.
 * ocn_mlp_train_step = gradients then one Adam step (lr; beta1 0.9, beta2 0.999, eps 1e-8);
 * set_params resets the Adam state.  Parameter updates (set_params from device memory,
 * ocn_mlp_adam, ocn_mlp_train_step without loss) are ordered on the network's stream only:
 * a model that uses the network on another stream must be ordered after them by the caller
 * (for example by synchronising the network's stream).  Errors: OCN_ERR_ARG (sizes, batch, null pointers),
 * OCN_ERR_STATE (no arena), OCN_ERR_CUDA, OCN_ERR_TIMEOUT (a bounded wait for the tensor
 * cores gave up; the results are then invalid). */
#define OCN_MLP_MAX_LAYERS 8
typedef struct ocn_mlp ocn_mlp;
ocn_status ocn_mlp_create(int nlayers, const int* sizes, int max_batch, void* stream, ocn_mlp** out);
void ocn_mlp_destroy(ocn_mlp* mlp);
ocn_status ocn_mlp_arena_bytes(const ocn_mlp* mlp, size_t* bytes);
ocn_status ocn_mlp_bind_arena(ocn_mlp* mlp, void* device_ptr, size_t bytes);
ocn_status ocn_mlp_num_params(const ocn_mlp* mlp, size_t* count);
ocn_status ocn_mlp_set_params(ocn_mlp* mlp, const float* params, size_t count, int src_is_device);
ocn_status ocn_mlp_get_params(ocn_mlp* mlp, float* params, size_t count, int dst_is_device);
ocn_status ocn_mlp_forward(ocn_mlp* mlp, const float* X, int M, float* Y);
ocn_status ocn_mlp_gradients(ocn_mlp* mlp, const float* X, const float* T, const float* mask, int M, float* grads,
                             double* loss);
ocn_status ocn_mlp_adam(ocn_mlp* mlp, const float* grads, double lr, double beta1, double beta2, double eps);
ocn_status ocn_mlp_train_step(ocn_mlp* mlp, const float* X, const float* T, const float* mask, int M, double lr,
                              double* loss);

/* Time stepper (Appendix A.1).  OCN_STEPPER_RK3 (default): the low-storage RK3 of Eq. rk3, three
 * substages per step.  OCN_STEPPER_QAB2: Eq. qab2, one tendency evaluation and one projection per
 * step, G^{m+1} weights (3/2 + chi, -(1/2 + chi)); the first step after any state field is set is
 * forward Euler (chi = -1/2), and restoring an OCN_FIELD_G field marks the run as continuing (set
 * the state first, then G, to restart a QAB2 run bitwise).  Errors: OCN_ERR_ARG. */
enum { OCN_STEPPER_RK3 = 0, OCN_STEPPER_QAB2 = 1 };
ocn_status ocn_set_time_stepper(ocn_model* model, int scheme, double chi);

/* Vertical diffusion with diffusivity profiles (Eq. tracer-with-tendency and Eq.
 * momentum-tendency-definition): nu_faces applies to u, v, w and kappa_faces to every tracer,
 * both given at the Nz+1 w-faces in host memory (copied; NULL = none; values finite and >= 0).
 * Second-order finite volumes with no flux through the walls; w uses the mean of the two faces
 * at each centre.  implicit = 0 adds d/dz(kappa dq/dz) to the explicit tendency; implicit = 1
 * solves (1 - dtau d/dz kappa d/dz) q = q~ down every column after each stage update (Eq.
 * tracer-time-discretization, Eq. predictor-velocity), dtau the stage step ((gamma - zeta) dt,
 * dt for QAB2), before the projection.  The implicit solver keeps 4 Nz factor values in shared
 * memory: Nz <= 3072 in FP32 and 1536 in FP64, else OCN_ERR_UNSUPPORTED.  ocn_compute_tendencies
 * and ocn_profiles include only the explicit form.  Errors: OCN_ERR_ARG, OCN_ERR_STATE, OCN_ERR_UNSUPPORTED, OCN_ERR_CUDA. */
ocn_status ocn_set_vertical_diffusivity(ocn_model* model, const double* nu_faces, const double* kappa_faces,
                                        int implicit);

/* Learned column closure of a model (FP32 buoyancy-tracer models; others give
 * OCN_ERR_UNSUPPORTED).  Each w-face k of each cell-centre column (i, j) gets a
 * vertical flux F_q, q in {b, ubar, vbar} (ubar = (u_i + u_{i+1})/2, vbar likewise),
 * predicted by a 32-128-128-128-16 network of ocn_mlp_* from 20 raw features:
 *   0-4   db/dz at faces k-2..k+2, 5-9 dubar/dz, 10-14 dvbar/dz (0 outside faces 1..Nz-1),
 *   15    surface buoyancy flux (top_flux of tracer 0), 16 f, 17 N2_background,
 *   18    depth zf[Nz] - zf[k],
 *   19    mixed-layer depth estimate sum_{q=1}^{Nz-1} max(0, 1 - (db/dz)_q / N2_background) dz_f[q]
 *         (0 when N2_background <= 0),
 * normalised x_n = (x - mu) / sigma (features 20..31 are 0), F_q = out_scale[q] y_q, and
 * zero at the walls.  Each tendency evaluation then adds -dF_b/dz to G_b, and -dF/dz of the
 * ubar (vbar) flux averaged onto the u (v) columns to G_u (G_v), on top of the model's own
 * closure (which stays the fallback: ocn_set_column_closure(m, NULL, NULL) removes the learned
 * part).  The network is borrowed: it must stay alive and bound while the model steps; later
 * training of it takes effect at once.  The paper motivates closures calibrated on LES
 * (Sec. 3.2.3) without specifying one; this closure is an extension.
 * ocn_closure_features writes the raw features of every face of the current state to X
 * (device FP32 [(Nz+1)*Ny*Nx][32], sample order k, j, i with i fastest).
 * ocn_column_fluxes writes F (device FP32 [3][Nz+1][Ny][Nx]) of the current state: which 0 =
 * the model's own closure flux -kappa_f dq/dz (b), -nu_f dq/dz (ubar, vbar) with face
 * diffusivities the mean of the two adjacent centres; which 1 = the learned flux.
 * ocn_coarse_grain box-filters the current state onto a cx x cy horizontal grid (cx | Nx,
 * cy | Ny; vertical grid kept) into out (device FP64, cx*cy*(7*Nz+4) values):
 *   [u_c Nz*cy*cx][v_c Nz*cy*cx][w_c (Nz+1)*cy*cx][b_c Nz*cy*cx][tau 3*(Nz+1)*cy*cx],
 * u_c the mean of u over the fine faces on coarse face I, v_c likewise, w_c and b_c box means,
 * tau_q = <w q_f> - <w><q_f> + <F_q of which 0> at interior faces, q_f = (q_{k-1} + q_k)/2 (the
 * subfilter vertical flux that a coarse model does not resolve), 0 at the walls.
 * All three enqueue on the model stream and return.  Errors: OCN_ERR_ARG, OCN_ERR_STATE,
 * OCN_ERR_UNSUPPORTED, OCN_ERR_CUDA; a bounded wait that gave up inside the network makes
 * the next ocn_diagnostics return OCN_ERR_TIMEOUT. */
typedef struct {
  float mu[32];              /* feature means */
  float sigma[32];           /* feature scales, > 0 */
  float out_scale[3];        /* flux scales of b, ubar, vbar */
  double N2_background;      /* background stratification (feature 17 and the depth estimate) */
} ocn_column_closure_desc;
ocn_status ocn_set_column_closure(ocn_model* model, const ocn_mlp* mlp, const ocn_column_closure_desc* desc);
/* How the learned column closure enters the step.  mode 0 (the default): the network's outputs
 * are face fluxes F_b, F_ubar, F_vbar, applied explicitly as above.  mode 1: outputs 0 and 1 are
 * eddy diffusivities kappa = max(0, out_scale[0] y_0) and nu = max(0, out_scale[1] y_1) at every
 * interior w-face of every column (output 2 is unused); in each substage, after the stage update,
 * their horizontal means over the grid become the vertical diffusivity profiles (kappa for the
 * tracers, nu for u, v and w; zero at the walls) of the semi-implicit column solve of
 * ocn_set_vertical_diffusivity (Eq. tracer-time-discretization, Eq. predictor-velocity),
 * (I - dtau d/dz K d/dz) q = q~, so a large learned diffusivity cannot make the step unstable.
 * The network's fluxes are then -kappa db/dz, -nu dubar/dz, -nu dvbar/dz.  A tendency evaluation
 * (ocn_compute_tendencies) takes nothing from the closure in this mode, as with any implicit
 * vertical diffusion.  Mode 1 needs an FP32 buoyancy-tracer model without profiles of its own
 * (ocn_set_vertical_diffusivity refuses them while it is active).  The mode is kept when the
 * network is replaced or removed.  Errors: OCN_ERR_ARG (mode not 0 or 1), OCN_ERR_UNSUPPORTED,
 * OCN_ERR_STATE. */
ocn_status ocn_set_column_closure_mode(ocn_model* model, int mode);
ocn_status ocn_closure_features(ocn_model* model, double N2_background, float* X);
ocn_status ocn_column_fluxes(ocn_model* model, int which, float* F);
ocn_status ocn_coarse_grain(ocn_model* model, int cx, int cy, double* out, size_t nout);

/* The tensor-core product under the network, exposed for testing: D = A B^T with
 * A [M][K] and B [N][K] BF16 device arrays (K contiguous; lda, ldb >= K and multiples
 * of 8; 16-byte aligned), D [M][ldd] FP32, 16 <= N <= 256 with N a multiple of 16, K a
 * positive multiple of 8.  status (device int, may be NULL) is set to 1 if a bounded
 * wait gave up.  Enqueued on stream.  Errors: OCN_ERR_ARG, OCN_ERR_CUDA. */
ocn_status ocn_gemm_bf16(int M, int N, int K, const void* A, int lda, const void* B, int ldb, float* D, int ldd,
                         int* status, void* stream);

/* Measured FP32 FMA throughput of the current device in TFLOP/s (an FMA counts 2): independent
 * fused multiply-add chains on every SM for about 10 ms; the measured denominator of ALU-bound
 * rooflines.  Synchronises the stream.  Errors: OCN_ERR_ARG, OCN_ERR_CUDA. */
ocn_status ocn_fp32_fma_peak(double* tflops, void* stream);

/* Failure-detection test of the tensor-core kernels' bounded waits: launches the GEMM kernel with its
 * MMA and commit left out, so the bounded mbarrier wait runs out after about 0.5 s; the kernel sets
 * *status (device int) to 1, waits once more (bounded), frees its tensor memory and returns, leaving
 * the context usable.  Enqueued on stream.  This entry allocates 20 KB of device memory on first use
 * (kept until exit) -- the one exception to the no-allocation rule, for tests only. */
ocn_status ocn_gemm_timeout_test(int* status, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* OCN_H */
