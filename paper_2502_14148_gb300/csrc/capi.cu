// C ABI (include/ocn.h): grid and model objects, the device arena layout, the
// RK3 substage sequence and its CUDA-graph replay.
//
// One RK3 substage m (Appendix A.1 Eq. rk3, Appendix A.2):
//   1. eddy diffusivities (Smagorinsky-Lilly / AMD)            k_closure
//   2. tendencies, u~ = u + dt(gamma G^m - zeta G^{m-1}),
//      tracers c^{m+1} likewise, G^{m-1} <- G^m              k_tendency
//   3. projection with the stage step (gamma-zeta) dt        k_div_fftx ... k_correct
// The state is double buffered (the tendency stencil reads neighbours of the
// old state while the new one is written); every substage swaps buffers.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "batch.cuh"
#include "ocn_internal.cuh"

using namespace ocn;

namespace ocn {
// step graphs kept per model or ensemble (keyed by time step, buffer parity, stepper state)
constexpr size_t kGraphCacheMax = 32;

LaunchRecorder*& active_recorder() {
  static thread_local LaunchRecorder* r = nullptr;
  return r;
}

cudaError_t raise_smem_limit(const void* fn, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> limit;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  size_t& cur = limit[{dev, fn}];
  if (bytes <= cur) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}
}  // namespace ocn

namespace {

thread_local std::string g_err;

ocn_status fail(ocn_status s, const std::string& msg) {
  g_err = msg;
  return s;
}
ocn_status cuda_fail(cudaError_t e, const char* what) {
  return fail(OCN_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

bool is_2a3b(int n) {
  if (n < 1) return false;
  while (n % 2 == 0) n /= 2;
  while (n % 3 == 0) n /= 3;
  return n == 1;
}

FftPlan make_plan(int n) {
  FftPlan p;
  memset(&p, 0, sizeof(p));
  p.n = n;
  int m = n;
  while (m % 8 == 0 && p.npass < kMaxFftPasses) { p.radix[p.npass++] = 8; m /= 8; }
  while (m % 4 == 0 && p.npass < kMaxFftPasses) { p.radix[p.npass++] = 4; m /= 4; }
  while (m % 2 == 0 && p.npass < kMaxFftPasses) { p.radix[p.npass++] = 2; m /= 2; }
  while (m % 3 == 0 && p.npass < kMaxFftPasses) { p.radix[p.npass++] = 3; m /= 3; }
  return p;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int now = -1;
    if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
  }
};

std::mutex g_tab_mu;
bool g_tab_ready = false;
WenoTables<double> g_tab;
uint64_t g_tab_devices = 0;

cudaError_t ensure_tables(int dev) {
  std::lock_guard<std::mutex> lk(g_tab_mu);
  if (!g_tab_ready) { derive_weno_tables(&g_tab); g_tab_ready = true; }
  if (dev < 64 && (g_tab_devices >> dev) & 1ull) return cudaSuccess;
  cudaError_t e = upload_weno_tables(g_tab);
  if (e == cudaSuccess && dev < 64) g_tab_devices |= (1ull << dev);
  return e;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

struct ocn_grid {
  int Nx, Ny, Nz;
  double Lx, Ly;
  std::vector<double> zf, zc, dzc, dzf;
  bool stretched;
};

struct ocn_model {
  const ocn_grid* g = nullptr;
  ocn_model_desc d;
  cudaStream_t stream = nullptr;
  int dev = 0;
  int R = 3;
  int es = 4;                       // element size
  int nf = 4;                       // prognostic fields: u, v, w, tracers
  bool fp64_piv = false;
  // arena layout (byte offsets)
  size_t bytes = 0;
  size_t off_state[2][3 + OCN_MAX_TRACERS];
  size_t off_G[3 + OCN_MAX_TRACERS];
  size_t off_p = 0, off_nu = 0, off_kap[OCN_MAX_TRACERS], off_spec = 0, off_cpiv = 0, off_pinv = 0;
  size_t off_dzc = 0, off_rdzc = 0, off_dzf = 0, off_rdzf = 0, off_lamx = 0, off_lamy = 0, off_twx = 0, off_twy = 0;
  size_t off_partial = 0, off_diag = 0, off_oob = 0;
  char* arena = nullptr;
  int cur = 0;
  bool graphs = true, sync_check = false;
  int variant = 4;                  // FP32 tendency tile variant (32x14: 128 registers, 16 warps, no spills)
  std::map<std::pair<uint64_t, int>, cudaGraphExec_t> graph_cache;
  unsigned graph_epoch = 0;        // bumped whenever captured graphs go stale (ensemble graphs key on it)
  int launches_per_step = 0;
  FftPlan px, py;
  // Tracers are stored as anomalies about a per-level reference profile (their
  // horizontal mean when set).  The kernels add the profile back wherever the
  // full value enters the arithmetic (z stencils, EOS, vertical gradients) and
  // use shift invariance elsewhere, so results are unchanged while FP32 state
  // storage keeps the digits of the dynamic part rather than of the mean
  // stratification.
  size_t off_cref[OCN_MAX_TRACERS] = {0, 0, 0, 0};
  std::vector<double> cref_host[OCN_MAX_TRACERS];
  // Host transfers.  ocn_set_field waits only for its copies (copy_done): the reference-profile
  // kernels of a tracer run afterwards on the model stream, and cref_host is read back from the
  // device where it is used (cref_pending), not in the set call, so that no small copy to the host
  // queues on the model stream behind the large copies of another model.  ocn_get_field runs on
  // xfer, a stream of the greatest priority ordered after the model stream (xfer_in) and the model
  // stream after it (xfer_out), so that its kernel is not queued behind the blocks of another
  // model's step that shares the GPU.
  cudaStream_t xfer = nullptr;
  cudaEvent_t xfer_in = nullptr, xfer_out = nullptr, copy_done = nullptr;
  bool cref_pending[OCN_MAX_TRACERS] = {false, false, false, false};
  // kernel timing (OCN_OPT_KERNEL_TIMING)
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  struct Rec { int kclass; cudaEvent_t a, b; };
  std::vector<Rec> recs;
  cudaEvent_t ev_open = nullptr;
  LaunchHook hook;
  // learned column closure (FP32 buoyancy-tracer models): face fluxes, mixed-layer depths,
  // face depths, the device status word of its bounded waits; the borrowed network and its
  // normalisation
  size_t off_colF = 0, off_colh = 0, off_depth = 0, off_status = 0;
  const ocn_mlp* colc = nullptr;
  float colc_mu[kColumnFeatures] = {0}, colc_isig[kColumnFeatures] = {0}, colc_scale[3] = {0, 0, 0};
  double colc_N2 = 0.0;
  int colc_version = 0;
  int colc_mode = 0;                // 0: face fluxes, explicit; 1: diffusivities through the implicit step
  // time stepper (Eq. rk3 or Eq. qab2) and vertical diffusivity profiles (explicit or semi-implicit)
  int stepper = OCN_STEPPER_RK3;
  double chi = 0.1;
  bool ab_started = false;         // QAB2: G^{m-1} holds a previous tendency
  size_t off_nuz = 0, off_kapz = 0;
  bool vnu = false, vkap = false, vimplicit = false;
};

struct ocn_ensemble {
  int n = 0;
  int dev = 0;
  int es = 4;
  cudaStream_t stream = nullptr;             // the ensemble's stream (member handles use it too)
  std::vector<ocn_grid*> grids;
  std::vector<ocn_model*> models;
  std::vector<cudaStream_t> fork_streams;    // one per member, joined back into `stream` in each graph
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  std::vector<size_t> offs;
  size_t bytes = 0;
  char* arena = nullptr;
  int mode = 0;                              // OCN_ENSEMBLE_CONCURRENT, _SEQUENTIAL or _BATCHED
  int branches = 4;                          // batched mode: graph branches per group of members
  std::map<std::string, cudaGraphExec_t> graphs;
  std::map<std::string, void*> graph_tables;  // device work lists of the batched graphs
  int launches_per_step = 0;
};

namespace {

// The transfer stream and its events, created on first use.
cudaError_t xfer_setup(ocn_model* m) {
  if (m->xfer) return cudaSuccess;
  int lo = 0, hi = 0;
  cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m->xfer_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m->xfer_out, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m->copy_done, cudaEventDisableTiming);
  cudaStream_t s = nullptr;
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, hi);
  if (e == cudaSuccess) m->xfer = s;
  return e;
}
void xfer_release(ocn_model* m) {
  if (m->xfer) cudaStreamDestroy(m->xfer);
  if (m->xfer_in) cudaEventDestroy(m->xfer_in);
  if (m->xfer_out) cudaEventDestroy(m->xfer_out);
  if (m->copy_done) cudaEventDestroy(m->copy_done);
  m->xfer = nullptr; m->xfer_in = m->xfer_out = m->copy_done = nullptr;
}
// Read back the reference profiles that ocn_set_field left pending into the host mirror (after the
// model stream has been synchronised past the kernels that formed them).
cudaError_t cref_refresh(ocn_model* m) {
  for (int t = 0; t < m->d.n_tracers; ++t) {
    if (!m->cref_pending[t]) continue;
    std::vector<char> hb((size_t)m->g->Nz * m->es);
    cudaError_t e = cudaMemcpy(hb.data(), m->arena + m->off_cref[t], hb.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return e;
    for (int k = 0; k < m->g->Nz; ++k)
      m->cref_host[t][k] = (m->es == 4) ? (double)reinterpret_cast<const float*>(hb.data())[k] : reinterpret_cast<const double*>(hb.data())[k];
    m->cref_pending[t] = false;
  }
  return cudaSuccess;
}

cudaEvent_t take_event(ocn_model* m) {
  if (!m->ev_pool.empty()) { cudaEvent_t e = m->ev_pool.back(); m->ev_pool.pop_back(); return e; }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
void hook_before(void* ctx, int) {
  ocn_model* m = static_cast<ocn_model*>(ctx);
  m->ev_open = take_event(m);
  cudaEventRecord(m->ev_open, m->stream);
}
void hook_after(void* ctx, int kclass) {
  ocn_model* m = static_cast<ocn_model*>(ctx);
  cudaEvent_t b = take_event(m);
  cudaEventRecord(b, m->stream);
  m->recs.push_back({kclass, m->ev_open, b});
  m->ev_open = nullptr;
}

size_t field_elems(const ocn_model* m, int f) {
  size_t plane = (size_t)m->g->Nx * m->g->Ny;
  return plane * (size_t)(f == OCN_FIELD_W ? m->g->Nz + 1 : m->g->Nz);
}

template <typename T>
T* at(const ocn_model* m, size_t off) { return reinterpret_cast<T*>(m->arena + off); }

template <typename T>
StatePtrs<T> state_ptrs(const ocn_model* m, int which) {
  StatePtrs<T> s;
  s.u = at<T>(m, m->off_state[which][0]);
  s.v = at<T>(m, m->off_state[which][1]);
  s.w = at<T>(m, m->off_state[which][2]);
  for (int t = 0; t < kMaxTracers; ++t) s.c[t] = (t < m->d.n_tracers) ? at<T>(m, m->off_state[which][3 + t]) : nullptr;
  return s;
}

template <typename T>
StatePtrs<T> g_ptrs(const ocn_model* m) {
  StatePtrs<T> s;
  s.u = at<T>(m, m->off_G[0]);
  s.v = at<T>(m, m->off_G[1]);
  s.w = at<T>(m, m->off_G[2]);
  for (int t = 0; t < kMaxTracers; ++t) s.c[t] = (t < m->d.n_tracers) ? at<T>(m, m->off_G[3 + t]) : nullptr;
  return s;
}

bool column_closure_capable(const ocn_model* m) {
  return m->es == 4 && m->d.eos == OCN_EOS_BUOYANCY_TRACER;
}

void layout(ocn_model* m) {
  const ocn_grid* g = m->g;
  const size_t plane = (size_t)g->Nx * g->Ny;
  const size_t Nc = plane * g->Nz, Nw = plane * (g->Nz + 1);
  const size_t es = (size_t)m->es;
  size_t o = 0;
  auto take = [&](size_t nbytes) { size_t at_ = o; o = align256(o + nbytes); return at_; };
  for (int b = 0; b < 2; ++b)
    for (int f = 0; f < m->nf; ++f) m->off_state[b][f] = take(es * (f == 2 ? Nw : Nc));
  for (int f = 0; f < m->nf; ++f) m->off_G[f] = take(es * (f == 2 ? Nw : Nc));
  m->off_p = take(es * Nc);
  const bool stress = m->d.closure == OCN_CLOSURE_SMAGORINSKY || m->d.closure == OCN_CLOSURE_AMD;
  m->off_nu = stress ? take(es * Nc) : 0;
  for (int t = 0; t < OCN_MAX_TRACERS; ++t)
    m->off_kap[t] = (m->d.closure == OCN_CLOSURE_AMD && t < m->d.n_tracers) ? take(es * Nc) : 0;
  const size_t S = (size_t)spec_row_stride(g->Nx / 2) * g->Ny * g->Nz;
  m->off_spec = take(2 * es * S);
  m->off_cpiv = take(es * S);
  m->off_pinv = take(es * S);
  m->off_dzc = take(es * g->Nz);
  m->off_rdzc = take(es * g->Nz);
  m->off_dzf = take(es * (g->Nz + 1));
  m->off_rdzf = take(es * (g->Nz + 1));
  m->off_lamx = take(es * (g->Nx / 2 + 1));
  m->off_lamy = take(es * g->Ny);
  m->off_twx = take(2 * es * g->Nx);
  m->off_twy = take(2 * es * g->Ny);
  for (int t = 0; t < OCN_MAX_TRACERS; ++t) m->off_cref[t] = (t < m->d.n_tracers) ? take(es * g->Nz) : 0;
  m->off_partial = take(sizeof(double) * (size_t)diag_blocks() * (OCN_MAX_TRACERS + 6));
  m->off_diag = take(sizeof(double) * 16);
  m->off_oob = take(sizeof(unsigned));
  m->off_nuz = take(es * (g->Nz + 1));
  m->off_kapz = take(es * (g->Nz + 1));
  if (column_closure_capable(m)) {
    m->off_colF = take(sizeof(float) * 3 * Nw);
    m->off_colh = take(sizeof(float) * plane);
    m->off_depth = take(sizeof(float) * (g->Nz + 1));
    m->off_status = take(sizeof(int));
  }
  m->bytes = o;
}

template <typename T>
std::vector<char> metrics_blob(const ocn_model* m) {
  // host images of the metric tables, placed at their arena offsets relative to off_dzc
  const ocn_grid* g = m->g;
  std::vector<char> blob(m->off_twy + 2 * sizeof(T) * g->Ny - m->off_dzc, 0);
  auto put = [&](size_t off, size_t idx, T v) { memcpy(blob.data() + (off - m->off_dzc) + idx * sizeof(T), &v, sizeof(T)); };
  for (int k = 0; k < g->Nz; ++k) { put(m->off_dzc, k, (T)g->dzc[k]); put(m->off_rdzc, k, (T)(1.0 / g->dzc[k])); }
  for (int k = 0; k <= g->Nz; ++k) {
    put(m->off_dzf, k, (T)g->dzf[k]);
    put(m->off_rdzf, k, (T)((k >= 1 && k < g->Nz) ? 1.0 / g->dzf[k] : 0.0));
  }
  const double dx = g->Lx / g->Nx, dy = g->Ly / g->Ny;
  for (int kx = 0; kx <= g->Nx / 2; ++kx) { double s = 2.0 * sin(M_PI * kx / g->Nx) / dx; put(m->off_lamx, kx, (T)(-s * s)); }
  for (int ky = 0; ky < g->Ny; ++ky) { double s = 2.0 * sin(M_PI * ky / g->Ny) / dy; put(m->off_lamy, ky, (T)(-s * s)); }
  for (int t = 0; t < g->Nx; ++t) {
    double th = -2.0 * M_PI * (double)t / g->Nx;
    put(m->off_twx, 2 * t, (T)cos(th)); put(m->off_twx, 2 * t + 1, (T)sin(th));
  }
  for (int t = 0; t < g->Ny; ++t) {
    double th = -2.0 * M_PI * (double)t / g->Ny;
    put(m->off_twy, 2 * t, (T)cos(th)); put(m->off_twy, 2 * t + 1, (T)sin(th));
  }
  return blob;
}

template <typename T>
PoissonArgs<T> poisson_args(const ocn_model* m, int which, double dts) {
  const ocn_grid* g = m->g;
  PoissonArgs<T> a;
  memset(&a, 0, sizeof(a));
  StatePtrs<T> s = state_ptrs<T>(m, which);
  a.u = s.u; a.v = s.v; a.w = s.w;
  a.p = at<T>(m, m->off_p);
  a.spec = at<T>(m, m->off_spec);
  a.cpiv = at<T>(m, m->off_cpiv);
  a.pinv = at<T>(m, m->off_pinv);
  a.rdzc = at<T>(m, m->off_rdzc); a.rdzf = at<T>(m, m->off_rdzf); a.dzc = at<T>(m, m->off_dzc);
  a.lamx = at<T>(m, m->off_lamx); a.lamy = at<T>(m, m->off_lamy);
  a.twx = at<T>(m, m->off_twx); a.twy = at<T>(m, m->off_twy);
  a.Nx = g->Nx; a.Ny = g->Ny; a.Nz = g->Nz; a.Mx = g->Nx / 2; a.Sp = spec_row_stride(a.Mx);
  a.oob = at<unsigned>(m, m->off_oob);
  a.rdx = (T)(g->Nx / g->Lx); a.rdy = (T)(g->Ny / g->Ly);
  a.inv_dt = (T)(1.0 / dts); a.dt = (T)dts;
  a.scale = (T)(1.0 / ((double)(g->Nx / 2) * g->Ny));
  a.Htot = (T)(g->zf[g->Nz] - g->zf[0]);
  a.fp64_pivots = m->fp64_piv ? 1 : 0;
  a.px = m->px; a.py = m->py;
  return a;
}

// FP32 Smagorinsky-Lilly and AMD models compute their eddy diffusivities inside the tendency kernel
// (nu_e is written to the arena as they go), so a time step or a tendency evaluation launches no
// closure kernel for them.
inline bool tendency_computes_nu(const ocn_model* m) {
  return m->es == 4 && (m->d.closure == OCN_CLOSURE_SMAGORINSKY || m->d.closure == OCN_CLOSURE_AMD);
}

// The eddy-diffusivity kernel; with before_tendency, nothing when the tendency kernel that
// follows computes nu_e itself.
template <typename T>
cudaError_t enqueue_closure(ocn_model* m, int which, bool before_tendency = false) {
  const ocn_grid* g = m->g;
  if (!(m->d.closure == OCN_CLOSURE_SMAGORINSKY || m->d.closure == OCN_CLOSURE_AMD)) return cudaSuccess;
  if (before_tendency && tendency_computes_nu(m)) return cudaSuccess;
  ClosureArgs<T> c;
  memset(&c, 0, sizeof(c));
  c.cur = state_ptrs<T>(m, which);
  for (int t = 0; t < kMaxTracers; ++t) c.cref[t] = m->off_cref[t] ? at<T>(m, m->off_cref[t]) : nullptr;
  c.nu = at<T>(m, m->off_nu);
  for (int t = 0; t < kMaxTracers; ++t) c.kap[t] = m->off_kap[t] ? at<T>(m, m->off_kap[t]) : nullptr;
  c.dzc = at<T>(m, m->off_dzc); c.rdzc = at<T>(m, m->off_rdzc); c.rdzf = at<T>(m, m->off_rdzf);
  c.Nx = g->Nx; c.Ny = g->Ny; c.Nz = g->Nz; c.nt = m->d.n_tracers;
  c.dx = (T)(g->Lx / g->Nx); c.dy = (T)(g->Ly / g->Ny); c.rdx = (T)(g->Nx / g->Lx); c.rdy = (T)(g->Ny / g->Ly);
  c.closure = m->d.closure;
  c.Cs = (T)m->d.Cs; c.Cb = (T)m->d.Cb; c.inv_Pr = (T)(1.0 / m->d.Pr); c.C_amd = (T)m->d.C_amd;
  c.eos = m->d.eos;
  c.g_alpha = (T)(m->d.g * m->d.alpha); c.g_beta = (T)(m->d.g * m->d.beta); c.T0 = (T)m->d.T0; c.S0 = (T)m->d.S0;
  m->hook.pre(OCN_K_CLOSURE);
  cudaError_t e = launch_closure<T>(c, m->stream);
  m->hook.post(OCN_K_CLOSURE);
  return e;
}

template <typename T>
cudaError_t enqueue_tendency(ocn_model* m, int which, double dt_gamma, double dt_zeta, int mode) {
  const ocn_grid* g = m->g;
  TendencyArgs<T> a;
  memset(&a, 0, sizeof(a));
  a.cur = state_ptrs<T>(m, which);
  a.nxt = state_ptrs<T>(m, 1 - which);
  a.G = g_ptrs<T>(m);
  a.nu = m->off_nu ? at<T>(m, m->off_nu) : nullptr;
  for (int t = 0; t < kMaxTracers; ++t) a.kap[t] = m->off_kap[t] ? at<T>(m, m->off_kap[t]) : nullptr;
  a.rdzc = at<T>(m, m->off_rdzc); a.rdzf = at<T>(m, m->off_rdzf); a.dzf = at<T>(m, m->off_dzf);
  a.Nx = g->Nx; a.Ny = g->Ny; a.Nz = g->Nz; a.nt = m->d.n_tracers;
  a.rdx = (T)(g->Nx / g->Lx); a.rdy = (T)(g->Ny / g->Ly);
  for (int t = 0; t < kMaxTracers; ++t) a.cref[t] = m->off_cref[t] ? at<T>(m, m->off_cref[t]) : nullptr;
  a.closure = m->d.closure;
  a.nu0 = (T)m->d.nu; a.kappa0 = (T)m->d.kappa; a.inv_Pr = (T)(1.0 / m->d.Pr);
  a.f = (T)m->d.f;
  a.eos = m->d.eos;
  a.g_alpha = (T)(m->d.g * m->d.alpha); a.g_beta = (T)(m->d.g * m->d.beta); a.T0 = (T)m->d.T0; a.S0 = (T)m->d.S0;
  for (int n = 0; n < 2 + kMaxTracers; ++n) { a.top[n] = (T)m->d.top_flux[n]; a.bot[n] = (T)m->d.bottom_flux[n]; }
  a.dt_gamma = (T)dt_gamma; a.dt_zeta = (T)dt_zeta;
  a.mode = mode;
  a.variant = m->variant;
  a.nu_out = m->off_nu ? at<T>(m, m->off_nu) : nullptr;
  a.dzc = at<T>(m, m->off_dzc);
  a.dx = (T)(g->Lx / g->Nx); a.dy = (T)(g->Ly / g->Ny);
  a.Cs = (T)m->d.Cs; a.Cb = (T)m->d.Cb; a.C_amd = (T)m->d.C_amd;
  a.oob = at<unsigned>(m, m->off_oob);
  m->hook.pre(OCN_K_TENDENCY);
  cudaError_t e = launch_tendency<T>(a, m->R, m->stream);
  m->hook.post(OCN_K_TENDENCY);
  return e;
}

ColumnArgs column_args(const ocn_model* m, int which, double N2bg) {
  const ocn_grid* g = m->g;
  ColumnArgs c;
  memset(&c, 0, sizeof(c));
  StatePtrs<float> s = state_ptrs<float>(m, which);
  c.b = s.c[0]; c.cref = at<float>(m, m->off_cref[0]);
  c.u = s.u; c.v = s.v; c.w = s.w;
  c.rdzf = at<float>(m, m->off_rdzf); c.rdzc = at<float>(m, m->off_rdzc); c.dzf = at<float>(m, m->off_dzf);
  c.depth = at<float>(m, m->off_depth);
  c.nu = m->off_nu ? at<float>(m, m->off_nu) : nullptr;
  c.kap = m->off_kap[0] ? at<float>(m, m->off_kap[0]) : nullptr;
  c.closure = m->d.closure; c.nu0 = (float)m->d.nu; c.kappa0 = (float)m->d.kappa; c.inv_Pr = (float)(1.0 / m->d.Pr);
  c.Nx = g->Nx; c.Ny = g->Ny; c.Nz = g->Nz;
  c.Jb = (float)m->d.top_flux[2]; c.f = (float)m->d.f; c.N2bg = (float)N2bg;
  c.h = at<float>(m, m->off_colh);
  return c;
}

// The learned closure's face fluxes for state `which` into F ([3][Nz+1][Ny][Nx] FP32).
cudaError_t enqueue_learned_flux(ocn_model* m, int which, float* F, int* nlaunch) {
  MlpClosureArgs a;
  memset(&a, 0, sizeof(a));
  a.col = column_args(m, which, m->colc_N2);
  if (!mlp_closure_layers(m->colc, a.W, a.bias)) return cudaErrorInvalidValue;
  for (int q = 0; q < kColumnFeatures; ++q) { a.mu[q] = m->colc_mu[q]; a.inv_sigma[q] = m->colc_isig[q]; }
  for (int q = 0; q < 3; ++q) a.scale[q] = m->colc_scale[q];
  a.relu = (m->colc_mode == 1) ? 1 : 0;
  a.F = F;
  a.status = at<int>(m, m->off_status);
  m->hook.pre(OCN_K_COLUMN_CLOSURE);
  cudaError_t e = launch_column_h(a.col, m->stream);
  if (e == cudaSuccess) e = launch_mlp_closure(a, m->stream);
  m->hook.post(OCN_K_COLUMN_CLOSURE);
  if (nlaunch) *nlaunch += 2;
  return e;
}

// Learned column closure after the tendency kernel: G += dG, and in mode 0 the new state
// += dt_gamma dG, with dG = -dF/dz of the learned face fluxes of the stage state.
template <typename T>
cudaError_t enqueue_column_closure(ocn_model* m, int which, double dt_gamma, int mode, int* nlaunch) {
  if constexpr (!std::is_same<T, float>::value) {
    return cudaSuccess;
  } else {
    if (!m->colc) return cudaSuccess;
    float* F = at<float>(m, m->off_colF);
    if (m->colc_mode == 1) {
      // diffusivities: their column means become the vertical diffusivity profiles of this
      // substage (tracers: output 0; momentum: output 1), applied by the implicit step that
      // follows; a tendency evaluation alone (mode 1) takes nothing from them
      if (mode == 1) return cudaSuccess;
      cudaError_t e = enqueue_learned_flux(m, which, F, nlaunch);
      if (e != cudaSuccess) return e;
      FaceMeanArgs fm;
      fm.F = F;
      fm.p0 = at<float>(m, m->off_kapz);
      fm.p1 = at<float>(m, m->off_nuz);
      fm.Nx = m->g->Nx; fm.Ny = m->g->Ny; fm.Nz = m->g->Nz;
      m->hook.pre(OCN_K_COLUMN_CLOSURE);
      e = launch_face_mean(fm, m->stream);
      m->hook.post(OCN_K_COLUMN_CLOSURE);
      if (nlaunch) *nlaunch += 1;
      return e;
    }
    cudaError_t e = enqueue_learned_flux(m, which, F, nlaunch);
    if (e != cudaSuccess) return e;
    FaceFluxArgs f;
    memset(&f, 0, sizeof(f));
    StatePtrs<float> G = g_ptrs<float>(m), N = state_ptrs<float>(m, 1 - which);
    f.F = F;
    f.Gu = G.u; f.Gv = G.v; f.Gb = G.c[0];
    f.nu_ = N.u; f.nv = N.v; f.nb = N.c[0];
    f.rdzc = at<float>(m, m->off_rdzc);
    f.Nx = m->g->Nx; f.Ny = m->g->Ny; f.Nz = m->g->Nz; f.mode = mode;
    f.dt_gamma = (float)dt_gamma;
    m->hook.pre(OCN_K_COLUMN_CLOSURE);
    e = launch_apply_face_flux(f, m->stream);
    m->hook.post(OCN_K_COLUMN_CLOSURE);
    if (nlaunch) *nlaunch += 1;
    return e;
  }
}

// Vertical diffusion of the substage: explicit (G += D(stage state), new state += dt_gamma D) or
// semi-implicit (new state <- (I - dtau D)^{-1} new state); mode 1 (tendencies only) adds the
// explicit term to G and skips the implicit step.
template <typename T>
cudaError_t enqueue_vertical(ocn_model* m, int which, double dt_gamma, double dtau, int mode, int* nlaunch) {
  // a learned closure in diffusivity mode supplies both profiles every substage, applied implicitly
  const bool learned = m->colc && m->colc_mode == 1;
  const bool vnu = m->vnu || learned, vkap = m->vkap || learned, vimplicit = m->vimplicit || learned;
  if (!vnu && !vkap) return cudaSuccess;
  if (vimplicit && mode == 1) return cudaSuccess;
  VDiffArgs<T> a;
  memset(&a, 0, sizeof(a));
  StatePtrs<T> cur = state_ptrs<T>(m, which), nxt = state_ptrs<T>(m, 1 - which), G = g_ptrs<T>(m);
  a.qin[0] = cur.u; a.qin[1] = cur.v; a.qin[2] = cur.w;
  a.qout[0] = nxt.u; a.qout[1] = nxt.v; a.qout[2] = nxt.w;
  a.G[0] = G.u; a.G[1] = G.v; a.G[2] = G.w;
  for (int t = 0; t < m->d.n_tracers; ++t) {
    a.qin[3 + t] = cur.c[t]; a.qout[3 + t] = nxt.c[t]; a.G[3 + t] = G.c[t];
    a.cref[t] = at<T>(m, m->off_cref[t]);
  }
  a.nuz = at<T>(m, m->off_nuz); a.kapz = at<T>(m, m->off_kapz);
  a.dzc = at<T>(m, m->off_dzc); a.dzf = at<T>(m, m->off_dzf);
  a.Nx = m->g->Nx; a.Ny = m->g->Ny; a.Nz = m->g->Nz; a.nt = m->d.n_tracers;
  a.fields = (vnu ? 7 : 0) | (vkap ? (((1 << m->d.n_tracers) - 1) << 3) : 0);
  a.mode = mode;
  a.dt_gamma = (T)dt_gamma; a.dtau = (T)dtau;
  // the spectral work space is free between projections
  a.tab = at<T>(m, m->off_spec);
  a.tab_cap = 2 * (size_t)spec_row_stride(m->g->Nx / 2) * m->g->Ny * m->g->Nz;
  m->hook.pre(OCN_K_VERTICAL);
  cudaError_t e = launch_vertical_diffusion<T>(a, vimplicit, m->stream, nlaunch);
  m->hook.post(OCN_K_VERTICAL);
  return e;
}

cudaError_t check_sync(ocn_model* m, cudaError_t e) {
  if (e != cudaSuccess || !m->sync_check) return e;
  return cudaStreamSynchronize(m->stream);
}

// Enqueue one full time step starting from buffer `which` (three RK3 substages, or one QAB2 stage
// whose chi is -1/2 on the first step after the state was set); returns the final buffer.
template <typename T>
cudaError_t enqueue_step(ocn_model* m, double dt, int* which, int* nlaunch) {
  static const double gam[3] = {8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0};
  static const double zet[3] = {0.0, 17.0 / 60.0, 5.0 / 12.0};
  const bool qab2 = m->stepper == OCN_STEPPER_QAB2;
  const double chi = m->ab_started ? m->chi : -0.5;
  const int nst = qab2 ? 1 : 3;
  int n = 0;
  for (int st = 0; st < nst; ++st) {
    const double g = qab2 ? 1.5 + chi : gam[st], z = qab2 ? 0.5 + chi : zet[st];
    const double dtau = (g - z) * dt;
    cudaError_t e = check_sync(m, enqueue_closure<T>(m, *which, true));
    if (e != cudaSuccess) return e;
    if (m->off_nu && !tendency_computes_nu(m)) ++n;
    e = check_sync(m, enqueue_tendency<T>(m, *which, g * dt, z * dt, 0));
    if (e != cudaSuccess) return e;
    ++n;
    e = check_sync(m, enqueue_column_closure<T>(m, *which, g * dt, 0, &n));
    if (e != cudaSuccess) return e;
    e = check_sync(m, enqueue_vertical<T>(m, *which, g * dt, dtau, 0, &n));
    if (e != cudaSuccess) return e;
    int np = 0;
    e = check_sync(m, launch_projection<T>(poisson_args<T>(m, 1 - *which, dtau), m->stream, &np, m->hook));
    if (e != cudaSuccess) return e;
    n += np;
    *which = 1 - *which;
  }
  if (nlaunch) *nlaunch = n;
  return cudaSuccess;
}

void drop_graphs(ocn_model* m);

template <typename T>
ocn_status time_step_t(ocn_model* m, double dt, int nsteps) {
  const bool use_graph = m->graphs && m->stream != nullptr && !m->sync_check && !m->timing;
  for (int s = 0; s < nsteps; ++s) {
    if (!use_graph) {
      int w = m->cur, nl = 0;
      cudaError_t e = enqueue_step<T>(m, dt, &w, &nl);
      if (e != cudaSuccess) return cuda_fail(e, "time step launch");
      m->cur = w;
      m->launches_per_step = nl;
      if (m->stepper == OCN_STEPPER_QAB2) m->ab_started = true;
      continue;
    }
    uint64_t key;
    memcpy(&key, &dt, sizeof(key));
    const int gk = m->cur + 2 * (m->ab_started ? 1 : 0) + 4 * m->stepper;
    auto it = m->graph_cache.find({key, gk});
    cudaGraphExec_t exec = nullptr;
    int w = m->cur;
    if (it == m->graph_cache.end()) {
      if (m->graph_cache.size() >= kGraphCacheMax) {   // many time steps (adaptive dt): start over
        cudaError_t es = cudaStreamSynchronize(m->stream);
        if (es != cudaSuccess) return cuda_fail(es, "graph cache reset");
        drop_graphs(m);
      }
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return cuda_fail(e, "begin capture");
      int nl = 0;
      cudaError_t el = enqueue_step<T>(m, dt, &w, &nl);
      e = cudaStreamEndCapture(m->stream, &graph);
      if (el != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return cuda_fail(el, "capture step"); }
      if (e != cudaSuccess) return cuda_fail(e, "end capture");
      e = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
      m->graph_cache[{key, gk}] = exec;
      m->launches_per_step = nl;
    } else {
      exec = it->second;
      w = (m->cur + 3) & 1;
    }
    cudaError_t e = cudaGraphLaunch(exec, m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "graph launch");
    m->cur = w;
    if (m->stepper == OCN_STEPPER_QAB2) m->ab_started = true;
  }
  return OCN_OK;
}

void drop_graphs(ocn_model* m) {
  for (auto& kv : m->graph_cache) cudaGraphExecDestroy(kv.second);
  m->graph_cache.clear();
  ++m->graph_epoch;
}

void drop_events(ocn_model* m) {
  for (auto& r : m->recs) { m->ev_pool.push_back(r.a); m->ev_pool.push_back(r.b); }
  m->recs.clear();
}

bool field_valid(const ocn_model* m, int field) {
  if (field & OCN_FIELD_RAW) {
    const int f = field & ~OCN_FIELD_RAW;
    return f >= OCN_FIELD_TRACER0 && f < OCN_FIELD_TRACER0 + m->d.n_tracers;
  }
  if (field >= OCN_FIELD_TRACER_REF0 && field < OCN_FIELD_TRACER_REF0 + m->d.n_tracers) return true;
  if (field == OCN_FIELD_U || field == OCN_FIELD_V || field == OCN_FIELD_W || field == OCN_FIELD_P) return true;
  if (field >= OCN_FIELD_TRACER0 && field < OCN_FIELD_TRACER0 + m->d.n_tracers) return true;
  if (field >= OCN_FIELD_G && field < OCN_FIELD_G + m->nf) return true;
  if (field == OCN_FIELD_NU_E && m->off_nu) return true;
  return false;
}

char* field_ptr(const ocn_model* m, int field, size_t* elems) {
  field &= ~OCN_FIELD_RAW;
  if (field >= OCN_FIELD_TRACER_REF0 && field < OCN_FIELD_TRACER_REF0 + m->d.n_tracers) {
    *elems = (size_t)m->g->Nz;
    return m->arena + m->off_cref[field - OCN_FIELD_TRACER_REF0];
  }
  if (field >= OCN_FIELD_G && field < OCN_FIELD_G + m->nf) {
    *elems = field_elems(m, field - OCN_FIELD_G);
    return m->arena + m->off_G[field - OCN_FIELD_G];
  }
  if (field == OCN_FIELD_P) { *elems = field_elems(m, OCN_FIELD_U); return m->arena + m->off_p; }
  if (field == OCN_FIELD_NU_E) { *elems = field_elems(m, OCN_FIELD_U); return m->arena + m->off_nu; }
  *elems = field_elems(m, field);
  return m->arena + m->off_state[m->cur][field];
}

}  // namespace

extern "C" {

int ocn_abi_version(void) { return OCN_ABI_VERSION; }

const char* ocn_last_error(void) { return g_err.c_str(); }

ocn_status ocn_grid_create(const ocn_grid_desc* desc, ocn_grid** out) {
  if (!desc || !out) return fail(OCN_ERR_ARG, "null argument");
  *out = nullptr;
  if (desc->Nx < 4 || desc->Ny < 4 || (desc->Nx % 2) || (desc->Ny % 2) || !is_2a3b(desc->Nx) || !is_2a3b(desc->Ny))
    return fail(OCN_ERR_ARG, "Nx and Ny must be even, >= 4 and of the form 2^a 3^b");
  if ((long long)desc->Nx * desc->Ny > 2147483647LL)
    return fail(OCN_ERR_ARG, "Nx * Ny must be below 2^31 (kernels index a level with 32-bit offsets)");
  if (desc->Nz < 1) return fail(OCN_ERR_ARG, "Nz must be >= 1");
  if (!(desc->Lx > 0) || !(desc->Ly > 0)) return fail(OCN_ERR_ARG, "Lx and Ly must be positive");
  if (!desc->z_faces) return fail(OCN_ERR_ARG, "z_faces is null");
  for (int k = 0; k < desc->Nz; ++k)
    if (!(desc->z_faces[k + 1] > desc->z_faces[k])) return fail(OCN_ERR_ARG, "z_faces must be strictly ascending");
  ocn_grid* g = new (std::nothrow) ocn_grid;
  if (!g) return fail(OCN_ERR_OOM, "grid allocation");
  g->Nx = desc->Nx; g->Ny = desc->Ny; g->Nz = desc->Nz; g->Lx = desc->Lx; g->Ly = desc->Ly;
  g->zf.assign(desc->z_faces, desc->z_faces + desc->Nz + 1);
  g->zc.resize(g->Nz); g->dzc.resize(g->Nz); g->dzf.assign(g->Nz + 1, 0.0);
  for (int k = 0; k < g->Nz; ++k) { g->zc[k] = 0.5 * (g->zf[k] + g->zf[k + 1]); g->dzc[k] = g->zf[k + 1] - g->zf[k]; }
  for (int k = 1; k < g->Nz; ++k) g->dzf[k] = g->zc[k] - g->zc[k - 1];
  g->dzf[0] = g->dzc[0]; g->dzf[g->Nz] = g->dzc[g->Nz - 1];
  g->stretched = false;
  for (int k = 1; k < g->Nz; ++k)
    if (fabs(g->dzc[k] - g->dzc[0]) > 1e-12 * fabs(g->dzc[0])) g->stretched = true;
  *out = g;
  return OCN_OK;
}

void ocn_grid_destroy(ocn_grid* grid) { delete grid; }

ocn_status ocn_model_create(const ocn_grid* grid, const ocn_model_desc* desc, void* stream, ocn_model** out) {
  if (!grid || !desc || !out) return fail(OCN_ERR_ARG, "null argument");
  *out = nullptr;
  if (desc->precision != 32 && desc->precision != 64) return fail(OCN_ERR_ARG, "precision must be 32 or 64");
  if (desc->n_tracers < 1 || desc->n_tracers > OCN_MAX_TRACERS) return fail(OCN_ERR_ARG, "n_tracers must be 1..4");
  if (desc->closure < OCN_CLOSURE_NONE || desc->closure > OCN_CLOSURE_AMD) return fail(OCN_ERR_ARG, "unknown closure");
  if (desc->eos != OCN_EOS_BUOYANCY_TRACER && desc->eos != OCN_EOS_LINEAR_TS) return fail(OCN_ERR_ARG, "unknown eos");
  if (desc->eos == OCN_EOS_LINEAR_TS && desc->n_tracers < 2) return fail(OCN_ERR_ARG, "linear T,S EOS needs 2 tracers");
  if (desc->closure == OCN_CLOSURE_SMAGORINSKY && !(desc->Pr > 0)) return fail(OCN_ERR_ARG, "Pr must be positive");
  if (desc->weno_order != 5 && desc->weno_order != 9) return fail(OCN_ERR_UNSUPPORTED, "weno_order must be 5 or 9");
  if (desc->n_tracers > 2) return fail(OCN_ERR_UNSUPPORTED, "the CUDA tendency kernel is built for 1 or 2 tracers");
  ocn_model* m = new (std::nothrow) ocn_model;
  if (!m) return fail(OCN_ERR_OOM, "model allocation");
  m->g = grid;
  m->d = *desc;
  m->stream = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaGetDevice(&m->dev);
  if (e != cudaSuccess) { delete m; return cuda_fail(e, "cudaGetDevice"); }
  m->R = (desc->weno_order + 1) / 2;
  m->es = desc->precision / 8;
  m->nf = 3 + desc->n_tracers;
  m->fp64_piv = desc->fp64_pivots > 0 || (desc->fp64_pivots < 0 && grid->stretched);
  for (int t = 0; t < desc->n_tracers; ++t) m->cref_host[t].assign(grid->Nz, 0.0);
  m->px = make_plan(grid->Nx / 2);
  m->py = make_plan(grid->Ny);
  layout(m);
  *out = m;
  return OCN_OK;
}

void ocn_model_destroy(ocn_model* model) {
  if (!model) return;
  {
    DeviceGuard dg(model->dev);
    drop_graphs(model);
    cudaStreamSynchronize(model->stream);
    drop_events(model);
    for (cudaEvent_t e : model->ev_pool) cudaEventDestroy(e);
    model->ev_pool.clear();
    if (model->xfer) cudaStreamSynchronize(model->xfer);
    xfer_release(model);
  }
  delete model;
}

ocn_status ocn_model_arena_bytes(const ocn_model* model, size_t* bytes) {
  if (!model || !bytes) return fail(OCN_ERR_ARG, "null argument");
  *bytes = model->bytes;
  return OCN_OK;
}

ocn_status ocn_model_bind_arena(ocn_model* m, void* device_ptr, size_t bytes) {
  if (!m || !device_ptr) return fail(OCN_ERR_ARG, "null argument");
  if (bytes < m->bytes) return fail(OCN_ERR_ARG, "arena smaller than ocn_model_arena_bytes()");
  if (reinterpret_cast<uintptr_t>(device_ptr) % 256) return fail(OCN_ERR_ARG, "arena must be 256-byte aligned");
  DeviceGuard dg(m->dev);
  cudaError_t e = ensure_tables(m->dev);
  if (e != cudaSuccess) return cuda_fail(e, "upload reconstruction tables");
  drop_graphs(m);
  m->arena = reinterpret_cast<char*>(device_ptr);
  m->cur = 0;
  for (int t = 0; t < m->d.n_tracers; ++t) { m->cref_host[t].assign(m->g->Nz, 0.0); m->cref_pending[t] = false; }
  e = cudaMemsetAsync(m->arena, 0, m->bytes, m->stream);
  if (e != cudaSuccess) return cuda_fail(e, "clear arena");
  std::vector<char> blob = (m->es == 4) ? metrics_blob<float>(m) : metrics_blob<double>(m);
  e = cudaMemcpyAsync(m->arena + m->off_dzc, blob.data(), blob.size(), cudaMemcpyHostToDevice, m->stream);
  if (e != cudaSuccess) return cuda_fail(e, "upload metrics");
  // the projection's tridiagonal systems depend only on the grid: factor them once
  e = (m->es == 4) ? launch_tridiag_factor<float>(poisson_args<float>(m, 0, 1.0), m->stream)
                   : launch_tridiag_factor<double>(poisson_args<double>(m, 0, 1.0), m->stream);
  if (e != cudaSuccess) return cuda_fail(e, "tridiagonal factorisation");
  std::vector<float> depth;
  if (m->off_depth) {
    for (int k = 0; k <= m->g->Nz; ++k) depth.push_back((float)(m->g->zf[m->g->Nz] - m->g->zf[k]));
    e = cudaMemcpyAsync(m->arena + m->off_depth, depth.data(), depth.size() * sizeof(float), cudaMemcpyHostToDevice, m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "upload depths");
  }
  e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return cuda_fail(e, "bind synchronise");
  return OCN_OK;
}

}  // extern "C"

namespace {

// The work of setting one field that follows its copy into dst: the QAB2 restart flag, the host
// mirror of a reference profile set as is, the reference profile and anomaly of a tracer (its
// profile read back into the pinned staging array), and the wall faces of w.
ocn_status set_followup(ocn_model* m, int field, char* dst, size_t nbytes) {
  cudaError_t e = cudaSuccess;
  // QAB2 restarts with an Euler step after the state is set, and continues when G^{m-1} is restored
  m->ab_started = (field >= OCN_FIELD_G && field < OCN_FIELD_G + 3 + OCN_MAX_TRACERS);
  const int tr = (field & OCN_FIELD_RAW) ? -1 : field - OCN_FIELD_TRACER0;
  const int rf = field - OCN_FIELD_TRACER_REF0;
  if (rf >= 0 && rf < m->d.n_tracers) {   // a reference profile set as is: refresh the host mirror
    std::vector<char> hb(nbytes);
    e = cudaMemcpyAsync(hb.data(), dst, nbytes, cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "reference profile read");
    for (int k = 0; k < m->g->Nz; ++k)
      m->cref_host[rf][k] = (m->es == 4) ? (double)reinterpret_cast<float*>(hb.data())[k] : reinterpret_cast<double*>(hb.data())[k];
    m->cref_pending[rf] = false;
  }
  if (tr >= 0 && tr < m->d.n_tracers) {
    // new reference profile = the horizontal mean of each level; store the anomaly
    const size_t plane = (size_t)m->g->Nx * m->g->Ny;
    char* ref = m->arena + m->off_cref[tr];
    if (m->es == 4) {
      e = launch_level_mean<float>(reinterpret_cast<float*>(dst), plane, m->g->Nz, reinterpret_cast<float*>(ref), m->stream);
      if (e == cudaSuccess) e = launch_level_shift<float>(reinterpret_cast<float*>(dst), plane, m->g->Nz, reinterpret_cast<float*>(ref), -1.0f, m->stream);
    } else {
      e = launch_level_mean<double>(reinterpret_cast<double*>(dst), plane, m->g->Nz, reinterpret_cast<double*>(ref), m->stream);
      if (e == cudaSuccess) e = launch_level_shift<double>(reinterpret_cast<double*>(dst), plane, m->g->Nz, reinterpret_cast<double*>(ref), -1.0, m->stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "tracer reference profile");
    m->cref_pending[tr] = true;      // the host mirror is read back where it is used
  }
  if (field == OCN_FIELD_W || field == OCN_FIELD_G + OCN_FIELD_W) {
    size_t pb = (size_t)m->g->Nx * m->g->Ny * m->es;
    e = cudaMemsetAsync(dst, 0, pb, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(dst + (size_t)m->g->Nz * pb, 0, pb, m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "wall faces");
  }
  return OCN_OK;
}

// Set n fields: every copy first, back to back on the model stream, then the follow-up work of
// each field in order; from host memory the call returns once the copies are done (the host
// buffers are borrowed for them only).
ocn_status set_fields(ocn_model* m, int n, const int* fields, const void* const* srcs, const size_t* nbytes,
                      int src_is_device) {
  if (!m || n < 0 || (n > 0 && (!fields || !srcs || !nbytes))) return fail(OCN_ERR_ARG, "null argument");
  if (src_is_device < 0 || src_is_device > OCN_HOST_ASYNC) return fail(OCN_ERR_ARG, "src_is_device must be 0, 1 or OCN_HOST_ASYNC");
  if (!m->arena) return fail(OCN_ERR_STATE, "arena not bound");
  std::vector<char*> dst(n);
  for (int i = 0; i < n; ++i) {
    if (!srcs[i]) return fail(OCN_ERR_ARG, "null argument");
    if (!field_valid(m, fields[i]) || fields[i] == OCN_FIELD_NU_E) return fail(OCN_ERR_ARG, "invalid field id for set");
    size_t elems = 0;
    dst[i] = field_ptr(m, fields[i], &elems);
    if (nbytes[i] != elems * (size_t)m->es) return fail(OCN_ERR_ARG, "byte count does not match the field size");
  }
  DeviceGuard dg(m->dev);
  const bool host = src_is_device != 1;              // 0: host, waited for; OCN_HOST_ASYNC: host, not waited for
  cudaError_t e = cudaSuccess;
  if (host) {
    e = xfer_setup(m);
    if (e != cudaSuccess) return cuda_fail(e, "transfer stream");
  }
  for (int i = 0; i < n; ++i) {
    e = cudaMemcpyAsync(dst[i], srcs[i], nbytes[i], host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "set field copy");
  }
  if (host) {
    e = cudaEventRecord(m->copy_done, m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "set field copy event");
  }
  for (int i = 0; i < n; ++i) {
    const ocn_status st = set_followup(m, fields[i], dst[i], nbytes[i]);
    if (st != OCN_OK) return st;
  }
  if (src_is_device == 0) {
    e = cudaEventSynchronize(m->copy_done);   // the host buffers are only borrowed for the copies
    if (e != cudaSuccess) return cuda_fail(e, "set field synchronise");
  }
  return OCN_OK;
}

// Get n fields on the high-priority transfer stream, after the work queued on the model stream
// so far (the model stream's later work waits for it).  A tracer's full value (stored anomaly +
// reference profile) is formed in a work array first: the spectral work space for a single
// field; for several fields, tracer t's slot of the state buffer that is not current (it holds
// the stage state the last step no longer needs, and the next step overwrites it), so that every
// tracer's kernel runs before any copy.
ocn_status get_fields(ocn_model* m, int n, const int* fields, void* const* dsts, const size_t* nbytes,
                      int dst_is_device) {
  if (!m || n < 0 || (n > 0 && (!fields || !dsts || !nbytes))) return fail(OCN_ERR_ARG, "null argument");
  if (dst_is_device < 0 || dst_is_device > OCN_HOST_ASYNC) return fail(OCN_ERR_ARG, "dst_is_device must be 0, 1 or OCN_HOST_ASYNC");
  if (!m->arena) return fail(OCN_ERR_STATE, "arena not bound");
  std::vector<char*> src(n);
  for (int i = 0; i < n; ++i) {
    if (!dsts[i]) return fail(OCN_ERR_ARG, "null argument");
    if (!field_valid(m, fields[i])) return fail(OCN_ERR_ARG, "invalid field id");
    size_t elems = 0;
    src[i] = field_ptr(m, fields[i], &elems);
    if (nbytes[i] != elems * (size_t)m->es) return fail(OCN_ERR_ARG, "byte count does not match the field size");
  }
  DeviceGuard dg(m->dev);
  cudaError_t e = xfer_setup(m);
  if (e == cudaSuccess) e = cudaEventRecord(m->xfer_in, m->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(m->xfer, m->xfer_in, 0);
  if (e != cudaSuccess) return cuda_fail(e, "transfer stream");
  for (int i = 0; i < n; ++i) {
    const int tr = (fields[i] & OCN_FIELD_RAW) ? -1 : fields[i] - OCN_FIELD_TRACER0;
    if (tr < 0 || tr >= m->d.n_tracers) continue;
    // add the reference profile back in a work array
    char* scratch = (n == 1) ? m->arena + m->off_spec : m->arena + m->off_state[1 - m->cur][OCN_FIELD_TRACER0 + tr];
    const size_t plane = (size_t)m->g->Nx * m->g->Ny;
    const char* ref = m->arena + m->off_cref[tr];
    e = (m->es == 4) ? launch_level_add<float>(reinterpret_cast<float*>(scratch), reinterpret_cast<const float*>(src[i]), plane, m->g->Nz, reinterpret_cast<const float*>(ref), m->xfer)
                     : launch_level_add<double>(reinterpret_cast<double*>(scratch), reinterpret_cast<const double*>(src[i]), plane, m->g->Nz, reinterpret_cast<const double*>(ref), m->xfer);
    if (e != cudaSuccess) return cuda_fail(e, "tracer reference profile");
    src[i] = scratch;
  }
  for (int i = 0; i < n; ++i) {
    e = cudaMemcpyAsync(dsts[i], src[i], nbytes[i], dst_is_device == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, m->xfer);
    if (e != cudaSuccess) return cuda_fail(e, "get field copy");
  }
  e = cudaEventRecord(m->xfer_out, m->xfer);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(m->stream, m->xfer_out, 0);
  if (e != cudaSuccess) return cuda_fail(e, "get field copy");
  if (dst_is_device == 0) {
    e = cudaEventSynchronize(m->xfer_out);
    if (e != cudaSuccess) return cuda_fail(e, "get field synchronise");
  }
  return OCN_OK;
}

}  // namespace

extern "C" {

ocn_status ocn_set_field(ocn_model* m, int field, const void* src, size_t nbytes, int src_is_device) {
  if (!m || !src) return fail(OCN_ERR_ARG, "null argument");
  return set_fields(m, 1, &field, &src, &nbytes, src_is_device);
}

ocn_status ocn_get_field(ocn_model* m, int field, void* dst, size_t nbytes, int dst_is_device) {
  if (!m || !dst) return fail(OCN_ERR_ARG, "null argument");
  return get_fields(m, 1, &field, &dst, &nbytes, dst_is_device);
}

ocn_status ocn_set_fields(ocn_model* m, int n, const int* fields, const void* const* srcs, const size_t* nbytes,
                          int src_is_device) {
  return set_fields(m, n, fields, srcs, nbytes, src_is_device);
}

ocn_status ocn_get_fields(ocn_model* m, int n, const int* fields, void* const* dsts, const size_t* nbytes,
                          int dst_is_device) {
  return get_fields(m, n, fields, dsts, nbytes, dst_is_device);
}

ocn_status ocn_bounds_status(ocn_model* m, unsigned* status, int* checked) {
  if (!m || !status) return fail(OCN_ERR_ARG, "null argument");
  if (!m->arena) return fail(OCN_ERR_STATE, "arena not bound");
  if (checked) *checked = OCN_BOUNDS_CHECK;
  DeviceGuard dg(m->dev);
  unsigned v = 0;
  cudaError_t e = cudaStreamSynchronize(m->stream);
  if (e == cudaSuccess) e = cudaMemcpy(&v, m->arena + m->off_oob, sizeof(v), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->arena + m->off_oob, 0, sizeof(v), m->stream);
  if (e != cudaSuccess) return cuda_fail(e, "bounds status");
  *status = v;
  return OCN_OK;
}

ocn_status ocn_wait_transfers(ocn_model* m) {
  if (!m) return fail(OCN_ERR_ARG, "null argument");
  if (!m->xfer) return OCN_OK;                      // no host transfer issued yet
  DeviceGuard dg(m->dev);
  cudaError_t e = cudaEventSynchronize(m->copy_done);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->xfer);
  if (e != cudaSuccess) return cuda_fail(e, "wait for transfers");
  return OCN_OK;
}

ocn_status ocn_project(ocn_model* m) {
  if (!m) return fail(OCN_ERR_ARG, "null argument");
  if (!m->arena) return fail(OCN_ERR_STATE, "arena not bound");
  DeviceGuard dg(m->dev);
  cudaError_t e = (m->es == 4) ? launch_projection<float>(poisson_args<float>(m, m->cur, 1.0), m->stream, nullptr)
                               : launch_projection<double>(poisson_args<double>(m, m->cur, 1.0), m->stream, nullptr);
  e = check_sync(m, e);
  if (e != cudaSuccess) return cuda_fail(e, "projection");
  return OCN_OK;
}

ocn_status ocn_time_step(ocn_model* m, double dt, int nsteps) {
  if (!m) return fail(OCN_ERR_ARG, "null argument");
  if (!m->arena) return fail(OCN_ERR_STATE, "arena not bound");
  if (nsteps < 0 || !isfinite(dt)) return fail(OCN_ERR_ARG, "nsteps must be >= 0 and dt finite");
  DeviceGuard dg(m->dev);
  return (m->es == 4) ? time_step_t<float>(m, dt, nsteps) : time_step_t<double>(m, dt, nsteps);
}

ocn_status ocn_compute_tendencies(ocn_model* m) {
  if (!m) return fail(OCN_ERR_ARG, "null argument");
  if (!m->arena) return fail(OCN_ERR_STATE, "arena not bound");
  DeviceGuard dg(m->dev);
  cudaError_t e;
  if (m->es == 4) {
    e = check_sync(m, enqueue_closure<float>(m, m->cur, true));
    if (e == cudaSuccess) e = check_sync(m, enqueue_tendency<float>(m, m->cur, 0.0, 0.0, 1));
    if (e == cudaSuccess) e = check_sync(m, enqueue_column_closure<float>(m, m->cur, 0.0, 1, nullptr));
    if (e == cudaSuccess) e = check_sync(m, enqueue_vertical<float>(m, m->cur, 0.0, 0.0, 1, nullptr));
  } else {
    e = check_sync(m, enqueue_closure<double>(m, m->cur));
    if (e == cudaSuccess) e = check_sync(m, enqueue_tendency<double>(m, m->cur, 0.0, 0.0, 1));
    if (e == cudaSuccess) e = check_sync(m, enqueue_vertical<double>(m, m->cur, 0.0, 0.0, 1, nullptr));
  }
  if (e != cudaSuccess) return cuda_fail(e, "tendencies");
  return OCN_OK;
}

ocn_status ocn_diagnostics(ocn_model* m, double dt, double* out, int nout) {
  if (!m || !out) return fail(OCN_ERR_ARG, "null argument");
  if (!m->arena) return fail(OCN_ERR_STATE, "arena not bound");
  const int nt = m->d.n_tracers;
  if (nout < nt + 6) return fail(OCN_ERR_ARG, "nout must be >= n_tracers + 6");
  DeviceGuard dg(m->dev);
  const ocn_grid* g = m->g;
  cudaError_t e;
  auto fill = [&](auto tag) {
    typedef decltype(tag) T;
    DiagArgs<T> a;
    memset(&a, 0, sizeof(a));
    a.cur = state_ptrs<T>(m, m->cur);
    a.dzc = at<T>(m, m->off_dzc); a.dzf = at<T>(m, m->off_dzf); a.rdzc = at<T>(m, m->off_rdzc); a.rdzf = at<T>(m, m->off_rdzf);
    a.Nx = g->Nx; a.Ny = g->Ny; a.Nz = g->Nz; a.nt = nt;
    a.dx = (T)(g->Lx / g->Nx); a.dy = (T)(g->Ly / g->Ny); a.rdx = (T)(g->Nx / g->Lx); a.rdy = (T)(g->Ny / g->Ly);
    a.partial = at<double>(m, m->off_partial);
    a.out = at<double>(m, m->off_diag);
    a.nblocks = diag_blocks();
    return launch_diagnostics<T>(a, m->stream);
  };
  e = (m->es == 4) ? fill(0.0f) : fill(0.0);
  if (e != cudaSuccess) return cuda_fail(e, "diagnostics launch");
  double vals[OCN_MAX_TRACERS + 6];
  e = cudaMemcpyAsync(vals, m->arena + m->off_diag, sizeof(double) * (nt + 6), cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e == cudaSuccess) e = cref_refresh(m);
  if (e != cudaSuccess) return cuda_fail(e, "diagnostics read");
  for (int v = 0; v < nt + 6; ++v) out[v] = vals[v];
  for (int t = 0; t < nt; ++t)
    for (int k = 0; k < g->Nz; ++k) out[t] += m->cref_host[t][k] * g->Lx * g->Ly * g->dzc[k];
  out[nt + 4] *= dt;
  if (m->off_status) {
    int st = 0;
    e = cudaMemcpy(&st, m->arena + m->off_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "status read");
    if (st) return fail(OCN_ERR_TIMEOUT, "a bounded wait of the learned column closure gave up");
  }
  if (out[nt + 5] > 0 || !isfinite(out[nt + 3])) return fail(OCN_ERR_NONFINITE, "non-finite values in the state");
  if (out[nt + 4] > 1.0) return fail(OCN_ERR_CFL, "advective CFL number above 1");
  return OCN_OK;
}

ocn_status ocn_set_option(ocn_model* m, int option, long long value) {
  if (!m) return fail(OCN_ERR_ARG, "null argument");
  if (option == OCN_OPT_GRAPHS) { m->graphs = value != 0; return OCN_OK; }
  if (option == OCN_OPT_SYNC_CHECK) { m->sync_check = value != 0; return OCN_OK; }
  if (option == OCN_OPT_TENDENCY_VARIANT) {
    if (value < 0 || value >= kTendencyVariants) return fail(OCN_ERR_ARG, "tendency variant out of range");
    DeviceGuard dg(m->dev);
    if (m->variant != (int)value) drop_graphs(m);
    m->variant = (int)value;
    return OCN_OK;
  }
  if (option == OCN_OPT_KERNEL_TIMING) {
    DeviceGuard dg(m->dev);
    cudaStreamSynchronize(m->stream);
    drop_events(m);
    m->timing = value != 0;
    m->hook = LaunchHook();
    if (m->timing) { m->hook.before = hook_before; m->hook.after = hook_after; m->hook.ctx = m; }
    return OCN_OK;
  }
  return fail(OCN_ERR_ARG, "unknown option");
}

ocn_status ocn_autotune(ocn_model* m, int* best, double* ms) {
  if (!m) return fail(OCN_ERR_ARG, "null argument");
  if (!m->arena) return fail(OCN_ERR_STATE, "arena not bound");
  DeviceGuard dg(m->dev);
  const int nv = (m->es == 4) ? kTendencyVariants : 1;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return cuda_fail(e, "autotune events");
  const int saved = m->variant;
  const bool saved_timing = m->timing;
  const LaunchHook saved_hook = m->hook;
  m->timing = false;
  m->hook = LaunchHook();
  int arg = 0;
  float bestms = 1e30f;
  for (int v = 0; v < kTendencyVariants; ++v) {
    float t = 1e30f;
    if (v < nv) {
      m->variant = v;
      e = (m->es == 4) ? enqueue_tendency<float>(m, m->cur, 0.0, 0.0, 1) : enqueue_tendency<double>(m, m->cur, 0.0, 0.0, 1);
      if (e == cudaSuccess) e = cudaEventRecord(e0, m->stream);
      for (int r = 0; r < 2 && e == cudaSuccess; ++r)
        e = (m->es == 4) ? enqueue_tendency<float>(m, m->cur, 0.0, 0.0, 1) : enqueue_tendency<double>(m, m->cur, 0.0, 0.0, 1);
      if (e == cudaSuccess) e = cudaEventRecord(e1, m->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
      if (e != cudaSuccess) break;
      t *= 0.5f;
      if (t < bestms) { bestms = t; arg = v; }
    }
    if (ms) ms[v] = (v < nv) ? (double)t : -1.0;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  m->timing = saved_timing;
  m->hook = saved_hook;
  if (e != cudaSuccess) { m->variant = saved; return cuda_fail(e, "autotune"); }
  if (arg != saved) drop_graphs(m);
  m->variant = arg;
  m->ab_started = false;            // G was overwritten: QAB2 restarts with its Euler step
  if (best) *best = arg;
  return OCN_OK;
}

ocn_status ocn_profiles(ocn_model* m, double* out, int nout) {
  if (!m || !out) return fail(OCN_ERR_ARG, "null argument");
  if (!m->arena) return fail(OCN_ERR_STATE, "arena not bound");
  const ocn_grid* g = m->g;
  const int Nz = g->Nz;
  if (nout < 3 * Nz + 3 * (Nz + 1)) return fail(OCN_ERR_ARG, "nout must be >= 3*Nz + 3*(Nz+1)");
  if ((size_t)7 * Nz > (size_t)diag_blocks() * (OCN_MAX_TRACERS + 6)) return fail(OCN_ERR_UNSUPPORTED, "Nz too large for profiles");
  DeviceGuard dg(m->dev);
  cudaError_t e;
  auto run = [&](auto tag) -> cudaError_t {
    typedef decltype(tag) T;
    cudaError_t err = enqueue_closure<T>(m, m->cur, true);
    if (err == cudaSuccess) err = enqueue_tendency<T>(m, m->cur, 0.0, 0.0, 1);   // unsplit G, state untouched
    if (err == cudaSuccess) err = enqueue_column_closure<T>(m, m->cur, 0.0, 1, nullptr);
    if (err == cudaSuccess) err = enqueue_vertical<T>(m, m->cur, 0.0, 0.0, 1, nullptr);
    if (err != cudaSuccess) return err;
    ProfileArgs<T> pa;
    memset(&pa, 0, sizeof(pa));
    StatePtrs<T> G = g_ptrs<T>(m), S = state_ptrs<T>(m, m->cur);
    pa.Gu = G.u; pa.Gv = G.v; pa.Gc0 = G.c[0]; pa.Gc1 = (m->d.n_tracers > 1) ? G.c[1] : nullptr;
    pa.u = S.u; pa.v = S.v; pa.c0 = S.c[0]; pa.c1 = (m->d.n_tracers > 1) ? S.c[1] : nullptr;
    pa.cref0 = at<T>(m, m->off_cref[0]); pa.cref1 = (m->d.n_tracers > 1) ? at<T>(m, m->off_cref[1]) : nullptr;
    pa.plane = (size_t)g->Nx * g->Ny; pa.Nz = Nz; pa.eos = m->d.eos;
    pa.g_alpha = m->d.g * m->d.alpha; pa.g_beta = m->d.g * m->d.beta; pa.T0 = m->d.T0; pa.S0 = m->d.S0;
    pa.out = at<double>(m, m->off_partial);
    return launch_profile_means<T>(pa, m->stream);
  };
  e = (m->es == 4) ? run(0.0f) : run(0.0);
  if (e != cudaSuccess) return cuda_fail(e, "profiles launch");
  std::vector<double> mean((size_t)7 * Nz);
  e = cudaMemcpyAsync(mean.data(), m->arena + m->off_partial, mean.size() * sizeof(double), cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return cuda_fail(e, "profiles read");
  const double* mGu = &mean[0]; const double* mGv = &mean[Nz]; const double* mG0 = &mean[2 * Nz];
  const double* mG1 = &mean[3 * Nz]; const double* mu = &mean[4 * Nz]; const double* mv = &mean[5 * Nz];
  const double* mb = &mean[6 * Nz];
  for (int k = 0; k < Nz; ++k) { out[k] = mb[k]; out[Nz + k] = mu[k]; out[2 * Nz + k] = mv[k]; }
  // mean face fluxes from the mean budget, integrated up from the bottom wall:
  // <G_c> = -(F_{k+1} - F_k)/dz_c;  <G_u> = -(...)/dz_c + f <v>;  <G_v> = -(...)/dz_c - f <u>
  double* Fb = out + 3 * Nz; double* Fu = Fb + (Nz + 1); double* Fv = Fu + (Nz + 1);
  const double f = m->d.f;
  double F0 = m->d.bottom_flux[2], F1 = m->d.bottom_flux[3];
  Fu[0] = m->d.bottom_flux[0]; Fv[0] = m->d.bottom_flux[1];
  const bool ts = m->d.eos == OCN_EOS_LINEAR_TS;
  const double ga = m->d.g * m->d.alpha, gb = m->d.g * m->d.beta;
  Fb[0] = ts ? ga * F0 - gb * F1 : F0;
  for (int k = 0; k < Nz; ++k) {
    const double dz = g->dzc[k];
    Fu[k + 1] = Fu[k] - dz * (mGu[k] - f * mv[k]);
    Fv[k + 1] = Fv[k] - dz * (mGv[k] + f * mu[k]);
    F0 -= dz * mG0[k];
    if (ts) F1 -= dz * mG1[k];
    Fb[k + 1] = ts ? ga * F0 - gb * F1 : F0;
  }
  return OCN_OK;
}

ocn_status ocn_set_time_stepper(ocn_model* m, int scheme, double chi) {
  if (!m) return fail(OCN_ERR_ARG, "null argument");
  if (scheme != OCN_STEPPER_RK3 && scheme != OCN_STEPPER_QAB2) return fail(OCN_ERR_ARG, "unknown time stepper");
  if (!isfinite(chi)) return fail(OCN_ERR_ARG, "chi must be finite");
  DeviceGuard dg(m->dev);
  m->stepper = scheme;
  m->chi = chi;
  m->ab_started = false;
  drop_graphs(m);
  return OCN_OK;
}

ocn_status ocn_set_vertical_diffusivity(ocn_model* m, const double* nu_faces, const double* kappa_faces, int implicit) {
  if (!m) return fail(OCN_ERR_ARG, "null argument");
  if (!m->arena) return fail(OCN_ERR_STATE, "arena not bound");
  const int n = m->g->Nz + 1;
  for (const double* p : {nu_faces, kappa_faces})
    if (p)
      for (int k = 0; k < n; ++k)
        if (!(p[k] >= 0.0) || !isfinite(p[k])) return fail(OCN_ERR_ARG, "diffusivities must be finite and >= 0");
  if (implicit && 4 * (size_t)m->es * m->g->Nz > 48 * 1024) return fail(OCN_ERR_UNSUPPORTED, "Nz too large for the implicit solver");
  if (m->colc_mode == 1 && (nu_faces || kappa_faces))
    return fail(OCN_ERR_STATE, "the learned column closure (diffusivity mode) sets the profiles");
  DeviceGuard dg(m->dev);
  std::vector<char> buf((size_t)n * m->es);
  auto upload = [&](const double* p, size_t off) -> cudaError_t {
    for (int k = 0; k < n; ++k) {
      if (m->es == 4) reinterpret_cast<float*>(buf.data())[k] = (float)p[k];
      else reinterpret_cast<double*>(buf.data())[k] = p[k];
    }
    cudaError_t e = cudaMemcpyAsync(m->arena + off, buf.data(), buf.size(), cudaMemcpyHostToDevice, m->stream);
    return e == cudaSuccess ? cudaStreamSynchronize(m->stream) : e;
  };
  cudaError_t e = cudaSuccess;
  if (nu_faces) e = upload(nu_faces, m->off_nuz);
  if (e == cudaSuccess && kappa_faces) e = upload(kappa_faces, m->off_kapz);
  if (e != cudaSuccess) return cuda_fail(e, "vertical diffusivity upload");
  m->vnu = nu_faces != nullptr;
  m->vkap = kappa_faces != nullptr;
  m->vimplicit = implicit != 0;
  drop_graphs(m);
  return OCN_OK;
}

ocn_status ocn_set_column_closure(ocn_model* m, const ocn_mlp* mlp, const ocn_column_closure_desc* d) {
  if (!m) return fail(OCN_ERR_ARG, "null argument");
  if (!m->arena) return fail(OCN_ERR_STATE, "arena not bound");
  if (mlp) {
    if (!m->off_colF) return fail(OCN_ERR_UNSUPPORTED, "the learned column closure needs an FP32 buoyancy-tracer model");
    if (!d) return fail(OCN_ERR_ARG, "null closure descriptor");
    const void* W[4];
    const float* b[4];
    if (!mlp_closure_layers(mlp, W, b)) return fail(OCN_ERR_UNSUPPORTED, "the network must be 32-128-128-128-16 with a bound arena");
    for (int q = 0; q < kColumnFeatures; ++q)
      if (!(d->sigma[q] > 0.0f) || !isfinite(d->mu[q])) return fail(OCN_ERR_ARG, "sigma must be positive, mu finite");
    for (int q = 0; q < kColumnFeatures; ++q) { m->colc_mu[q] = d->mu[q]; m->colc_isig[q] = 1.0f / d->sigma[q]; }
    for (int q = 0; q < 3; ++q) m->colc_scale[q] = d->out_scale[q];
    m->colc_N2 = d->N2_background;
  }
  DeviceGuard dg(m->dev);
  m->colc = mlp;
  m->colc_version += 1;
  drop_graphs(m);
  return OCN_OK;
}

ocn_status ocn_set_column_closure_mode(ocn_model* m, int mode) {
  if (!m) return fail(OCN_ERR_ARG, "null argument");
  if (mode != 0 && mode != 1) return fail(OCN_ERR_ARG, "mode must be 0 (face fluxes) or 1 (diffusivities)");
  if (mode == 1 && !m->off_colF) return fail(OCN_ERR_UNSUPPORTED, "the learned column closure needs an FP32 buoyancy-tracer model");
  if (mode == 1 && (m->vnu || m->vkap)) return fail(OCN_ERR_STATE, "the model has its own vertical diffusivity profiles");
  DeviceGuard dg(m->dev);
  if (mode != m->colc_mode) {
    m->colc_mode = mode;
    m->colc_version += 1;
    drop_graphs(m);
  }
  return OCN_OK;
}

ocn_status ocn_closure_features(ocn_model* m, double N2_background, float* X) {
  if (!m || !X) return fail(OCN_ERR_ARG, "null argument");
  if (!m->arena) return fail(OCN_ERR_STATE, "arena not bound");
  if (!m->off_colF) return fail(OCN_ERR_UNSUPPORTED, "column features need an FP32 buoyancy-tracer model");
  DeviceGuard dg(m->dev);
  cudaError_t e = launch_closure_features(column_args(m, m->cur, N2_background), X, m->stream);
  if (e != cudaSuccess) return cuda_fail(e, "features");
  return OCN_OK;
}

ocn_status ocn_column_fluxes(ocn_model* m, int which, float* F) {
  if (!m || !F) return fail(OCN_ERR_ARG, "null argument");
  if (!m->arena) return fail(OCN_ERR_STATE, "arena not bound");
  if (!m->off_colF) return fail(OCN_ERR_UNSUPPORTED, "column fluxes need an FP32 buoyancy-tracer model");
  DeviceGuard dg(m->dev);
  cudaError_t e;
  if (which == 0) {
    e = enqueue_closure<float>(m, m->cur);
    if (e == cudaSuccess) e = launch_column_sgs_flux(column_args(m, m->cur, 0.0), F, m->stream);
  } else if (which == 1) {
    if (!m->colc) return fail(OCN_ERR_STATE, "no learned column closure set");
    e = enqueue_learned_flux(m, m->cur, F, nullptr);
  } else {
    return fail(OCN_ERR_ARG, "which must be 0 (closure) or 1 (learned)");
  }
  if (e != cudaSuccess) return cuda_fail(e, "column fluxes");
  return OCN_OK;
}

ocn_status ocn_coarse_grain(ocn_model* m, int cx, int cy, double* out, size_t nout) {
  if (!m || !out) return fail(OCN_ERR_ARG, "null argument");
  if (!m->arena) return fail(OCN_ERR_STATE, "arena not bound");
  if (!m->off_colF) return fail(OCN_ERR_UNSUPPORTED, "coarse-graining needs an FP32 buoyancy-tracer model");
  const ocn_grid* g = m->g;
  if (cx < 1 || cy < 1 || g->Nx % cx || g->Ny % cy) return fail(OCN_ERR_ARG, "cx, cy must divide Nx, Ny");
  const size_t need = (size_t)cx * cy * (7 * (size_t)g->Nz + 4);
  if (nout < need) return fail(OCN_ERR_ARG, "out too small: cx*cy*(7*Nz+4) doubles");
  DeviceGuard dg(m->dev);
  cudaError_t e = enqueue_closure<float>(m, m->cur);
  if (e == cudaSuccess) e = launch_coarse_grain(column_args(m, m->cur, 0.0), cx, cy, out, m->stream);
  if (e != cudaSuccess) return cuda_fail(e, "coarse grain");
  return OCN_OK;
}

ocn_status ocn_regrid(const double* zf_in, int nin, const double* in, const double* zf_out, int nout, double* out) {
  if (!zf_in || !in || !zf_out || !out || nin < 1 || nout < 1) return fail(OCN_ERR_ARG, "invalid regrid arguments");
  for (int i = 0; i < nin; ++i)
    if (!(zf_in[i + 1] > zf_in[i])) return fail(OCN_ERR_ARG, "input faces must ascend");
  for (int j = 0; j < nout; ++j)
    if (!(zf_out[j + 1] > zf_out[j])) return fail(OCN_ERR_ARG, "output faces must ascend");
  // one sweep over both face lists: each input cell contributes value x overlap to the output
  // cells it intersects
  int i = 0;
  for (int j = 0; j < nout; ++j) {
    const double lo = zf_out[j], hi = zf_out[j + 1];
    while (i < nin && zf_in[i + 1] <= lo) ++i;
    double acc = 0.0;
    for (int c = i; c < nin && zf_in[c] < hi; ++c) {
      const double a = fmax(zf_in[c], lo), b = fmin(zf_in[c + 1], hi);
      if (b > a) acc += in[c] * (b - a);
    }
    out[j] = acc / (hi - lo);
  }
  return OCN_OK;
}

// ------------------------------------------------------------------------------------------
// Ensembles: many independent members stepped together.
}  // extern "C"

namespace {
void clear_graphs(ocn_ensemble* e) {
  for (auto& kv : e->graphs) cudaGraphExecDestroy(kv.second);
  e->graphs.clear();
  for (auto& kv : e->graph_tables) cudaFree(kv.second);
  e->graph_tables.clear();
}
}  // namespace

extern "C" {

ocn_status ocn_ensemble_create(int n, const ocn_grid_desc* grids, const ocn_model_desc* models, void* stream,
                               ocn_ensemble** out) {
  if (!grids || !models || !out || n < 1) return fail(OCN_ERR_ARG, "invalid ensemble arguments");
  *out = nullptr;
  ocn_ensemble* e = new (std::nothrow) ocn_ensemble;
  if (!e) return fail(OCN_ERR_OOM, "ensemble allocation");
  e->n = n;
  e->stream = reinterpret_cast<cudaStream_t>(stream);
  cudaGetDevice(&e->dev);
  ocn_status st = OCN_OK;
  for (int i = 0; i < n && st == OCN_OK; ++i) {
    if (models[i].precision != models[0].precision) { st = fail(OCN_ERR_ARG, "members must share one precision"); break; }
    ocn_grid* g = nullptr;
    st = ocn_grid_create(&grids[i], &g);
    if (st != OCN_OK) break;
    e->grids.push_back(g);
    ocn_model* m = nullptr;
    st = ocn_model_create(g, &models[i], stream, &m);
    if (st != OCN_OK) break;
    e->models.push_back(m);
  }
  if (st != OCN_OK) { ocn_ensemble_destroy(e); return st; }
  e->es = e->models[0]->es;
  size_t o = 0;
  for (ocn_model* m : e->models) { e->offs.push_back(o); o = align256(o + m->bytes); }
  e->bytes = o;
  cudaError_t ce = cudaEventCreateWithFlags(&e->fork, cudaEventDisableTiming);
  for (int i = 0; i < n && ce == cudaSuccess; ++i) {
    cudaStream_t fs = nullptr;
    ce = cudaStreamCreateWithFlags(&fs, cudaStreamNonBlocking);
    if (ce != cudaSuccess) break;
    e->fork_streams.push_back(fs);
    cudaEvent_t ev = nullptr;
    ce = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (ce != cudaSuccess) break;
    e->join.push_back(ev);
  }
  if (ce != cudaSuccess) { ocn_ensemble_destroy(e); return cuda_fail(ce, "ensemble streams"); }
  *out = e;
  return OCN_OK;
}

void ocn_ensemble_destroy(ocn_ensemble* e) {
  if (!e) return;
  {
    DeviceGuard dg(e->dev);
    clear_graphs(e);
    for (cudaStream_t fs : e->fork_streams) cudaStreamDestroy(fs);
    for (cudaEvent_t ev : e->join) cudaEventDestroy(ev);
    if (e->fork) cudaEventDestroy(e->fork);
  }
  for (ocn_model* m : e->models) ocn_model_destroy(m);
  for (ocn_grid* g : e->grids) ocn_grid_destroy(g);
  delete e;
}

ocn_status ocn_ensemble_arena_bytes(const ocn_ensemble* e, size_t* bytes) {
  if (!e || !bytes) return fail(OCN_ERR_ARG, "null argument");
  *bytes = e->bytes;
  return OCN_OK;
}

ocn_status ocn_ensemble_bind_arena(ocn_ensemble* e, void* device_ptr, size_t bytes) {
  if (!e || !device_ptr) return fail(OCN_ERR_ARG, "null argument");
  if (bytes < e->bytes) return fail(OCN_ERR_ARG, "arena smaller than ocn_ensemble_arena_bytes()");
  if (reinterpret_cast<uintptr_t>(device_ptr) % 256) return fail(OCN_ERR_ARG, "arena must be 256-byte aligned");
  clear_graphs(e);
  e->arena = reinterpret_cast<char*>(device_ptr);
  for (int i = 0; i < e->n; ++i) {
    ocn_status st = ocn_model_bind_arena(e->models[i], e->arena + e->offs[i], e->models[i]->bytes);
    if (st != OCN_OK) return st;
  }
  return OCN_OK;
}

ocn_status ocn_ensemble_member(ocn_ensemble* e, int i, ocn_model** out) {
  if (!e || !out || i < 0 || i >= e->n) return fail(OCN_ERR_ARG, "invalid member index");
  *out = e->models[i];
  return OCN_OK;
}

}  // extern "C"

namespace {

// Batched ensemble step (OCN_ENSEMBLE_BATCHED).  Every member's step is first recorded (the
// launch functions append their kernels and arguments instead of launching); members whose
// kernel sequences agree form a group, and each kernel of a group's sequence becomes one launch
// of its batched form over the group's members (work list: member m owns a contiguous range of
// the flattened blocks).  A group is split into up to e->branches branches of about equal cell
// counts; branches run concurrently.
struct BatchLaunch {
  const void* fn;
  dim3 grid, block;
  size_t smem;
  int carveout;
  int n;                                // members in the launch
  unsigned stride;                      // payload bytes per member
  size_t start_off, dims_off, payload_off;   // byte offsets of the work-list parts in the table buffer
  int branch;
};
struct BatchPlan {
  std::vector<BatchLaunch> launches;
  int nbranch = 0;
  void* dtab = nullptr;                 // device copy of the work lists (owned by the plan's user)
};

// Record each member's launches: enqueue(m) runs with the recorder active, hooks and per-launch
// synchronisation off.
template <class F>
ocn_status record_members(ocn_ensemble* e, std::vector<LaunchRecorder>& recs, F enqueue) {
  recs.assign(e->n, LaunchRecorder());
  for (int i = 0; i < e->n; ++i) {
    ocn_model* m = e->models[i];
    const LaunchHook hook = m->hook;
    const bool sc = m->sync_check;
    m->hook = LaunchHook();
    m->sync_check = false;
    active_recorder() = &recs[i];
    cudaError_t el = enqueue(i, m);
    active_recorder() = nullptr;
    m->hook = hook;
    m->sync_check = sc;
    if (el != cudaSuccess) return cuda_fail(el, "ensemble launch record");
  }
  return OCN_OK;
}

// Group, split into branches, build and upload the work lists.
ocn_status plan_batched(ocn_ensemble* e, const std::vector<LaunchRecorder>& recs, BatchPlan* plan) {
  const int n = e->n;
  std::map<std::string, std::vector<int>> groups;
  std::vector<std::string> order;
  for (int i = 0; i < n; ++i) {
    std::string k;
    for (const LaunchRecord& r : recs[i].list) {
      const unsigned vals[5] = {r.block.x, r.block.y, r.block.z, (unsigned)r.persistent, (unsigned)r.payload.size()};
      k.append(reinterpret_cast<const char*>(&r.fn), sizeof(r.fn));
      k.append(reinterpret_cast<const char*>(vals), sizeof(vals));
    }
    if (!groups.count(k)) order.push_back(k);
    groups[k].push_back(i);
  }
  // split every group into up to e->branches branches of about equal cell counts (largest member
  // first onto the lightest branch); each branch is one chain of batched launches
  std::vector<std::vector<int>> branch_members;
  for (const std::string& k : order) {
    std::vector<int> mem = groups[k];
    const int nb = std::min<int>(e->branches, (int)mem.size());
    auto cells = [&](int i) { const ocn_grid* g = e->models[i]->g; return (double)g->Nx * g->Ny * g->Nz; };
    std::stable_sort(mem.begin(), mem.end(), [&](int a, int b) { return cells(a) > cells(b); });
    std::vector<std::vector<int>> br(nb);
    std::vector<double> load(nb, 0.0);
    for (int i : mem) {
      const int b = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      br[b].push_back(i);
      load[b] += cells(i);
    }
    for (auto& b : br) {
      std::sort(b.begin(), b.end());
      branch_members.push_back(b);
    }
  }
  // one batched launch per (branch, position, members sharing the launch's shared arguments)
  std::vector<unsigned char> host;
  auto reserve = [&](size_t bytes) { size_t o = (host.size() + 255) / 256 * 256; host.resize(o + bytes); return o; };
  plan->launches.clear();
  plan->nbranch = (int)branch_members.size();
  for (size_t gi = 0; gi < branch_members.size(); ++gi) {
    const std::vector<int>& mem = branch_members[gi];
    const size_t npos = recs[mem[0]].list.size();
    for (size_t p = 0; p < npos; ++p) {
      std::map<std::vector<unsigned char>, std::vector<int>> sub;
      std::vector<const std::vector<unsigned char>*> sub_order;
      for (int i : mem) {
        const LaunchRecord& r = recs[i].list[p];
        auto it = sub.find(r.shared);
        if (it == sub.end()) { sub_order.push_back(&r.shared); sub[r.shared].push_back(i); }
        else it->second.push_back(i);
      }
      for (const auto* sk : sub_order) {
        const std::vector<int>& ms = sub[*sk];
        const LaunchRecord& r0 = recs[ms[0]].list[p];
        BatchLaunch L;
        L.fn = r0.fn; L.block = r0.block; L.smem = 0; L.carveout = r0.carveout;
        L.n = (int)ms.size(); L.branch = (int)gi;
        L.stride = (unsigned)r0.payload.size();
        L.start_off = reserve(sizeof(unsigned) * (ms.size() + 1));
        L.dims_off = reserve(sizeof(uint3) * ms.size());
        L.payload_off = reserve((size_t)L.stride * ms.size());
        unsigned total = 0;
        for (size_t q = 0; q < ms.size(); ++q) {
          const LaunchRecord& r = recs[ms[q]].list[p];
          const uint3 d = make_uint3(r.grid.x, r.grid.y, r.grid.z);
          memcpy(host.data() + L.start_off + q * sizeof(unsigned), &total, sizeof(unsigned));
          memcpy(host.data() + L.dims_off + q * sizeof(uint3), &d, sizeof(uint3));
          memcpy(host.data() + L.payload_off + q * L.stride, r.payload.data(), L.stride);
          total += d.x * d.y * d.z;
          L.smem = std::max(L.smem, r.smem);
        }
        memcpy(host.data() + L.start_off + ms.size() * sizeof(unsigned), &total, sizeof(unsigned));
        unsigned blocks = total;
        if (r0.persistent > 0) {
          blocks = (total + (unsigned)r0.per_block - 1) / (unsigned)r0.per_block;
          if (blocks > (unsigned)r0.persistent) blocks = (unsigned)r0.persistent;
          if (blocks == 0) blocks = 1;
        }
        L.grid = dim3(blocks);
        plan->launches.push_back(L);
      }
    }
  }
  cudaError_t ce = cudaMalloc(&plan->dtab, std::max<size_t>(host.size(), 256));
  if (ce != cudaSuccess) { plan->dtab = nullptr; return cuda_fail(ce, "ensemble work lists"); }
  ce = cudaMemcpy(plan->dtab, host.data(), host.size(), cudaMemcpyHostToDevice);
  for (const BatchLaunch& L : plan->launches) {
    if (ce != cudaSuccess) break;
    ce = raise_smem_limit(L.fn, L.smem);
    if (ce == cudaSuccess && L.carveout >= 0)
      ce = cudaFuncSetAttribute(L.fn, cudaFuncAttributePreferredSharedMemoryCarveout, L.carveout);
  }
  if (ce != cudaSuccess) { cudaFree(plan->dtab); plan->dtab = nullptr; return cuda_fail(ce, "ensemble work lists"); }
  return OCN_OK;
}

// Enqueue the plan's launches: fork from e->stream, a chain per branch, join back.
cudaError_t enqueue_batched(ocn_ensemble* e, const BatchPlan& plan) {
  const unsigned char* base = static_cast<const unsigned char*>(plan.dtab);
  cudaError_t el = cudaEventRecord(e->fork, e->stream);
  for (int gi = 0; gi < plan.nbranch && el == cudaSuccess; ++gi) {
    cudaStream_t fs = e->fork_streams[gi];
    el = cudaStreamWaitEvent(fs, e->fork, 0);
    for (const BatchLaunch& L : plan.launches) {
      if (L.branch != gi || el != cudaSuccess) continue;
      BatchTable t;
      t.start = reinterpret_cast<const unsigned*>(base + L.start_off);
      t.dims = reinterpret_cast<const uint3*>(base + L.dims_off);
      t.payload = base + L.payload_off;
      t.stride = L.stride;
      t.n = L.n;
      void* args[] = {&t};
      el = cudaLaunchKernel(L.fn, L.grid, L.block, args, L.smem, fs);
    }
    if (el == cudaSuccess) el = cudaEventRecord(e->join[gi], fs);
    if (el == cudaSuccess) el = cudaStreamWaitEvent(e->stream, e->join[gi], 0);
  }
  return el;
}

template <typename T>
ocn_status build_batched_graph(ocn_ensemble* e, double dt, std::vector<int>& w, cudaGraphExec_t* out_exec,
                               void** out_tables, int* out_launches) {
  std::vector<LaunchRecorder> recs;
  ocn_status st = record_members(e, recs, [&](int i, ocn_model* m) {
    w[i] = m->cur;
    int nl = 0;
    return enqueue_step<T>(m, dt, &w[i], &nl);
  });
  if (st != OCN_OK) return st;
  BatchPlan plan;
  st = plan_batched(e, recs, &plan);
  if (st != OCN_OK) return st;
  cudaError_t ce = cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal);
  if (ce != cudaSuccess) { cudaFree(plan.dtab); return cuda_fail(ce, "ensemble begin capture"); }
  cudaError_t el = enqueue_batched(e, plan);
  cudaGraph_t graph = nullptr;
  ce = cudaStreamEndCapture(e->stream, &graph);
  if (el != cudaSuccess || ce != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaFree(plan.dtab);
    return cuda_fail(el != cudaSuccess ? el : ce, "ensemble batched capture");
  }
  cudaGraphExec_t exec = nullptr;
  ce = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) { cudaFree(plan.dtab); return cuda_fail(ce, "ensemble graph instantiate"); }
  *out_exec = exec;
  *out_tables = plan.dtab;
  *out_launches = (int)plan.launches.size();
  return OCN_OK;
}

template <typename T>
ocn_status ensemble_step_t(ocn_ensemble* e, double dt, int nsteps) {
  for (ocn_model* m : e->models) if (!m->arena) return fail(OCN_ERR_STATE, "arena not bound");
  if (e->mode == OCN_ENSEMBLE_SEQUENTIAL) {   // every member on the ensemble stream in turn
    for (int s = 0; s < nsteps; ++s) {
      int total = 0;
      for (ocn_model* m : e->models) {
        ocn_status st = time_step_t<T>(m, dt, 1);
        if (st != OCN_OK) return st;
        total += m->launches_per_step;
      }
      e->launches_per_step = total;
    }
    return OCN_OK;
  }
  for (int s = 0; s < nsteps; ++s) {
    std::string key(reinterpret_cast<const char*>(&dt), sizeof(dt));
    key.push_back((char)('0' + e->mode));
    key += std::to_string(e->branches); key.push_back('/');
    for (ocn_model* m : e->models) {
      key.push_back((char)('0' + m->cur)); key.push_back((char)('0' + m->variant));
      key += std::to_string(m->colc_version); key.push_back('/');
      key += std::to_string(m->graph_epoch); key.push_back('/');
      key.push_back((char)('0' + m->stepper)); key.push_back(m->ab_started ? 'a' : 'e');
    }
    auto it = e->graphs.find(key);
    std::vector<int> w(e->n);
    if (it == e->graphs.end() && e->graphs.size() >= kGraphCacheMax) {   // many time steps: start over
      cudaError_t es = cudaStreamSynchronize(e->stream);
      if (es != cudaSuccess) return cuda_fail(es, "graph cache reset");
      clear_graphs(e);
    }
    if (it == e->graphs.end() && e->mode == OCN_ENSEMBLE_BATCHED) {
      cudaGraphExec_t exec = nullptr;
      void* tables = nullptr;
      int nl = 0;
      ocn_status st = build_batched_graph<T>(e, dt, w, &exec, &tables, &nl);
      if (st != OCN_OK) return st;
      it = e->graphs.emplace(key, exec).first;
      e->graph_tables[key] = tables;
      e->launches_per_step = nl;
    } else if (it == e->graphs.end()) {
      // One graph for the whole ensemble step: fork a branch per member, join at the end;
      // the branches are independent, so their kernels run concurrently.
      cudaError_t ce = cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal);
      if (ce != cudaSuccess) return cuda_fail(ce, "ensemble begin capture");
      cudaError_t el = cudaEventRecord(e->fork, e->stream);
      int total = 0;
      for (int i = 0; i < e->n && el == cudaSuccess; ++i) {
        ocn_model* m = e->models[i];
        el = cudaStreamWaitEvent(e->fork_streams[i], e->fork, 0);
        if (el != cudaSuccess) break;
        m->stream = e->fork_streams[i];
        w[i] = m->cur;
        int nl = 0;
        el = enqueue_step<T>(m, dt, &w[i], &nl);
        m->stream = e->stream;
        total += nl;
        if (el == cudaSuccess) el = cudaEventRecord(e->join[i], e->fork_streams[i]);
        if (el == cudaSuccess) el = cudaStreamWaitEvent(e->stream, e->join[i], 0);
      }
      cudaGraph_t graph = nullptr;
      ce = cudaStreamEndCapture(e->stream, &graph);
      if (el != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return cuda_fail(el, "ensemble capture"); }
      if (ce != cudaSuccess) return cuda_fail(ce, "ensemble end capture");
      cudaGraphExec_t exec = nullptr;
      ce = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ce != cudaSuccess) return cuda_fail(ce, "ensemble graph instantiate");
      it = e->graphs.emplace(key, exec).first;
      e->launches_per_step = total;
    } else {
      for (int i = 0; i < e->n; ++i) w[i] = 1 - e->models[i]->cur;
    }
    cudaError_t ce = cudaGraphLaunch(it->second, e->stream);
    if (ce != cudaSuccess) return cuda_fail(ce, "ensemble graph launch");
    for (int i = 0; i < e->n; ++i) {
      e->models[i]->cur = w[i];
      if (e->models[i]->stepper == OCN_STEPPER_QAB2) e->models[i]->ab_started = true;
    }
  }
  return OCN_OK;
}
}  // namespace

extern "C" {

ocn_status ocn_ensemble_time_step(ocn_ensemble* e, double dt, int nsteps) {
  if (!e) return fail(OCN_ERR_ARG, "null argument");
  if (nsteps < 0 || !isfinite(dt)) return fail(OCN_ERR_ARG, "nsteps must be >= 0 and dt finite");
  DeviceGuard dg(e->dev);
  return (e->es == 4) ? ensemble_step_t<float>(e, dt, nsteps) : ensemble_step_t<double>(e, dt, nsteps);
}

ocn_status ocn_ensemble_set_option(ocn_ensemble* e, int option, long long value) {
  if (!e) return fail(OCN_ERR_ARG, "null argument");
  if (option == OCN_OPT_ENSEMBLE_MODE) {
    if (value != OCN_ENSEMBLE_CONCURRENT && value != OCN_ENSEMBLE_SEQUENTIAL && value != OCN_ENSEMBLE_BATCHED)
      return fail(OCN_ERR_ARG, "unknown ensemble mode");
    e->mode = (int)value;
    return OCN_OK;
  }
  if (option == OCN_OPT_ENSEMBLE_BRANCHES) {
    if (value < 1 || value > 64) return fail(OCN_ERR_ARG, "ensemble branches must be in 1..64");
    if (e->branches != (int)value) clear_graphs(e);
    e->branches = (int)value;
    return OCN_OK;
  }
  for (ocn_model* m : e->models) {
    ocn_status st = ocn_set_option(m, option, value);
    if (st != OCN_OK) return st;
  }
  return OCN_OK;
}

ocn_status ocn_ensemble_autotune(ocn_ensemble* e, int* variants) {
  if (!e) return fail(OCN_ERR_ARG, "null argument");
  for (ocn_model* m : e->models) if (!m->arena) return fail(OCN_ERR_STATE, "arena not bound");
  DeviceGuard dg(e->dev);
  const int nv = (e->es == 4) ? kTendencyVariants : 1;
  std::vector<int> saved(e->n);
  std::vector<LaunchHook> hooks(e->n);
  std::vector<bool> timing(e->n);
  for (int i = 0; i < e->n; ++i) {
    ocn_model* m = e->models[i];
    saved[i] = m->variant; hooks[i] = m->hook; timing[i] = m->timing;
    m->hook = LaunchHook(); m->timing = false;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  auto tendency_only = [&](ocn_model* m) -> cudaError_t {
    return (m->es == 4) ? enqueue_tendency<float>(m, m->cur, 0.0, 0.0, 1) : enqueue_tendency<double>(m, m->cur, 0.0, 0.0, 1);
  };
  ocn_status st = OCN_OK;
  // every member's tendency (G only) as in a step of the ensemble's mode: batched launches over the
  // members, or each member on its own branch; ms per pass (best of two after a warm-up)
  auto pass = [&](const std::vector<int>& var) -> float {
    float best = 1e30f;
    if (e->mode == OCN_ENSEMBLE_BATCHED) {
      for (int i = 0; i < e->n; ++i) e->models[i]->variant = var[i];
      std::vector<LaunchRecorder> recs;
      BatchPlan plan;
      if (st == OCN_OK) st = record_members(e, recs, [&](int, ocn_model* m) { return tendency_only(m); });
      if (st == OCN_OK) st = plan_batched(e, recs, &plan);
      if (st != OCN_OK) { if (ce == cudaSuccess) ce = cudaErrorUnknown; return best; }
      for (int r = 0; r < 3 && ce == cudaSuccess; ++r) {
        ce = cudaEventRecord(e0, e->stream);
        if (ce == cudaSuccess) ce = enqueue_batched(e, plan);
        if (ce == cudaSuccess) ce = cudaEventRecord(e1, e->stream);
        if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
        float t = 0.0f;
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&t, e0, e1);
        if (r > 0 && t < best) best = t;
      }
      cudaFree(plan.dtab);
      return best;
    }
    for (int r = 0; r < 3 && ce == cudaSuccess; ++r) {      // the first pass warms up
      ce = cudaEventRecord(e->fork, e->stream);
      if (ce == cudaSuccess) ce = cudaEventRecord(e0, e->stream);
      for (int i = 0; i < e->n && ce == cudaSuccess; ++i) {
        ocn_model* m = e->models[i];
        ce = cudaStreamWaitEvent(e->fork_streams[i], e->fork, 0);
        if (ce != cudaSuccess) break;
        m->variant = var[i];
        m->stream = e->fork_streams[i];
        ce = tendency_only(m);
        m->stream = e->stream;
        if (ce == cudaSuccess) ce = cudaEventRecord(e->join[i], e->fork_streams[i]);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(e->stream, e->join[i], 0);
      }
      if (ce == cudaSuccess) ce = cudaEventRecord(e1, e->stream);
      if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
      float t = 0.0f;
      if (ce == cudaSuccess) ce = cudaEventElapsedTime(&t, e0, e1);
      if (r > 0 && t < best) best = t;
    }
    return best;
  };
  std::vector<int> var(e->n, 0);
  if (nv > 1) {
    // one variant for every member
    float best = 1e30f;
    int arg = 0;
    for (int v = 0; v < nv && ce == cudaSuccess; ++v) {
      std::vector<int> t(e->n, v);
      const float ms = pass(t);
      if (ms < best) { best = ms; arg = v; }
    }
    var.assign(e->n, arg);
    // then per member shape, keeping a change only if the whole pass gets 2 % faster
    std::map<std::string, std::vector<int>> shapes;
    for (int i = 0; i < e->n; ++i) {
      const ocn_model* m = e->models[i];
      char buf[96];
      snprintf(buf, sizeof(buf), "%d %d %d %d %d %d", m->g->Nx, m->g->Ny, m->g->Nz, m->R, m->d.closure, m->d.n_tracers);
      shapes[buf].push_back(i);
    }
    if (shapes.size() > 1)
      for (auto& kv : shapes) {
        for (int v = 0; v < nv && ce == cudaSuccess; ++v) {
          if (v == var[kv.second[0]]) continue;
          std::vector<int> t = var;
          for (int i : kv.second) t[i] = v;
          const float ms = pass(t);
          if (ms < 0.98f * best) { best = ms; var = t; }
        }
      }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  for (int i = 0; i < e->n; ++i) {
    ocn_model* m = e->models[i];
    m->hook = hooks[i]; m->timing = timing[i];
    m->variant = (ce == cudaSuccess) ? var[i] : saved[i];
    if (m->variant != saved[i]) drop_graphs(m);
    if (ce == cudaSuccess) m->ab_started = false;   // G was overwritten: QAB2 restarts with its Euler step
    if (variants) variants[i] = m->variant;
  }
  clear_graphs(e);
  if (st != OCN_OK) return st;
  if (ce != cudaSuccess) return cuda_fail(ce, "ensemble autotune");
  return OCN_OK;
}

ocn_status ocn_ensemble_launches_per_step(const ocn_ensemble* e, int* launches) {
  if (!e || !launches) return fail(OCN_ERR_ARG, "null argument");
  *launches = e->launches_per_step;
  return OCN_OK;
}

ocn_status ocn_kernel_times(ocn_model* m, int* counts, double* ms) {
  if (!m || !counts || !ms) return fail(OCN_ERR_ARG, "null argument");
  DeviceGuard dg(m->dev);
  cudaError_t e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return cuda_fail(e, "kernel timing synchronise");
  for (int k = 0; k < OCN_K_COUNT; ++k) { counts[k] = 0; ms[k] = 0.0; }
  for (const auto& r : m->recs) {
    float t = 0.0f;
    e = cudaEventElapsedTime(&t, r.a, r.b);
    if (e != cudaSuccess) return cuda_fail(e, "kernel timing read");
    if (r.kclass >= 0 && r.kclass < OCN_K_COUNT) { counts[r.kclass] += 1; ms[r.kclass] += t; }
  }
  return OCN_OK;
}

ocn_status ocn_launches_per_step(const ocn_model* m, int* launches) {
  if (!m || !launches) return fail(OCN_ERR_ARG, "null argument");
  *launches = m->launches_per_step;
  return OCN_OK;
}

}  // extern "C"

namespace ocn {
ocn_status set_last_error(ocn_status s, const char* msg) {
  g_err = msg;
  return s;
}
}  // namespace ocn
