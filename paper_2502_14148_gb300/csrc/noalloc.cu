// ocn_project_noalloc: the pressure projection of ocn_project for callers that
// cannot allocate device memory.  Everything the projection needs besides the
// caller's velocity and pressure arrays -- the half spectrum, the tridiagonal
// pivots, the grid metrics and the FFT twiddles -- lives in one fixed array
// declared in this file, sized for grids with at most OCN_NOALLOC_MAX_MODES
// horizontal-wavenumber x level entries.  The array exists once per device
// that loads the library and stays until the process exits.  No call here
// allocates device memory.
//
// Host code cannot use the array's name as a device address (it is a host-side
// stand-in), so the first call on each device looks the address up with
// cudaGetSymbolAddress while that device is current and keeps it.  Calls share
// the array: each call rewrites every part of it that it reads before reading
// it, so nothing has to start at zero, but calls whose work overlaps on the GPU
// (for example on two streams at once) race on it.  Every call uploads its grid
// tables from a host array, so a stream that is being captured is refused.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <mutex>

#include "ocn_internal.cuh"

using namespace ocn;

namespace {

constexpr size_t kModes = OCN_NOALLOC_MAX_MODES;
constexpr int kN = OCN_NOALLOC_MAX_N;
// Word (8-byte) offsets of the parts of the array; all 32-word aligned.
constexpr size_t al32(size_t x) { return (x + 31) & ~(size_t)31; }
constexpr size_t kOffSpec = 0;                                   // complex half spectrum
constexpr size_t kOffPiv = al32(kOffSpec + 2 * kModes);          // Thomas pivots
constexpr size_t kOffMet = al32(kOffPiv + kModes);               // metric tables (below)
constexpr size_t kMetWords = al32(kN) * 2 + al32(kN + 1) * 2 + al32(kN / 2 + 1) + al32(kN) + 2 * al32(2 * kN);
constexpr size_t kWords = kOffMet + kMetWords;

static __device__ __align__(256) double g_noalloc_scratch[kWords];

std::mutex g_mu;                 // guards the address table and the host staging array
void* g_addr[64] = {nullptr};
double g_metrics[kMetWords];     // host staging of the metric tables (static storage, no allocation)

struct Result {
  ocn_status st;
  const char* msg;               // string literal
};
Result bad(ocn_status s, const char* msg) { return {s, msg}; }

bool is_2a3b(int n) {
  if (n < 1) return false;
  while (n % 2 == 0) n /= 2;
  while (n % 3 == 0) n /= 3;
  return n == 1;
}

FftPlan plan_for(int n) {
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

// Device address of the array on the current device (looked up once per device;
// the caller holds g_mu).
Result scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return bad(OCN_ERR_CUDA, "cudaGetDevice failed");
  if (dev < 0 || dev >= 64) return bad(OCN_ERR_UNSUPPORTED, "device index above 63");
  if (!g_addr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) return bad(OCN_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed");
    g_addr[dev] = ptr;
  }
  *out = g_addr[dev];
  return {OCN_OK, ""};
}

template <typename T>
Result project_t(int Nx, int Ny, int Nz, double Lx, double Ly, const double* zf, T* u, T* v, T* w, T* p,
                 cudaStream_t s, char* scratch) {
  // metric tables in the model precision, staged on the host, at fixed offsets
  T* met = reinterpret_cast<T*>(g_metrics);
  size_t o = 0;
  auto take = [&](size_t words) { size_t at = o; o += words; return at; };   // offsets in 8-byte words
  const size_t wDzc = take(al32(kN)), wRdzc = take(al32(kN)), wDzf = take(al32(kN + 1)), wRdzf = take(al32(kN + 1));
  const size_t wLx = take(al32(kN / 2 + 1)), wLy = take(al32(kN)), wTx = take(al32(2 * kN)), wTy = take(al32(2 * kN));
  auto at = [&](size_t word) { return reinterpret_cast<T*>(reinterpret_cast<char*>(met) + word * 8); };
  bool stretched = false;
  const double dz0 = zf[1] - zf[0];
  for (int k = 0; k < Nz; ++k) {
    const double dz = zf[k + 1] - zf[k];
    if (fabs(dz - dz0) > 1e-12 * fabs(dz0)) stretched = true;
    at(wDzc)[k] = (T)dz;
    at(wRdzc)[k] = (T)(1.0 / dz);
  }
  for (int k = 0; k <= Nz; ++k) {
    double dzf;
    if (k == 0) dzf = zf[1] - zf[0];
    else if (k == Nz) dzf = zf[Nz] - zf[Nz - 1];
    else dzf = 0.5 * (zf[k + 1] + zf[k]) - 0.5 * (zf[k] + zf[k - 1]);
    at(wDzf)[k] = (T)dzf;
    at(wRdzf)[k] = (T)((k >= 1 && k < Nz) ? 1.0 / dzf : 0.0);
  }
  const double dx = Lx / Nx, dy = Ly / Ny;
  for (int kx = 0; kx <= Nx / 2; ++kx) { const double sn = 2.0 * sin(M_PI * kx / Nx) / dx; at(wLx)[kx] = (T)(-sn * sn); }
  for (int ky = 0; ky < Ny; ++ky) { const double sn = 2.0 * sin(M_PI * ky / Ny) / dy; at(wLy)[ky] = (T)(-sn * sn); }
  for (int t = 0; t < Nx; ++t) {
    const double th = -2.0 * M_PI * (double)t / Nx;
    at(wTx)[2 * t] = (T)cos(th); at(wTx)[2 * t + 1] = (T)sin(th);
  }
  for (int t = 0; t < Ny; ++t) {
    const double th = -2.0 * M_PI * (double)t / Ny;
    at(wTy)[2 * t] = (T)cos(th); at(wTy)[2 * t + 1] = (T)sin(th);
  }
  char* dmet = scratch + kOffMet * 8;
  // from pageable host memory: returns once the staging buffer has been consumed
  cudaError_t e = cudaMemcpyAsync(dmet, g_metrics, o * 8, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return bad(OCN_ERR_CUDA, "metric upload failed");

  PoissonArgs<T> a;
  memset(&a, 0, sizeof(a));
  a.u = u; a.v = v; a.w = w; a.p = p;
  a.spec = reinterpret_cast<T*>(scratch + kOffSpec * 8);
  a.cpiv = reinterpret_cast<T*>(scratch + kOffPiv * 8);
  auto dat = [&](size_t word) { return reinterpret_cast<const T*>(dmet + word * 8); };
  a.dzc = dat(wDzc); a.rdzc = dat(wRdzc); a.rdzf = dat(wRdzf);
  a.lamx = dat(wLx); a.lamy = dat(wLy); a.twx = dat(wTx); a.twy = dat(wTy);
  a.Nx = Nx; a.Ny = Ny; a.Nz = Nz; a.Mx = Nx / 2; a.Sp = Nx / 2 + 1;   // unpadded: the array's size limit
  a.rdx = (T)(Nx / Lx); a.rdy = (T)(Ny / Ly);
  a.inv_dt = (T)1; a.dt = (T)1;
  a.scale = (T)(1.0 / ((double)(Nx / 2) * Ny));
  a.Htot = (T)(zf[Nz] - zf[0]);
  a.fp64_pivots = stretched ? 1 : 0;
  a.px = plan_for(Nx / 2);
  a.py = plan_for(Ny);
  e = launch_projection<T>(a, s, nullptr);
  if (e != cudaSuccess) return bad(OCN_ERR_CUDA, "projection kernel launch failed");
  return {OCN_OK, ""};
}

}  // namespace

extern "C" ocn_status ocn_project_noalloc(int precision, int Nx, int Ny, int Nz, double Lx, double Ly,
                                          const double* z_faces, void* u, void* v, void* w, void* p, void* stream,
                                          const char** error) {
  Result r = {OCN_OK, ""};
  if (!z_faces || !u || !v || !w || !p) r = bad(OCN_ERR_ARG, "null argument");
  else if (precision != 32 && precision != 64) r = bad(OCN_ERR_ARG, "precision must be 32 or 64");
  else if (Nx < 4 || Ny < 4 || (Nx % 2) || (Ny % 2) || !is_2a3b(Nx) || !is_2a3b(Ny))
    r = bad(OCN_ERR_ARG, "Nx and Ny must be even, >= 4 and of the form 2^a 3^b");
  else if (Nz < 1) r = bad(OCN_ERR_ARG, "Nz must be >= 1");
  else if (Nx > kN || Ny > kN || Nz > kN) r = bad(OCN_ERR_ARG, "Nx, Ny and Nz must not exceed OCN_NOALLOC_MAX_N");
  else if ((size_t)(Nx / 2 + 1) * (size_t)Ny * (size_t)Nz > kModes)
    r = bad(OCN_ERR_ARG, "(Nx/2+1)*Ny*Nz exceeds OCN_NOALLOC_MAX_MODES");
  else if (!(Lx > 0) || !(Ly > 0)) r = bad(OCN_ERR_ARG, "Lx and Ly must be positive");
  else {
    for (int k = 0; k < Nz; ++k)
      if (!(z_faces[k + 1] > z_faces[k])) { r = bad(OCN_ERR_ARG, "z_faces must be strictly ascending"); break; }
  }
  if (r.st == OCN_OK) {
    // The metric tables are uploaded from a host array on every call, which a stream under
    // capture cannot record (and a graph that replayed it would read whatever a later call left
    // in that array), so a capturing stream is refused before anything is enqueued.
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(reinterpret_cast<cudaStream_t>(stream), &cs) != cudaSuccess ||
        cs != cudaStreamCaptureStatusNone)
      r = bad(OCN_ERR_UNSUPPORTED, "the stream is being captured into a CUDA graph; ocn_project_noalloc "
                                   "uploads its grid tables from host memory and cannot be captured");
  }
  if (r.st == OCN_OK) {
    std::lock_guard<std::mutex> lk(g_mu);
    void* scratch = nullptr;
    r = scratch_address(&scratch);
    if (r.st == OCN_OK) {
      cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
      r = (precision == 32)
              ? project_t<float>(Nx, Ny, Nz, Lx, Ly, z_faces, (float*)u, (float*)v, (float*)w, (float*)p, s, (char*)scratch)
              : project_t<double>(Nx, Ny, Nz, Lx, Ly, z_faces, (double*)u, (double*)v, (double*)w, (double*)p, s, (char*)scratch);
    }
  }
  if (error) *error = r.msg;
  return r.st;
}
