// Vertical diffusion with a z-profile of diffusivity (Eq. tracer-with-tendency and
// Eq. momentum-tendency-definition), either as an explicit tendency or with the semi-implicit
// step of Eq. tracer-time-discretization / Eq. predictor-velocity,
//   (1 - dtau d/dz kappa d/dz) q^{m+1} = q~,
// solved down every column by the Thomas algorithm.  Second-order finite volumes: fluxes
// -kappa_f (q_k - q_{k-1}) / dz_f through the interior faces, none through the walls; u, v and
// tracers live at centres (kappa at faces), w at faces (walls held at 0, diffusivity at the
// centres = the mean of the two faces).  Tracers are stored as anomalies a about a reference
// profile r: the explicit term uses a + r, the implicit step solves for a with the right-hand
// side a~ + dtau D(r), which is the same system.
#include <cuda_runtime.h>

#include "batch.cuh"
#include "ocn_internal.cuh"

namespace ocn {
namespace {

constexpr int kColsPerBlock = 128;

template <typename T>
__device__ __forceinline__ T qval(const VDiffArgs<T>& a, int f, const T* q, size_t idx, int k) {
  T v = q[idx];
  if (f >= 3 && a.cref[f - 3]) v += a.cref[f - 3][k];
  return v;
}

// Explicit: dG = D(q of the stage state); G += dG and (mode 0) the new state += dt_gamma dG.
template <typename T>
__device__ __forceinline__ void vdiff_explicit_body(const VDiffArgs<T>& a, const uint3 bid) {
  const int f = bid.y;
  if (!((a.fields >> f) & 1)) return;
  const size_t plane = (size_t)a.Nx * a.Ny;
  const size_t col = (size_t)bid.x * kColsPerBlock + threadIdx.x;
  if (col >= plane) return;
  const T* __restrict__ kf = (f < 3) ? a.nuz : a.kapz;
  const T* __restrict__ qi = a.qin[f];
  T* __restrict__ qo = a.qout[f];
  T* __restrict__ G = a.G[f];
  const int Nz = a.Nz;
  if (f != 2) {                                    // centres
    T qc = qval(a, f, qi, col, 0);
    T Fb = T(0);
    for (int k = 0; k < Nz; ++k) {
      T Ft = T(0), qn = qc;
      if (k + 1 < Nz) {
        qn = qval(a, f, qi, (size_t)(k + 1) * plane + col, k + 1);
        Ft = -kf[k + 1] * (qn - qc) / a.dzf[k + 1];
      }
      const T d = -(Ft - Fb) / a.dzc[k];
      const size_t id = (size_t)k * plane + col;
      G[id] += d;
      if (a.mode == 0) qo[id] += a.dt_gamma * d;
      Fb = Ft;
      qc = qn;
    }

  } else {                                         // w at faces 1..Nz-1
    for (int k = 1; k < Nz; ++k) {
      const T w0 = qi[(size_t)(k - 1) * plane + col], w1 = qi[(size_t)k * plane + col],
              w2 = qi[(size_t)(k + 1) * plane + col];
      const T Fb = -T(0.5) * (kf[k - 1] + kf[k]) * (w1 - w0) / a.dzc[k - 1];
      const T Ft = -T(0.5) * (kf[k] + kf[k + 1]) * (w2 - w1) / a.dzc[k];
      const T d = -(Ft - Fb) / a.dzf[k];
      const size_t id = (size_t)k * plane + col;
      G[id] += d;
      if (a.mode == 0) qo[id] += a.dt_gamma * d;
    }
  }
}

// Implicit: the tridiagonal of field f is the same for every column, so each block factors it
// once into shared memory (sub-diagonal a, 1/pivot, c', and for tracers dtau D(ref)) and every
// thread sweeps its column.  Levels move in chunks of kChunk: a chunk's loads are issued together,
// swept in registers, then stored, so the loads of a column are not serialised behind its stores.
constexpr int kChunk = 8;

template <typename T>
__device__ __forceinline__ void vdiff_implicit_body(const VDiffArgs<T>& a, const uint3 bid) {
  extern __shared__ __align__(16) unsigned char vsm[];
  const int f = bid.y;
  if (!((a.fields >> f) & 1)) return;
  const int Nz = a.Nz;
  const bool faces = (f == 2);
  const int n0 = faces ? 1 : 0, n = faces ? Nz - 1 : Nz;   // unknowns n0 .. n0+n-1
  if (n <= 0) return;
  T* sa = reinterpret_cast<T*>(vsm);
  T* sinv = sa + Nz;
  T* scp = sinv + Nz;
  T* sref = scp + Nz;
  const T* kf = (f < 3) ? a.nuz : a.kapz;
  const T* ref = (f >= 3) ? a.cref[f - 3] : nullptr;
  const T dtau = a.dtau;
  if (threadIdx.x == 0) {
    T cprev = T(0);
    for (int r = 0; r < n; ++r) {
      const int k = n0 + r;
      T lo, hi, h;
      if (!faces) {
        h = a.dzc[k];
        lo = (k > 0) ? kf[k] / a.dzf[k] : T(0);
        hi = (k < Nz - 1) ? kf[k + 1] / a.dzf[k + 1] : T(0);
      } else {
        h = a.dzf[k];
        lo = T(0.5) * (kf[k - 1] + kf[k]) / a.dzc[k - 1];
        hi = T(0.5) * (kf[k] + kf[k + 1]) / a.dzc[k];
      }
      const T sub = (r > 0) ? -dtau * lo / h : T(0);
      const T sup = (r < n - 1) ? -dtau * hi / h : T(0);
      const T diag = T(1) + dtau * (lo + hi) / h;
      const T inv = T(1) / (diag - sub * cprev);
      sa[r] = sub;
      sinv[r] = inv;
      scp[r] = sup * inv;
      cprev = scp[r];
      T dr = T(0);
      if (ref) {                                   // dtau D(ref) at centre k
        const T Fb = (k > 0) ? -kf[k] * (ref[k] - ref[k - 1]) / a.dzf[k] : T(0);
        const T Ft = (k < Nz - 1) ? -kf[k + 1] * (ref[k + 1] - ref[k]) / a.dzf[k + 1] : T(0);
        dr = dtau * (-(Ft - Fb) / a.dzc[k]);
      }
      sref[r] = dr;
    }
  }
  __syncthreads();
  const size_t plane = (size_t)a.Nx * a.Ny;
  const size_t col = (size_t)bid.x * kColsPerBlock + threadIdx.x;
  if (col >= plane) return;
  T* q = a.qout[f] + col + (size_t)n0 * plane;      // unknown r at q[r * plane]
  // forward sweep: d' overwrites the column
  T dprev = T(0);
  for (int r0 = 0; r0 < n; r0 += kChunk) {
    T d[kChunk];
#pragma unroll
    for (int u = 0; u < kChunk; ++u) d[u] = (r0 + u < n) ? q[(size_t)(r0 + u) * plane] : T(0);
#pragma unroll
    for (int u = 0; u < kChunk; ++u) {
      const int r = r0 + u;
      if (r < n) {
        dprev = (d[u] + sref[r] - sa[r] * dprev) * sinv[r];
        d[u] = dprev;
      }
    }
#pragma unroll
    for (int u = 0; u < kChunk; ++u)
      if (r0 + u < n) q[(size_t)(r0 + u) * plane] = d[u];
  }
  // back substitution, top down, chunk by chunk
  T x = dprev;
  for (int r1 = n - 2; r1 >= 0; r1 -= kChunk) {
    T d[kChunk];
#pragma unroll
    for (int u = 0; u < kChunk; ++u) d[u] = (r1 - u >= 0) ? q[(size_t)(r1 - u) * plane] : T(0);
#pragma unroll
    for (int u = 0; u < kChunk; ++u) {
      const int r = r1 - u;
      if (r >= 0) {
        x = d[u] - scp[r] * x;
        d[u] = x;
      }
    }
#pragma unroll
    for (int u = 0; u < kChunk; ++u)
      if (r1 - u >= 0) q[(size_t)(r1 - u) * plane] = d[u];
  }
}

template <typename T> struct VDiffExplicitK {
  typedef VDiffArgs<T> Payload;
  static constexpr int kThreads = kColsPerBlock, kMinBlocks = 1;
  static __device__ __forceinline__ void run(const Payload& a, uint3 bid, uint3) { vdiff_explicit_body<T>(a, bid); }
};
template <typename T> struct VDiffImplicitK {
  typedef VDiffArgs<T> Payload;
  static constexpr int kThreads = kColsPerBlock, kMinBlocks = 1;
  static __device__ __forceinline__ void run(const Payload& a, uint3 bid, uint3) { vdiff_implicit_body<T>(a, bid); }
};
template <typename T>
__global__ void __launch_bounds__(kColsPerBlock) k_vdiff_explicit(const VDiffArgs<T> a) { vdiff_explicit_body<T>(a, blockIdx); }
template <typename T>
__global__ void __launch_bounds__(kColsPerBlock) k_vdiff_implicit(const VDiffArgs<T> a) { vdiff_implicit_body<T>(a, blockIdx); }

}  // namespace

template <typename T>
cudaError_t launch_vertical_diffusion(const VDiffArgs<T>& a, bool implicit, cudaStream_t s) {
  const size_t plane = (size_t)a.Nx * a.Ny;
  dim3 grid((unsigned)((plane + kColsPerBlock - 1) / kColsPerBlock), 3 + a.nt);
  if (implicit) {
    const size_t smem = 4 * sizeof(T) * (size_t)a.Nz;
    if (smem > 48 * 1024) return cudaErrorInvalidValue;
    if (record_launch<VDiffImplicitK<T>>(a, grid, dim3(kColsPerBlock), smem, OCN_K_VERTICAL)) return cudaSuccess;
    k_vdiff_implicit<T><<<grid, kColsPerBlock, smem, s>>>(a);
  } else {
    if (record_launch<VDiffExplicitK<T>>(a, grid, dim3(kColsPerBlock), 0, OCN_K_VERTICAL)) return cudaSuccess;
    k_vdiff_explicit<T><<<grid, kColsPerBlock, 0, s>>>(a);
  }
  return cudaGetLastError();
}
template cudaError_t launch_vertical_diffusion<float>(const VDiffArgs<float>&, bool, cudaStream_t);
template cudaError_t launch_vertical_diffusion<double>(const VDiffArgs<double>&, bool, cudaStream_t);

}  // namespace ocn
