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

// Implicit, one thread per column (columns longer than the segmented solve below takes): the
// tridiagonal of field f is the same for every column, so each block factors it
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

// Segmented implicit solve: one read and one write of every unknown.  The matrix of field f is the
// same for every column, so its Thomas elimination is written as two first-order recurrences with
// column-independent coefficients,
//   forward   d'_r = alpha_r d'_{r-1} + beta_r rhs_r     (alpha_r = -sub_r / piv_r, beta_r = 1 / piv_r,
//                                                        rhs_r = q_r + dtau D(ref)_r),
//   backward  x_r  = d'_r + gamma_r x_{r+1}             (gamma_r = -sup_r / piv_r),
// and each column is split into kSegs segments of M rows held in the registers of one thread each
// (a block is 32 columns x kSegs segments, coalesced along x).  Over a segment, a recurrence maps
// its carry-in c to (local result with carry 0) + (product of the segment's coefficients) c, so:
// each segment runs the forward recurrence with carry 0 and publishes its last value; every thread
// combines the segments below it (y_t + G_t D, G_t the product of alpha over segment t) into its
// carry-in and runs the forward recurrence again from it, now exactly; the backward recurrence is
// done the same way from the top (H_t the product of gamma over segment t).  The matrix is
// diagonally dominant, so |alpha|, |gamma| < 1 and the products only decay.  k_vdiff_factor
// computes the per-row coefficients (alpha, beta, dtau D(ref), gamma) and the segment products
// once per call and field; a solve block copies its field's rows into shared memory.
constexpr int kSegs = 8;
constexpr int kMaxSeg = 64;
// work-space elements per field: 4 per row, then (G_t, H_t) per segment
__host__ __device__ constexpr size_t vtab_stride(int Nz) { return 4 * (size_t)Nz + 2 * kSegs; }

// One block per field.  The rows' matrix entries and dtau D(ref) are formed in parallel (their
// loads issued together), the pivot recurrence piv_r = diag_r - sub_r sup_{r-1} / piv_{r-1} runs
// in one thread over shared memory, and the coefficients and segment products are written in
// parallel again.
constexpr int kFactorThreads = 256;

template <typename T>
__device__ __forceinline__ void vdiff_factor_body(const VDiffArgs<T>& a, const uint3 bid) {
  __shared__ T s_sub[kSegs * kMaxSeg], s_sup[kSegs * kMaxSeg], s_dia[kSegs * kMaxSeg];
  const int f = bid.y;
  if (!((a.fields >> f) & 1)) return;              // uniform over the block
  const int Nz = a.Nz;
  const bool faces = (f == 2);
  const int n0 = faces ? 1 : 0, n = faces ? Nz - 1 : Nz;
  if (n <= 0) return;
  T* tb = a.tab + (size_t)f * vtab_stride(Nz);
  const T* kf = (f < 3) ? a.nuz : a.kapz;
  const T* ref = (f >= 3) ? a.cref[f - 3] : nullptr;
  const T dtau = a.dtau;
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
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
    s_sub[r] = (r > 0) ? -dtau * lo / h : T(0);
    s_sup[r] = (r < n - 1) ? -dtau * hi / h : T(0);
    s_dia[r] = T(1) + dtau * (lo + hi) / h;
    T dr = T(0);
    if (ref) {                                     // dtau D(ref) at centre k
      const T Fb = (k > 0) ? -kf[k] * (ref[k] - ref[k - 1]) / a.dzf[k] : T(0);
      const T Ft = (k < Nz - 1) ? -kf[k + 1] * (ref[k + 1] - ref[k]) / a.dzf[k + 1] : T(0);
      dr = dtau * (-(Ft - Fb) / a.dzc[k]);
    }
    tb[4 * r + 2] = dr;
  }
  __syncthreads();
  if (threadIdx.x == 0) {                          // the pivots; s_dia becomes 1 / piv
    T cprev = T(0);
    for (int r = 0; r < n; ++r) {
      const T inv = T(1) / (s_dia[r] - s_sub[r] * cprev);
      cprev = s_sup[r] * inv;
      s_dia[r] = inv;
    }
  }
  __syncthreads();
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    const T inv = s_dia[r];
    tb[4 * r] = -s_sub[r] * inv;
    tb[4 * r + 1] = inv;
    tb[4 * r + 3] = -(s_sup[r] * inv);
  }
  __syncthreads();
  const int M = a.seg;
  for (int sg = threadIdx.x; sg < kSegs; sg += blockDim.x) {   // segment products
    T g = T(1), hh = T(1);
    for (int r = sg * M; r < min(n, sg * M + M); ++r) { g *= tb[4 * r]; hh *= tb[4 * r + 3]; }
    tb[4 * (size_t)Nz + 2 * sg] = g;
    tb[4 * (size_t)Nz + 2 * sg + 1] = hh;
  }
}

// Row r of the shared coefficient table (alpha, beta, dtau D(ref), gamma), read where it is used:
// the loads are volatile so that the compiler does not keep every row of a segment live in
// registers between the passes (which would cost the occupancy the loads in flight need).
struct Row4f { float a, b, c, g; };
struct Row4d { double a, b, c, g; };
__device__ __forceinline__ Row4f srow(const float* st, int r) {
  Row4f o;
  const unsigned ad = (unsigned)__cvta_generic_to_shared(st + 4 * r);
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(o.a), "=f"(o.b), "=f"(o.c), "=f"(o.g) : "r"(ad));
  return o;
}
__device__ __forceinline__ Row4d srow(const double* st, int r) {
  Row4d o;
  const unsigned ad = (unsigned)__cvta_generic_to_shared(st + 4 * r);
  asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(o.a), "=d"(o.b) : "r"(ad));
  asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(o.c), "=d"(o.g) : "r"(ad + 16));
  return o;
}

template <typename T, int M>
__device__ __forceinline__ void vdiff_isolve_body(const VDiffArgs<T>& a, const uint3 bid) {
  extern __shared__ __align__(16) unsigned char vsm[];
  __shared__ T sY[kSegs][32], sZ[kSegs][32];
  const int f = bid.y;
  if (!((a.fields >> f) & 1)) return;            // uniform over the block
  const int Nz = a.Nz;
  const int n0 = (f == 2) ? 1 : 0, n = (f == 2) ? Nz - 1 : Nz;
  if (n <= 0) return;
  T* st = reinterpret_cast<T*>(vsm);             // the field's work space: 4 n + 2 kSegs values
  const T* tb = a.tab + (size_t)f * vtab_stride(Nz);
  const int tid = threadIdx.x + 32 * threadIdx.y;
  for (int i = tid; i < 4 * n; i += 32 * kSegs) st[i] = tb[i];
  if (tid < 2 * kSegs) st[4 * n + tid] = tb[4 * Nz + tid];
  const size_t plane = (size_t)a.Nx * a.Ny;
  const int lx = threadIdx.x, sg = threadIdx.y;
  const size_t col = (size_t)bid.x * 32 + lx;
  const bool valid = col < plane;
  const int r0 = sg * M;
  T* q = a.qout[f] + (valid ? col : 0) + (size_t)n0 * plane;   // unknown r at q[r plane]
  T v[M];
  {
    const T* ql = q + (size_t)r0 * plane;          // a running pointer: no per-row address is kept
#pragma unroll
    for (int u = 0; u < M; ++u, ql += plane) v[u] = (valid && r0 + u < n) ? *ql : T(0);
  }
  __syncthreads();
  const T* G = st + 4 * n;                        // G_t, H_t at G[2 t], G[2 t + 1]
  // forward recurrence with carry 0: the segment's last value
  T y = T(0);
#pragma unroll
  for (int u = 0; u < M; ++u) {
    const int r = r0 + u;
    if (r < n) { const auto c = srow(st, r); y = fma(c.a, y, c.b * (v[u] + c.c)); }
  }
  sY[sg][lx] = y;
  __syncthreads();
  T d = T(0);                                     // d' of row r0 - 1 (the segments below are full)
  if (r0 < n)
    for (int t = 0; t < sg; ++t) d = fma(G[2 * t], d, sY[t][lx]);
#pragma unroll
  for (int u = 0; u < M; ++u) {
    const int r = r0 + u;
    if (r < n) {
      const auto c = srow(st, r);
      d = fma(c.a, d, c.b * (v[u] + c.c));
      v[u] = d;
    }
  }
  // backward recurrence with carry 0: the segment's first value
  T z = T(0);
#pragma unroll
  for (int u = M - 1; u >= 0; --u) {
    const int r = r0 + u;
    if (r < n) z = fma(srow(st, r).g, z, v[u]);
  }
  sZ[sg][lx] = z;
  __syncthreads();
  T x = T(0);                                     // x of row r0 + M
  for (int t = kSegs - 1; t > sg; --t)
    if (t * M < n) x = fma(G[2 * t + 1], x, sZ[t][lx]);
  T* qs = q + (size_t)(r0 + M - 1) * plane;
#pragma unroll
  for (int u = M - 1; u >= 0; --u, qs -= plane) {
    const int r = r0 + u;
    if (r < n) {
      x = fma(srow(st, r).g, x, v[u]);
      if (valid) *qs = x;
    }
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
template <typename T> struct VDiffFactorK {
  typedef VDiffArgs<T> Payload;
  static constexpr int kThreads = kFactorThreads, kMinBlocks = 1;
  static __device__ __forceinline__ void run(const Payload& a, uint3 bid, uint3) { vdiff_factor_body<T>(a, bid); }
};
template <typename T, int M> struct VDiffSolveK {
  typedef VDiffArgs<T> Payload;
  static constexpr int kThreads = 32 * kSegs, kMinBlocks = 1;
  static __device__ __forceinline__ void run(const Payload& a, uint3 bid, uint3) { vdiff_isolve_body<T, M>(a, bid); }
};
template <typename T>
__global__ void __launch_bounds__(kFactorThreads) k_vdiff_factor(const VDiffArgs<T> a) { vdiff_factor_body<T>(a, blockIdx); }
template <typename T, int M>
__global__ void __launch_bounds__(32 * kSegs) k_vdiff_isolve(const VDiffArgs<T> a) { vdiff_isolve_body<T, M>(a, blockIdx); }
template <typename T>
__global__ void __launch_bounds__(kColsPerBlock) k_vdiff_explicit(const VDiffArgs<T> a) { vdiff_explicit_body<T>(a, blockIdx); }
template <typename T>
__global__ void __launch_bounds__(kColsPerBlock) k_vdiff_implicit(const VDiffArgs<T> a) { vdiff_implicit_body<T>(a, blockIdx); }

}  // namespace

template <typename T, int M>
cudaError_t launch_isolve(const VDiffArgs<T>& a, const size_t plane, cudaStream_t s) {
  dim3 grid((unsigned)((plane + 31) / 32), 3 + a.nt), block(32, kSegs);
  const size_t smem = sizeof(T) * vtab_stride(a.Nz);
  if (record_launch<VDiffSolveK<T, M>>(a, grid, block, smem, OCN_K_VERTICAL)) return cudaSuccess;
  k_vdiff_isolve<T, M><<<grid, block, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_vertical_diffusion(const VDiffArgs<T>& a_, bool implicit, cudaStream_t s, int* nlaunch) {
  const size_t plane = (size_t)a_.Nx * a_.Ny;
  dim3 grid((unsigned)((plane + kColsPerBlock - 1) / kColsPerBlock), 3 + a_.nt);
  if (implicit) {
    // segmented solve when the column fits kSegs segments of at most kMaxSeg rows and the work
    // space holds the coefficient tables
    VDiffArgs<T> a = a_;
    int M = 4;
    while (M < kMaxSeg && M * kSegs < a.Nz) M *= 2;
    if (a.tab && M * kSegs >= a.Nz && a.tab_cap >= (3 + a.nt) * vtab_stride(a.Nz)) {
      a.seg = M;
      cudaError_t e = cudaSuccess;
      const dim3 fgrid(1, 3 + a.nt);
      if (!record_launch<VDiffFactorK<T>>(a, fgrid, dim3(kFactorThreads), 0, OCN_K_VERTICAL)) {
        k_vdiff_factor<T><<<fgrid, kFactorThreads, 0, s>>>(a);
        e = cudaGetLastError();
      }
      if (e != cudaSuccess) return e;
      switch (M) {
        case 4: e = launch_isolve<T, 4>(a, plane, s); break;
        case 8: e = launch_isolve<T, 8>(a, plane, s); break;
        case 16: e = launch_isolve<T, 16>(a, plane, s); break;
        case 32: e = launch_isolve<T, 32>(a, plane, s); break;
        default: e = launch_isolve<T, 64>(a, plane, s); break;
      }
      if (nlaunch) *nlaunch += 2;
      return e;
    }
    const size_t smem = 4 * sizeof(T) * (size_t)a.Nz;
    if (smem > 48 * 1024) return cudaErrorInvalidValue;
    if (nlaunch) *nlaunch += 1;
    if (record_launch<VDiffImplicitK<T>>(a, grid, dim3(kColsPerBlock), smem, OCN_K_VERTICAL)) return cudaSuccess;
    k_vdiff_implicit<T><<<grid, kColsPerBlock, smem, s>>>(a);
  } else {
    if (nlaunch) *nlaunch += 1;
    if (record_launch<VDiffExplicitK<T>>(a_, grid, dim3(kColsPerBlock), 0, OCN_K_VERTICAL)) return cudaSuccess;
    k_vdiff_explicit<T><<<grid, kColsPerBlock, 0, s>>>(a_);
  }
  return cudaGetLastError();
}
template cudaError_t launch_vertical_diffusion<float>(const VDiffArgs<float>&, bool, cudaStream_t, int*);
template cudaError_t launch_vertical_diffusion<double>(const VDiffArgs<double>&, bool, cudaStream_t, int*);

}  // namespace ocn
