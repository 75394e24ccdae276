// Diagnostics: FP64 volume integrals (sum V c for every tracer, sum V u,
// sum V v, sum V w), max |div u|, the largest advective rate |u|/dx, |v|/dy,
// |w|/dz_f, and a count of non-finite values.  Conservation of the volume
// integrals in periodic, no-flux domains follows from the flux form
// (Eq. flux-divergence, Appendix B); div u = 0 from the projection (Eq.
// continuity, Appendix A.2).
// Two stages with a fixed reduction order (per-block partials, then one
// block), so the result is bitwise reproducible run to run.
#include <cuda_runtime.h>
#include <math.h>

#include "ocn_internal.cuh"

namespace ocn {

constexpr int kDiagBlocks = 1216;   // 8 x 152 SMs
constexpr int kDiagThreads = 256;
constexpr int kDiagVals = OCN_MAX_TRACERS + 6;

int diag_blocks() { return kDiagBlocks; }

template <typename T>
__global__ void __launch_bounds__(kDiagThreads) k_diag(const DiagArgs<T> a) {
  const int Nx = a.Nx, Ny = a.Ny, Nz = a.Nz, nt = a.nt;
  const size_t plane = (size_t)Nx * Ny;
  const size_t N = plane * Nz;
  double acc[kDiagVals];
#pragma unroll
  for (int v = 0; v < kDiagVals; ++v) acc[v] = 0.0;
  const double A = (double)a.dx * (double)a.dy;
  for (size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x; id < N; id += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(id / plane);
    const size_t r = id - (size_t)k * plane;
    const int j = (int)(r / Nx), i = (int)(r - (size_t)j * Nx);
    const int ip = (i + 1 == Nx) ? 0 : i + 1, jp = (j + 1 == Ny) ? 0 : j + 1;
    const double V = A * (double)a.dzc[k];
    double bad = 0.0;
#pragma unroll
    for (int t = 0; t < OCN_MAX_TRACERS; ++t) {
      if (t < nt) {
        const double c = (double)a.cur.c[t][id];
        acc[t] += V * c;
        if (!isfinite(c)) bad += 1.0;
      }
    }
    const double u = (double)a.cur.u[id], v = (double)a.cur.v[id], w = (double)a.cur.w[id];
    acc[nt] += V * u;
    acc[nt + 1] += V * v;
    const double div = ((double)a.cur.u[id - i + ip] - u) * (double)a.rdx +
                       ((double)a.cur.v[(size_t)k * plane + (size_t)jp * Nx + i] - v) * (double)a.rdy +
                       ((double)a.cur.w[id + plane] - w) * (double)a.rdzc[k];
    acc[nt + 3] = fmax(acc[nt + 3], fabs(div));
    double rate = fmax(fabs(u) * (double)a.rdx, fabs(v) * (double)a.rdy);
    if (k >= 1) {
      acc[nt + 2] += A * (double)a.dzf[k] * w;
      rate = fmax(rate, fabs(w) * (double)a.rdzf[k]);
    }
    acc[nt + 4] = fmax(acc[nt + 4], rate);
    if (!isfinite(u) || !isfinite(v) || !isfinite(w)) bad += 1.0;
    acc[nt + 5] += bad;
  }
  __shared__ double red[kDiagThreads / 32][kDiagVals];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int v = 0; v < kDiagVals; ++v) {
    double x = acc[v];
    const bool ismax = (v == nt + 3 || v == nt + 4);
    for (int o = 16; o > 0; o >>= 1) {
      const double y = __shfl_down_sync(0xffffffffu, x, o);
      x = ismax ? fmax(x, y) : x + y;
    }
    if (lane == 0) red[wid][v] = x;
  }
  __syncthreads();
  if (threadIdx.x < kDiagVals) {
    const int v = threadIdx.x;
    const bool ismax = (v == nt + 3 || v == nt + 4);
    double x = red[0][v];
    for (int w = 1; w < kDiagThreads / 32; ++w) x = ismax ? fmax(x, red[w][v]) : x + red[w][v];
    a.partial[(size_t)blockIdx.x * kDiagVals + v] = x;
  }
}

template <typename T>
__global__ void k_diag_final(const DiagArgs<T> a) {
  const int v = threadIdx.x;
  if (v >= kDiagVals) return;
  const int nt = a.nt;
  const bool ismax = (v == nt + 3 || v == nt + 4);
  double x = a.partial[v];
  for (int b = 1; b < a.nblocks; ++b) {
    const double y = a.partial[(size_t)b * kDiagVals + v];
    x = ismax ? fmax(x, y) : x + y;
  }
  a.out[v] = x;
}

template <typename T>
cudaError_t launch_diagnostics(const DiagArgs<T>& a, cudaStream_t s) {
  k_diag<T><<<a.nblocks, kDiagThreads, 0, s>>>(a);
  k_diag_final<T><<<1, 32, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_fill(T* p, size_t n, T v) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = v;
}
template <typename T>
__global__ void k_shift(T* p, size_t n, T v) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] += v;
}
template <typename T>
cudaError_t launch_fill(T* p, size_t n, T v, cudaStream_t s) {
  k_fill<T><<<1216, 256, 0, s>>>(p, n, v);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_shift(T* p, size_t n, T v, cudaStream_t s) {
  k_shift<T><<<1216, 256, 0, s>>>(p, n, v);
  return cudaGetLastError();
}

template <typename T>
__global__ void __launch_bounds__(256) k_level_mean(const T* p, size_t plane, T* ref) {
  const int k = blockIdx.x;
  const T* q = p + (size_t)k * plane;
  double acc = 0.0;
  for (size_t i = threadIdx.x; i < plane; i += blockDim.x) acc += (double)q[i];
  __shared__ double red[8];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    ref[k] = (T)(t / (double)plane);
  }
}
template <typename T>
__global__ void k_level_shift(T* p, size_t plane, int Nz, const T* ref, T sign) {
  const size_t n = plane * (size_t)Nz;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    p[i] += sign * ref[i / plane];
}
// dst = src + ref[level]: the same sum as a copy followed by k_level_shift with sign +1
template <typename T>
__global__ void k_level_add(T* __restrict__ dst, const T* __restrict__ src, size_t plane, int Nz, const T* ref) {
  const size_t n = plane * (size_t)Nz;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = src[i] + ref[i / plane];
}
template <typename T>
cudaError_t launch_level_mean(const T* p, size_t plane, int Nz, T* ref, cudaStream_t s) {
  k_level_mean<T><<<Nz, 256, 0, s>>>(p, plane, ref);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_level_shift(T* p, size_t plane, int Nz, const T* ref, T sign, cudaStream_t s) {
  k_level_shift<T><<<1216, 256, 0, s>>>(p, plane, Nz, ref, sign);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_level_add(T* dst, const T* src, size_t plane, int Nz, const T* ref, cudaStream_t s) {
  k_level_add<T><<<1216, 256, 0, s>>>(dst, src, plane, Nz, ref);
  return cudaGetLastError();
}
template cudaError_t launch_level_add<float>(float*, const float*, size_t, int, const float*, cudaStream_t);
template cudaError_t launch_level_add<double>(double*, const double*, size_t, int, const double*, cudaStream_t);
template cudaError_t launch_level_mean<float>(const float*, size_t, int, float*, cudaStream_t);
template cudaError_t launch_level_mean<double>(const double*, size_t, int, double*, cudaStream_t);
template cudaError_t launch_level_shift<float>(float*, size_t, int, const float*, float, cudaStream_t);
template cudaError_t launch_level_shift<double>(double*, size_t, int, const double*, double, cudaStream_t);

// One block per level: FP64 horizontal means of the tendencies and of u, v, b.
template <typename T>
__global__ void __launch_bounds__(256) k_profile_means(const ProfileArgs<T> a) {
  const int k = blockIdx.x;
  const size_t o = (size_t)k * a.plane;
  const double r0 = a.cref0 ? (double)a.cref0[k] : 0.0, r1 = a.cref1 ? (double)a.cref1[k] : 0.0;
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  for (size_t i = threadIdx.x; i < a.plane; i += blockDim.x) {
    acc[0] += (double)a.Gu[o + i];
    acc[1] += (double)a.Gv[o + i];
    acc[2] += (double)a.Gc0[o + i];
    if (a.Gc1) acc[3] += (double)a.Gc1[o + i];
    acc[4] += (double)a.u[o + i];
    acc[5] += (double)a.v[o + i];
    const double c0 = (double)a.c0[o + i] + r0;
    acc[6] += (a.eos == OCN_EOS_LINEAR_TS) ? a.g_alpha * (c0 - a.T0) - a.g_beta * ((double)a.c1[o + i] + r1 - a.S0) : c0;
  }
  __shared__ double red[8][7];
#pragma unroll
  for (int v = 0; v < 7; ++v) {
    double x = acc[v];
    for (int s = 16; s > 0; s >>= 1) x += __shfl_down_sync(0xffffffffu, x, s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][v] = x;
  }
  __syncthreads();
  if (threadIdx.x < 7) {
    double x = 0.0;
    for (int w = 0; w < 8; ++w) x += red[w][threadIdx.x];
    a.out[(size_t)threadIdx.x * a.Nz + k] = x / (double)a.plane;
  }
}
template <typename T>
cudaError_t launch_profile_means(const ProfileArgs<T>& a, cudaStream_t s) {
  k_profile_means<T><<<a.Nz, 256, 0, s>>>(a);
  return cudaGetLastError();
}
template cudaError_t launch_profile_means<float>(const ProfileArgs<float>&, cudaStream_t);
template cudaError_t launch_profile_means<double>(const ProfileArgs<double>&, cudaStream_t);

template cudaError_t launch_diagnostics<float>(const DiagArgs<float>&, cudaStream_t);
template cudaError_t launch_diagnostics<double>(const DiagArgs<double>&, cudaStream_t);
template cudaError_t launch_fill<float>(float*, size_t, float, cudaStream_t);
template cudaError_t launch_fill<double>(double*, size_t, double, cudaStream_t);
template cudaError_t launch_shift<float>(float*, size_t, float, cudaStream_t);
template cudaError_t launch_shift<double>(double*, size_t, double, cudaStream_t);

}  // namespace ocn
