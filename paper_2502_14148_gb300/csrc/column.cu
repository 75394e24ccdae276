// Column kernels of the learned closure: mixed-layer depth estimate, raw features,
// the closure's own vertical fluxes, box coarse-graining of a fine state (training
// data) and the face-flux divergence added to the tendencies.
#include <cuda_runtime.h>

#include "batch.cuh"
#include "column.cuh"

namespace ocn {
namespace {

// h = sum over interior faces of max(0, 1 - (db/dz)/N2bg) dzf (0 when N2bg <= 0): one thread per column.
__device__ __forceinline__ void column_h_body(const ColumnArgs& a, const uint3 bid) {
  const int c = bid.x * blockDim.x + threadIdx.x;
  if (c >= a.Nx * a.Ny) return;
  const int i = c % a.Nx, j = c / a.Nx;
  float acc = 0.0f;
  if (a.N2bg > 0.0f) {
    const float inv = 1.0f / a.N2bg;
    for (int k = 1; k < a.Nz; ++k) {
      const float def = 1.0f - col_grad(a, 0, i, j, k) * inv;
      if (def > 0.0f) acc += def * a.dzf[k];
    }
  }
  a.h[c] = acc;
}

__global__ void k_closure_features(const ColumnArgs a, float* X) {
  const size_t plane = (size_t)a.Nx * a.Ny, n = plane * (a.Nz + 1);
  for (size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x; s < n; s += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(s / plane), c = (int)(s % plane), i = c % a.Nx, j = c / a.Nx;
    float x[kColumnFeatures];
#pragma unroll
    for (int q = 0; q < kColumnFeatures; ++q) x[q] = 0.0f;
    column_features_b(a, i, j, k, x);
    column_features_uv(a, i, j, k, x);
    float4* o = reinterpret_cast<float4*>(X + s * kColumnFeatures);
#pragma unroll
    for (int q = 0; q < kColumnFeatures / 4; ++q) o[q] = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
  }
}

// face diffusivities of the closure: q = 0 tracer, else momentum
__device__ __forceinline__ float face_diff(const ColumnArgs& a, int q, size_t id0, size_t id1) {
  if (a.closure == OCN_CLOSURE_SCALAR) return q == 0 ? a.kappa0 : a.nu0;
  if (a.closure == OCN_CLOSURE_NONE) return 0.0f;
  if (q == 0) {
    if (a.closure == OCN_CLOSURE_AMD) return 0.5f * (a.kap[id0] + a.kap[id1]);
    return 0.5f * a.inv_Pr * (a.nu[id0] + a.nu[id1]);
  }
  return 0.5f * (a.nu[id0] + a.nu[id1]);
}

__global__ void k_column_sgs_flux(const ColumnArgs a, float* F) {
  const size_t plane = (size_t)a.Nx * a.Ny, NW = plane * (a.Nz + 1);
  for (size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x; s < NW; s += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(s / plane), c = (int)(s % plane), i = c % a.Nx, j = c / a.Nx;
    float f0 = 0.0f, f1 = 0.0f, f2 = 0.0f;
    if (k > 0 && k < a.Nz) {
      const size_t id0 = col_id(a, i, j, k - 1), id1 = col_id(a, i, j, k);
      f0 = -face_diff(a, 0, id0, id1) * col_grad(a, 0, i, j, k);
      const float nuf = face_diff(a, 1, id0, id1);
      f1 = -nuf * col_grad(a, 1, i, j, k);
      f2 = -nuf * col_grad(a, 2, i, j, k);
    }
    F[s] = f0; F[NW + s] = f1; F[2 * NW + s] = f2;
  }
}

// One thread per (coarse column, fine level/face); FP64 box sums.
__global__ void k_coarse_grain(const ColumnArgs a, int cx, int cy, double* out) {
  const int rx = a.Nx / cx, ry = a.Ny / cy, Nz = a.Nz;
  const size_t cp = (size_t)cx * cy;
  const size_t n = cp * (Nz + 1);
  double* uc = out;
  double* vc = uc + (size_t)Nz * cp;
  double* wc = vc + (size_t)Nz * cp;
  double* bc = wc + (size_t)(Nz + 1) * cp;
  double* tau = bc + (size_t)Nz * cp;
  const double inv = 1.0 / ((double)rx * ry);
  for (size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x; s < n; s += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(s / cp), cc = (int)(s % cp), I = cc % cx, J = cc / cx;
    double su = 0, sv = 0, sw = 0, sb = 0;
    double swq[3] = {0, 0, 0}, sq[3] = {0, 0, 0}, ssgs[3] = {0, 0, 0};
    for (int jj = 0; jj < ry; ++jj)
      for (int ii = 0; ii < rx; ++ii) {
        const int i = I * rx + ii, j = J * ry + jj;
        const double w = a.w[col_id(a, i, j, k)];
        sw += w;
        if (k < Nz) {
          sb += a.b[col_id(a, i, j, k)];
          if (ii == 0) su += a.u[col_id(a, i, j, k)];
          if (jj == 0) sv += a.v[col_id(a, i, j, k)];
        }
        if (k > 0 && k < Nz) {
          const size_t id0 = col_id(a, i, j, k - 1), id1 = col_id(a, i, j, k);
          const int ip = (i + 1 == a.Nx) ? 0 : i + 1, jp = (j + 1 == a.Ny) ? 0 : j + 1;
          // face values (b as the stored anomaly: the covariance is unchanged by the per-level shift)
          const double qf0 = 0.5 * ((double)a.b[id0] + a.b[id1]);
          const double qf1 = 0.25 * ((double)a.u[id0] + a.u[col_id(a, ip, j, k - 1)] + a.u[id1] + a.u[col_id(a, ip, j, k)]);
          const double qf2 = 0.25 * ((double)a.v[id0] + a.v[col_id(a, i, jp, k - 1)] + a.v[id1] + a.v[col_id(a, i, jp, k)]);
          swq[0] += w * qf0; sq[0] += qf0;
          swq[1] += w * qf1; sq[1] += qf1;
          swq[2] += w * qf2; sq[2] += qf2;
          const float nuf = face_diff(a, 1, id0, id1);
          ssgs[0] += -(double)face_diff(a, 0, id0, id1) * col_grad(a, 0, i, j, k);
          ssgs[1] += -(double)nuf * col_grad(a, 1, i, j, k);
          ssgs[2] += -(double)nuf * col_grad(a, 2, i, j, k);
        }
      }
    wc[s] = sw * inv;
    if (k < Nz) {
      bc[s] = sb * inv + (a.cref ? (double)a.cref[k] : 0.0);
      uc[s] = su / ry;
      vc[s] = sv / rx;
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      double t = 0.0;
      if (k > 0 && k < Nz) t = swq[q] * inv - (sw * inv) * (sq[q] * inv) + ssgs[q] * inv;
      tau[(size_t)q * (Nz + 1) * cp + s] = t;
    }
  }
}

__device__ __forceinline__ void apply_face_flux_body(const FaceFluxArgs& a, const uint3 bid, const uint3 gdim) {
  const size_t plane = (size_t)a.Nx * a.Ny, N = plane * a.Nz, NW = plane * (a.Nz + 1);
  const float* Fb = a.F;
  const float* Fu = a.F + NW;
  const float* Fv = a.F + 2 * NW;
  for (size_t s = bid.x * (size_t)blockDim.x + threadIdx.x; s < N; s += (size_t)gdim.x * blockDim.x) {
    const int k = (int)(s / plane), c = (int)(s % plane), i = c % a.Nx, j = c / a.Nx;
    const int im = (i == 0) ? a.Nx - 1 : i - 1, jm = (j == 0) ? a.Ny - 1 : j - 1;
    const size_t lo = (size_t)k * plane, hi = lo + plane;
    const float r = a.rdzc[k];
    const float dGb = -(Fb[hi + c] - Fb[lo + c]) * r;
    const size_t cim = (size_t)j * a.Nx + im, cjm = (size_t)jm * a.Nx + i;
    const float dGu = -0.5f * ((Fu[hi + cim] + Fu[hi + c]) - (Fu[lo + cim] + Fu[lo + c])) * r;
    const float dGv = -0.5f * ((Fv[hi + cjm] + Fv[hi + c]) - (Fv[lo + cjm] + Fv[lo + c])) * r;
    a.Gb[s] += dGb; a.Gu[s] += dGu; a.Gv[s] += dGv;
    if (a.mode == 0) {
      a.nb[s] += a.dt_gamma * dGb;
      a.nu_[s] += a.dt_gamma * dGu;
      a.nv[s] += a.dt_gamma * dGv;
    }
  }
}

struct ColumnHK {
  typedef ColumnArgs Payload;
  static constexpr int kThreads = 128, kMinBlocks = 1;
  static __device__ __forceinline__ void run(const Payload& a, uint3 bid, uint3) { column_h_body(a, bid); }
};
struct ApplyFaceFluxK {
  typedef FaceFluxArgs Payload;
  static constexpr int kThreads = 256, kMinBlocks = 1;
  static __device__ __forceinline__ void run(const Payload& a, uint3 bid, uint3 g) { apply_face_flux_body(a, bid, g); }
};
// One block per face k: the plane means of F[0][k] and F[1][k] (FP64 sums), 0 at the walls.
constexpr int kFaceMeanThreads = 256;
__device__ __forceinline__ void face_mean_body(const FaceMeanArgs& a, const uint3 bid) {
  const int k = bid.x;
  const size_t plane = (size_t)a.Nx * a.Ny, NW = plane * (a.Nz + 1);
  double s0 = 0.0, s1 = 0.0;
  if (k > 0 && k < a.Nz) {
    const float* f0 = a.F + (size_t)k * plane;
    const float* f1 = f0 + NW;
    for (size_t i = threadIdx.x; i < plane; i += kFaceMeanThreads) {
      s0 += (double)f0[i];
      s1 += (double)f1[i];
    }
  }
  __shared__ double r0[kFaceMeanThreads / 32], r1[kFaceMeanThreads / 32];
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_down_sync(0xffffffffu, s0, o);
    s1 += __shfl_down_sync(0xffffffffu, s1, o);
  }
  if ((threadIdx.x & 31) == 0) { r0[threadIdx.x >> 5] = s0; r1[threadIdx.x >> 5] = s1; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0.0, t1 = 0.0;
    for (int w = 0; w < kFaceMeanThreads / 32; ++w) { t0 += r0[w]; t1 += r1[w]; }
    a.p0[k] = (float)(t0 / (double)plane);
    a.p1[k] = (float)(t1 / (double)plane);
  }
}
struct FaceMeanK {
  typedef FaceMeanArgs Payload;
  static constexpr int kThreads = kFaceMeanThreads, kMinBlocks = 1;
  static __device__ __forceinline__ void run(const Payload& a, uint3 bid, uint3) { face_mean_body(a, bid); }
};
__global__ void __launch_bounds__(kFaceMeanThreads) k_face_mean(const FaceMeanArgs a) { face_mean_body(a, blockIdx); }

__global__ void k_column_h(const ColumnArgs a) { column_h_body(a, blockIdx); }
__global__ void k_apply_face_flux(const FaceFluxArgs a) { apply_face_flux_body(a, blockIdx, gridDim); }

int blocks_for(size_t n) {
  size_t b = (n + 255) / 256;
  return (int)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

}  // namespace

cudaError_t launch_column_h(const ColumnArgs& a, cudaStream_t s) {
  const int n = a.Nx * a.Ny;
  if (record_launch<ColumnHK>(a, dim3((n + 127) / 128), dim3(128), 0, OCN_K_COLUMN_CLOSURE)) return cudaSuccess;
  k_column_h<<<(n + 127) / 128, 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_closure_features(const ColumnArgs& a, float* X, cudaStream_t s) {
  cudaError_t e = launch_column_h(a, s);
  if (e != cudaSuccess) return e;
  k_closure_features<<<blocks_for((size_t)a.Nx * a.Ny * (a.Nz + 1)), 256, 0, s>>>(a, X);
  return cudaGetLastError();
}

cudaError_t launch_column_sgs_flux(const ColumnArgs& a, float* F, cudaStream_t s) {
  k_column_sgs_flux<<<blocks_for((size_t)a.Nx * a.Ny * (a.Nz + 1)), 256, 0, s>>>(a, F);
  return cudaGetLastError();
}

cudaError_t launch_coarse_grain(const ColumnArgs& a, int cx, int cy, double* out, cudaStream_t s) {
  if (cx < 1 || cy < 1 || a.Nx % cx || a.Ny % cy) return cudaErrorInvalidValue;
  const size_t n = (size_t)cx * cy * (a.Nz + 1);
  k_coarse_grain<<<(int)((n + 127) / 128), 128, 0, s>>>(a, cx, cy, out);
  return cudaGetLastError();
}

cudaError_t launch_face_mean(const FaceMeanArgs& a, cudaStream_t s) {
  const dim3 grid(a.Nz + 1);
  if (record_launch<FaceMeanK>(a, grid, dim3(kFaceMeanThreads), 0, OCN_K_COLUMN_CLOSURE)) return cudaSuccess;
  k_face_mean<<<grid, kFaceMeanThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_apply_face_flux(const FaceFluxArgs& a, cudaStream_t s) {
  const dim3 grid(blocks_for((size_t)a.Nx * a.Ny * a.Nz));
  if (record_launch<ApplyFaceFluxK>(a, grid, dim3(256), 0, OCN_K_COLUMN_CLOSURE)) return cudaSuccess;
  k_apply_face_flux<<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ocn
