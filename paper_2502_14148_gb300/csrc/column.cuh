// Device helpers of the learned column closure: column quantities, their vertical
// gradients and the raw feature vector of one w-face (shared by the feature kernel
// and the fused tensor-core closure kernel).
#pragma once

#include "ocn_internal.cuh"

namespace ocn {

__device__ __forceinline__ size_t col_id(const ColumnArgs& a, int i, int j, int k) {
  return ((size_t)k * a.Ny + j) * a.Nx + i;
}
// d q / dz across face k for q = 0 (b), 1 (ubar), 2 (vbar); zero outside the interior faces.
__device__ __forceinline__ float col_grad(const ColumnArgs& a, int q, int i, int j, int k) {
  if (k <= 0 || k >= a.Nz) return 0.0f;
  float d;
  if (q == 0) {
    d = a.b[col_id(a, i, j, k)] - a.b[col_id(a, i, j, k - 1)];
    if (a.cref) d += a.cref[k] - a.cref[k - 1];
  } else if (q == 1) {
    const int ip = (i + 1 == a.Nx) ? 0 : i + 1;
    d = 0.5f * ((a.u[col_id(a, i, j, k)] + a.u[col_id(a, ip, j, k)]) -
                (a.u[col_id(a, i, j, k - 1)] + a.u[col_id(a, ip, j, k - 1)]));
  } else {
    const int jp = (j + 1 == a.Ny) ? 0 : j + 1;
    d = 0.5f * ((a.v[col_id(a, i, j, k)] + a.v[col_id(a, i, jp, k)]) -
                (a.v[col_id(a, i, j, k - 1)] + a.v[col_id(a, i, jp, k - 1)]));
  }
  return d * a.rdzf[k];
}
// Raw features 0..19 of face k of column (i, j):
// 0-4 db/dz at faces k-2..k+2, 5-9 dubar/dz, 10-14 dvbar/dz, 15 Jb, 16 f, 17 N2bg, 18 depth, 19 h.
__device__ __forceinline__ void column_features_b(const ColumnArgs& a, int i, int j, int k, float* x) {
#pragma unroll
  for (int m = -2; m <= 2; ++m) x[m + 2] = col_grad(a, 0, i, j, k + m);
  x[15] = a.Jb; x[16] = a.f; x[17] = a.N2bg;
  x[18] = a.depth[k];
  x[19] = a.h[(size_t)j * a.Nx + i];
}
__device__ __forceinline__ void column_features_uv(const ColumnArgs& a, int i, int j, int k, float* x) {
#pragma unroll
  for (int m = -2; m <= 2; ++m) {
    x[5 + m + 2] = col_grad(a, 1, i, j, k + m);
    x[10 + m + 2] = col_grad(a, 2, i, j, k + m);
  }
}
}  // namespace ocn
