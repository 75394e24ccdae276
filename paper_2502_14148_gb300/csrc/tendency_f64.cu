// Fused tendency kernels in FP64 (parity configurations), WENO5 and WENO9.
#include "tendency_kernel.cuh"

namespace ocn {

template <int R, int NTR>
static cudaError_t launch_f64_rn(const TendencyArgs<double>& a, cudaStream_t s) {
  return launch_tendency_variant<double, R, NTR, 32, 8, 1, kClAny>(a, s);
}

cudaError_t launch_tendency_f64(const TendencyArgs<double>& a, int weno_r, cudaStream_t s) {
  if (weno_r == 3) return a.nt == 1 ? launch_f64_rn<3, 1>(a, s) : (a.nt == 2 ? launch_f64_rn<3, 2>(a, s) : cudaErrorInvalidValue);
  if (weno_r == 5) return a.nt == 1 ? launch_f64_rn<5, 1>(a, s) : (a.nt == 2 ? launch_f64_rn<5, 2>(a, s) : cudaErrorInvalidValue);
  return cudaErrorInvalidValue;
}

cudaError_t upload_tables_f64(const WenoTables<double>& t) { return upload_tables_here(t); }

// Dispatch by precision and order; float tile variants are selected by a.variant.
template <>
cudaError_t launch_tendency<float>(const TendencyArgs<float>& a, int weno_r, cudaStream_t s) {
  if (weno_r == 5) return launch_tendency_f32_r5(a, s);
  if (weno_r == 3) return launch_tendency_f32_r3(a, s);
  return cudaErrorInvalidValue;
}
template <>
cudaError_t launch_tendency<double>(const TendencyArgs<double>& a, int weno_r, cudaStream_t s) {
  return launch_tendency_f64(a, weno_r, s);
}

cudaError_t upload_weno_tables(const WenoTables<double>& t) {
  // only the FP64 kernels read the tables (the FP32 kernels use compile-time coefficients)
  cudaError_t e = upload_tables_f64(t);
  if (e == cudaSuccess) e = upload_tables_f64_batch(t);
  return e;
}

}  // namespace ocn
