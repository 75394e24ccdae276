// Fused tendency kernels: float, WENO order 5 (R = 3).
#include "tendency_kernel.cuh"

namespace ocn {

template <int NTR>
static cudaError_t launch_f32_r3_n(const TendencyArgs<float>& a, cudaStream_t s) {
  switch (a.variant) {
      case 0: return launch_tendency_variant<float, 3, NTR, 32, 8, 1>(a, s);
      case 1: return launch_tendency_variant<float, 3, NTR, 32, 8, 2>(a, s);
      case 2: return launch_tendency_variant<float, 3, NTR, 32, 16, 1>(a, s);
      case 3: return launch_tendency_variant<float, 3, NTR, 32, 4, 3>(a, s);
      case 4: return launch_tendency_variant<float, 3, NTR, 32, 14, 1>(a, s);
      case 5: return launch_tendency_variant<float, 3, NTR, 32, 12, 1>(a, s);
      case 6: return launch_tendency_variant<float, 3, NTR, 16, 16, 2>(a, s);
      default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_tendency_f32_r3(const TendencyArgs<float>& a, cudaStream_t s) {
  switch (a.nt) {
    case 1: return launch_f32_r3_n<1>(a, s);
    case 2: return launch_f32_r3_n<2>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t upload_tables_f32_r3(const WenoTables<double>& t) { return upload_tables_here(t); }

}  // namespace ocn
