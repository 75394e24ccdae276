// Fused tendency kernels in FP32, WENO order 9 (R = 5), AMD closure class, every tile variant.
#include "tendency_kernel.cuh"

namespace ocn {

#define OCN_INST(R, NTR, TX, TY, MINB, CL) \
  template cudaError_t launch_tendency_variant<float, R, NTR, TX, TY, MINB, CL>(const TendencyArgs<float>&, cudaStream_t);
OCN_F32_TILE_VARIANTS(OCN_INST, 5, 1, kClAmd)
OCN_F32_TILE_VARIANTS(OCN_INST, 5, 2, kClAmd)

}  // namespace ocn
