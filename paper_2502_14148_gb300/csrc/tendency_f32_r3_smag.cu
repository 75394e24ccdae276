// Fused tendency kernels in FP32, WENO order 5 (R = 3), Smagorinsky-Lilly closure class, every tile variant.
#include "tendency_kernel.cuh"

namespace ocn {

#define OCN_INST(R, NTR, TX, TY, MINB, CL) \
  template cudaError_t launch_tendency_variant<float, R, NTR, TX, TY, MINB, CL>(const TendencyArgs<float>&, cudaStream_t);
OCN_F32_TILE_VARIANTS(OCN_INST, 3, 1, kClSmag)
OCN_F32_TILE_VARIANTS(OCN_INST, 3, 2, kClSmag)

}  // namespace ocn
