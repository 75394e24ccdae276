// Batched twins (ensembles) of the FP32 WENO5 tendency kernels, Smagorinsky-Lilly closure class, one per tile
// variant.
#include "tendency_kernel.cuh"

namespace ocn {

template <typename T, int R, int NTR, int TX, int TY, int MINB, int CL>
const void* tendency_batched_kernel() {
  return reinterpret_cast<const void*>(&k_batched<TendencyK<T, R, NTR, TX, TY, MINB, CL>>);
}

#define OCN_INST(R, NTR, TX, TY, MINB, CL) template const void* tendency_batched_kernel<float, R, NTR, TX, TY, MINB, CL>();
OCN_F32_TILE_VARIANTS(OCN_INST, 3, 1, kClSmag)
OCN_F32_TILE_VARIANTS(OCN_INST, 3, 2, kClSmag)

}  // namespace ocn
