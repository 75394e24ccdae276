// Fused tendency kernels in FP32, WENO order 5 (R = 3): the dispatch over tracer count, closure
// class and tile variant, and the constant-diffusivity class.  The Smagorinsky-Lilly and AMD classes
// are compiled in tendency_f32_r3_smag.cu and tendency_f32_r3_amd.cu (so that the translation
// units build in parallel).
#include "tendency_kernel.cuh"

namespace ocn {

#define OCN_EXTERN(R, NTR, TX, TY, MINB, CL) \
  extern template cudaError_t launch_tendency_variant<float, R, NTR, TX, TY, MINB, CL>(const TendencyArgs<float>&, \
                                                                                      cudaStream_t);
OCN_F32_TILE_VARIANTS(OCN_EXTERN, 3, 1, kClSmag)
OCN_F32_TILE_VARIANTS(OCN_EXTERN, 3, 2, kClSmag)
OCN_F32_TILE_VARIANTS(OCN_EXTERN, 3, 1, kClAmd)
OCN_F32_TILE_VARIANTS(OCN_EXTERN, 3, 2, kClAmd)

template <int NTR, int CL>
static cudaError_t launch_f32_r3_ncl(const TendencyArgs<float>& a, cudaStream_t s) {
  switch (a.variant) {
    case 0: return launch_tendency_variant<float, 3, NTR, 32, 8, 1, CL>(a, s);
    case 1: return launch_tendency_variant<float, 3, NTR, 32, 8, 2, CL>(a, s);
    case 2: return launch_tendency_variant<float, 3, NTR, 32, 16, 1, CL>(a, s);
    case 3: return launch_tendency_variant<float, 3, NTR, 32, 4, 3, CL>(a, s);
    case 4: return launch_tendency_variant<float, 3, NTR, 32, 14, 1, CL>(a, s);
    case 5: return launch_tendency_variant<float, 3, NTR, 32, 12, 1, CL>(a, s);
    case 6: return launch_tendency_variant<float, 3, NTR, 16, 16, 2, CL>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int NTR>
static cudaError_t launch_f32_r3_n(const TendencyArgs<float>& a, cudaStream_t s) {
  switch (closure_class(a.closure)) {
    case kClSmag: return launch_f32_r3_ncl<NTR, kClSmag>(a, s);
    case kClAmd: return launch_f32_r3_ncl<NTR, kClAmd>(a, s);
    default: return launch_f32_r3_ncl<NTR, kClScalar>(a, s);
  }
}

cudaError_t launch_tendency_f32_r3(const TendencyArgs<float>& a, cudaStream_t s) {
  switch (a.nt) {
    case 1: return launch_f32_r3_n<1>(a, s);
    case 2: return launch_f32_r3_n<2>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ocn
