// Batched twins (ensembles) of the FP32 WENO9 tendency kernels, one per tile variant.
#include "tendency_kernel.cuh"

namespace ocn {

template <typename T, int R, int NTR, int TX, int TY, int MINB>
const void* tendency_batched_kernel() {
  return reinterpret_cast<const void*>(&k_batched<TendencyK<T, R, NTR, TX, TY, MINB>>);
}

template const void* tendency_batched_kernel<float, 5, 1, 32, 8, 1>();
template const void* tendency_batched_kernel<float, 5, 1, 32, 8, 2>();
template const void* tendency_batched_kernel<float, 5, 1, 32, 16, 1>();
template const void* tendency_batched_kernel<float, 5, 1, 32, 4, 3>();
template const void* tendency_batched_kernel<float, 5, 1, 32, 14, 1>();
template const void* tendency_batched_kernel<float, 5, 1, 32, 12, 1>();
template const void* tendency_batched_kernel<float, 5, 1, 16, 16, 2>();
template const void* tendency_batched_kernel<float, 5, 2, 32, 8, 1>();
template const void* tendency_batched_kernel<float, 5, 2, 32, 8, 2>();
template const void* tendency_batched_kernel<float, 5, 2, 32, 16, 1>();
template const void* tendency_batched_kernel<float, 5, 2, 32, 4, 3>();
template const void* tendency_batched_kernel<float, 5, 2, 32, 14, 1>();
template const void* tendency_batched_kernel<float, 5, 2, 32, 12, 1>();
template const void* tendency_batched_kernel<float, 5, 2, 16, 16, 2>();

cudaError_t upload_tables_f32_r5_batch(const WenoTables<double>& t) { return upload_tables_here(t); }

}  // namespace ocn
