// Batched twins (ensembles) of the FP64 tendency kernels.
#include "tendency_kernel.cuh"

namespace ocn {

template <typename T, int R, int NTR, int TX, int TY, int MINB, int CL>
const void* tendency_batched_kernel() {
  return reinterpret_cast<const void*>(&k_batched<TendencyK<T, R, NTR, TX, TY, MINB, CL>>);
}

template const void* tendency_batched_kernel<double, 3, 1, 32, 8, 1, kClAny>();
template const void* tendency_batched_kernel<double, 3, 2, 32, 8, 1, kClAny>();
template const void* tendency_batched_kernel<double, 5, 1, 32, 8, 1, kClAny>();
template const void* tendency_batched_kernel<double, 5, 2, 32, 8, 1, kClAny>();

cudaError_t upload_tables_f64_batch(const WenoTables<double>& t) { return upload_tables_here(t); }

}  // namespace ocn
