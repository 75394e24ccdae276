// Measured FP32 FMA throughput of this GPU: the denominator of the tendency kernel's ALU roofline.
// Every thread runs 8 independent FMA chains (enough to cover the pipeline latency) for `iters`
// rounds; the grid is 8 CTAs of 512 threads per SM.
#include <cuda_runtime.h>

#include "ocn_internal.cuh"

namespace ocn {
namespace {

__global__ void __launch_bounds__(512) k_fma_peak(float* out, int iters, float a, float b) {
  float x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int c = 0; c < 8; ++c) x[c] = fmaf(x[c], a, b);
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += x[c];
  if (s == 12345.678f) out[threadIdx.x] = s;   // keeps the chains alive; never true for these inputs
}

}  // namespace
}  // namespace ocn

extern "C" ocn_status ocn_fp32_fma_peak(double* tflops, void* stream) {
  if (!tflops) return ocn::set_last_error(OCN_ERR_ARG, "null pointer");
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return ocn::set_last_error(OCN_ERR_CUDA, cudaGetErrorString(e));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int blocks = 8 * nsm, threads = 512, iters = 4096;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float ms = 0.0f;
  if (e == cudaSuccess) {
    ocn::k_fma_peak<<<blocks, threads, 0, s>>>(nullptr, 64, 0.999f, 1e-4f);    // warm-up
    e = cudaEventRecord(e0, s);
    ocn::k_fma_peak<<<blocks, threads, 0, s>>>(nullptr, iters, 0.999f, 1e-4f);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return ocn::set_last_error(OCN_ERR_CUDA, cudaGetErrorString(e));
  const double flops = 2.0 * 8.0 * 16.0 * iters * (double)blocks * threads;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return OCN_OK;
}
