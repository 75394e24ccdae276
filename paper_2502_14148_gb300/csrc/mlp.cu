// Tensor-core GEMMs of the learned column closure (BF16 operands, FP32
// accumulation) on the 5th-generation tensor cores: tcgen05.mma issued by one
// thread, operands staged in shared memory in the no-swizzle K-major
// core-matrix layout, the accumulator in tensor memory (TMEM) read back with
// tcgen05.ld for the epilogue.  One kernel serves every product of the network:
//   D[M x N] = A[M x K] . B[N x K]^T        (A, B BF16, K contiguous)
// with epilogues for the hidden layers (bias + GELU, BF16 activations and their
// transpose), the output layer (bias), the backward pass (times GELU'(z)) and
// split-K FP32 partials (weight gradients, K = samples).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>
#include <stdio.h>
#include <math.h>

#include <algorithm>
#include <new>

#include "batch.cuh"
#include "column.cuh"
#include "ocn_internal.cuh"

namespace ocn {

namespace {

constexpr int kTileM = 128;      // rows per CTA (TMEM lanes)
constexpr int kChunkK = 64;      // K staged per round (4 MMA steps of 16)
constexpr int kMaxN = 256;
constexpr int kGemmSmem = 80 * 1024;   // >= 76 KB keeps at most two CTAs (2 x 256 TMEM columns) per SM

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait: false when the phase did not complete within about half a second.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t phase) {
  const uint64_t t0 = globaltimer_ns();
  for (int it = 0; it < (1 << 22); ++it) {
    if (mbar_try_wait(bar, phase)) return true;
    if ((it & 255) == 255 && globaltimer_ns() - t0 > 500000000ull) return false;
  }
  return false;
}
__device__ __forceinline__ void fence_barrier_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {   // one full warp
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {   // one full warp
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Shared-memory matrix descriptor: start, leading (K-direction) and stride
// (M/N-direction) byte offsets between 8x16-byte core matrices, version 1,
// no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
// Instruction descriptor, kind::f16: F32 accumulator, BF16 A and B, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
          d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// 32 lanes x 32 bits, 16 consecutive columns per thread.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 lanes x 32 bits, 32 consecutive columns per thread (one load, one wait).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Split form for software pipelining: the load's registers are not valid until tmem_wait16
// (which names them as operands, so that no use is scheduled before it).
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_wait16(uint32_t (&r)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
}

// GELU evaluated in the tanh form of Hendrycks & Gimpel (2016),
//   gelu(z) ~ z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))),
// with the hardware tanh approximation.  Its largest deviation from the erf definition
// z Phi(z) is 4.7e-4 (at z = 2.7, where gelu = 2.69), well inside the BF16 rounding that the
// activation receives next; gelu_prime_f is the derivative of the same form.
__device__ __forceinline__ float tanh_fast(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
constexpr float kGeluK = 0.7978845608028654f;    // sqrt(2/pi)
constexpr float kGeluC = 0.044715f;
constexpr float kGeluKC = kGeluK * kGeluC;
__device__ __forceinline__ float gelu_f(float z) {
  const float t = tanh_fast(z * fmaf(kGeluKC, z * z, kGeluK));
  const float hz = 0.5f * z;
  return fmaf(hz, t, hz);
}
// The same form on two BF16 values at once (packed BF16 arithmetic and the packed hardware tanh),
// for the inference epilogue, whose result is rounded to BF16 anyway: every operation rounds to
// BF16, which raises the network's output error from about 2.5 to 3.5 BF16 units (emulated on
// N(0,1) features with the seeded initial weights), inside the 16-unit tolerance.
__device__ __forceinline__ uint32_t tanh_bf16x2(uint32_t x) {
  uint32_t y;
  asm("tanh.approx.bf16x2 %0, %1;" : "=r"(y) : "r"(x));
  return y;
}
__device__ __forceinline__ uint32_t gelu_bf16x2(__nv_bfloat162 z) {
  const __nv_bfloat162 k = __float2bfloat162_rn(kGeluK), kc = __float2bfloat162_rn(kGeluKC);
  const __nv_bfloat162 half = __float2bfloat162_rn(0.5f);
  const __nv_bfloat162 u = __hmul2(z, __hfma2(kc, __hmul2(z, z), k));
  const uint32_t tu = tanh_bf16x2(*reinterpret_cast<const uint32_t*>(&u));
  const __nv_bfloat162 t = *reinterpret_cast<const __nv_bfloat162*>(&tu);
  const __nv_bfloat162 hz = __hmul2(half, z);
  const __nv_bfloat162 g = __hfma2(hz, t, hz);
  return *reinterpret_cast<const uint32_t*>(&g);
}
__device__ __forceinline__ float gelu_prime_f(float z) {
  const float z2 = z * z;
  const float t = tanh_fast(kGeluK * fmaf(kGeluC * z, z2, z));
  return 0.5f * (1.0f + t) + 0.5f * z * (1.0f - t * t) * kGeluK * fmaf(3.0f * kGeluC, z2, 1.0f);
}

// Copy a rows x kChunkK BF16 tile (row r, columns k0..k0+63 of a [rows][ld] array) into the
// core-matrix layout: byte (r/8)*SBO + (k/8)*128 + (r%8)*16 + (k%8)*2, SBO = 8*128.  Rows >= nrows
// and columns >= kend are zero.
__device__ __forceinline__ void stage_tile(unsigned char* s, const __nv_bfloat16* g, int ld, int row0, int nrows,
                                           int rows, int k0, int kend) {
  constexpr int cpr = kChunkK / 8;   // 16-byte chunks per row
  for (int c = threadIdx.x; c < rows * cpr; c += blockDim.x) {
    const int r = c / cpr, kc = c % cpr;
    const int gr = row0 + r, gk = k0 + 8 * kc;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (gr < nrows && gk < kend) v = *reinterpret_cast<const uint4*>(g + (size_t)gr * ld + gk);
    *reinterpret_cast<uint4*>(s + (r >> 3) * (cpr * 128) + kc * 128 + (r & 7) * 16) = v;
  }
}

}  // namespace

__global__ void __launch_bounds__(128, 1) k_gemm_tc(const GemmArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA = smem;                            // 128 x 64 BF16 = 16 KB
  unsigned char* sB = smem + kTileM * kChunkK * 2;     // <= 256 x 64 BF16 = 32 KB
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kTileM;
  const int kb = blockIdx.y * a.kchunk, ke = min(a.K, kb + a.kchunk);
  const int N = a.N;
  const uint32_t ncols = (N <= 32) ? 32u : (N <= 64 ? 64u : (N <= 128 ? 128u : 256u));
  if (warp == 0) tmem_alloc(&tmem_base, ncols);
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = idesc_bf16(kTileM, N);
  constexpr uint32_t kSBO = (kChunkK / 8) * 128;
  uint32_t phase = 0;
  bool ok = true, any = false;
  for (int k0 = kb; k0 < ke && ok; k0 += kChunkK) {
    stage_tile(sA, static_cast<const __nv_bfloat16*>(a.A), a.lda, m0, a.M, kTileM, k0, ke);
    stage_tile(sB, static_cast<const __nv_bfloat16*>(a.B), a.ldb, 0, N, N, k0, ke);
    fence_proxy_async();
    __syncthreads();
    if (tid == 0 && !a.no_issue) {
      tc_fence_after();
      const int steps = (min(kChunkK, ke - k0) + 15) / 16;
      for (int s = 0; s < steps; ++s) {
        const uint64_t ad = smem_desc(smem_u32(sA) + s * 256, 128, kSBO);
        const uint64_t bd = smem_desc(smem_u32(sB) + s * 256, 128, kSBO);
        mma_bf16(tmem, ad, bd, idesc, any ? 1u : 0u);
        any = true;
      }
      mma_commit(&bar);
    }
    const bool done = mbar_wait_bounded(&bar, phase);   // the MMAs have read shared memory and written TMEM
    phase ^= 1u;
    tc_fence_after();
    ok = __syncthreads_and(done) != 0;                  // uniform across the CTA
    any = __syncthreads_or(any) != 0;
  }
  if (!ok) {
    if (tid == 0 && a.status) atomicExch(a.status, 1);
    mbar_wait_bounded(&bar, phase ^ 1u);   // give an in-flight commit a bounded chance to land
  }
  // ---- epilogue: warp w owns TMEM lanes (rows) 32w .. 32w+31
  const int row = m0 + warp * 32 + lane;
  if (ok) {
    for (int c0 = 0; c0 < N; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (!any) {
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = 0.0f;
      }
      if (row >= a.M) continue;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int col = c0 + i;
        if (col >= N) break;
        float x = v[i];
        if (a.mode == 0) {
          a.D[((size_t)blockIdx.y * a.M + row) * a.ldd + col] = x;
        } else if (a.mode == 1) {
          const float z = x + a.bias[col];
          if (a.D) a.D[(size_t)row * a.ldd + col] = z;
          const float h = gelu_f(z);
          static_cast<__nv_bfloat16*>(a.H)[(size_t)row * a.ldh + col] = __float2bfloat16_rn(h);
          if (a.HT) static_cast<__nv_bfloat16*>(a.HT)[(size_t)col * a.ldht + row] = __float2bfloat16_rn(h);
        } else if (a.mode == 2) {
          a.D[(size_t)row * a.ldd + col] = x + a.bias[col];
        } else {
          const float gz = x * gelu_prime_f(a.Z[(size_t)row * a.ldz + col]);
          if (a.D) a.D[(size_t)row * a.ldd + col] = gz;
          static_cast<__nv_bfloat16*>(a.H)[(size_t)row * a.ldh + col] = __float2bfloat16_rn(gz);
          if (a.HT) static_cast<__nv_bfloat16*>(a.HT)[(size_t)col * a.ldht + row] = __float2bfloat16_rn(gz);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, ncols);
}

cudaError_t launch_gemm_tc(const GemmArgs& a, int nsplit, cudaStream_t s) {
  if (a.N < 16 || a.N > kMaxN || (a.N % 16) || (a.lda % 8) || (a.ldb % 8) || a.K <= 0 || (a.K % 8) || a.M <= 0 ||
      a.kchunk <= 0 || (nsplit > 1 && (a.kchunk % kChunkK)) || nsplit < 1 || a.lda < a.K || a.ldb < a.K ||
      (reinterpret_cast<uintptr_t>(a.A) & 15) || (reinterpret_cast<uintptr_t>(a.B) & 15))
    return cudaErrorInvalidValue;
  cudaError_t e = raise_smem_limit(k_gemm_tc, kGemmSmem);
  if (e != cudaSuccess) return e;
  dim3 grid((a.M + kTileM - 1) / kTileM, nsplit);
  k_gemm_tc<<<grid, 128, kGemmSmem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ocn

// ---------------------------------------------------------------------------------------------
// Fused learned column closure: for 128 w-faces at a time, the raw features are computed from
// the state, normalised and rounded to BF16 straight into shared memory, the four layers run on
// the tensor cores with the activations kept on chip (TMEM accumulator -> bias + GELU in
// registers -> BF16 operand in shared memory), and the three fluxes are written out.  The
// weights are staged once per CTA; the CTAs are persistent over the tiles.
namespace ocn {
namespace {

constexpr int kCF = kColumnFeatures, kCH = 128, kCO = 16;
constexpr int kGroups = 4;                          // tiles in flight per CTA, one per group of 4 warps
constexpr int kGroupThreads = 128;                  // one thread per tile row (TMEM lane)
constexpr int kClosureThreads = kGroups * kGroupThreads;
constexpr int kSW1 = 0;                             // W1 [128][32]
constexpr int kSW2 = kSW1 + kCH * kCF * 2;          // W2 [128][128]
constexpr int kSW3 = kSW2 + kCH * kCH * 2;          // W3 [128][128]
constexpr int kSW4 = kSW3 + kCH * kCH * 2;          // W4 [16][128]
constexpr int kSB = kSW4 + kCO * kCH * 2;           // biases (3*128 + 16 floats)
constexpr int kSA = (kSB + (3 * kCH + kCO) * 4 + 1023) / 1024 * 1024;   // the groups' activation buffers
constexpr int kSAB = 128 * kCH * 2;                 // [128][128] BF16 per group; the features [128][32] live
                                                    // at its start until layer 1's MMA has read them
constexpr int kClosureSmem = kSA + kGroups * kSAB;
// one CTA per SM: the weights are staged once and shared by the four tiles in flight, which use
// all 512 TMEM columns (128 each), so the allocation never waits on another CTA of this kernel
static_assert(kClosureSmem + 1024 <= 227 * 1024 && 2 * kClosureSmem > 228 * 1024, "one CTA per SM");

// byte offset of element (r, c) of a [rows][K] K-major BF16 matrix in the no-swizzle core-matrix layout
__device__ __forceinline__ uint32_t cm_off(int r, int c, int K) {
  return (uint32_t)((r >> 3) * (K / 8) * 128 + (c >> 3) * 128 + (r & 7) * 16 + (c & 7) * 2);
}

__device__ __forceinline__ void stage_weights(unsigned char* dst, const __nv_bfloat16* W, int no, int ni) {
  const int cpr = ni / 8;
  for (int q = threadIdx.x; q < no * cpr; q += blockDim.x) {
    const int r = q / cpr, kc = q % cpr;
    *reinterpret_cast<uint4*>(dst + cm_off(r, 8 * kc, ni)) = *reinterpret_cast<const uint4*>(W + (size_t)r * ni + 8 * kc);
  }
}

// Issue one layer: D[128 x N] = A[128 x K] . B[N x K]^T (one thread), then commit to the barrier.
__device__ __forceinline__ void closure_layer_mma(uint32_t tmem, uint32_t a_addr, uint32_t b_addr, int K, int N,
                                                  uint64_t* bar) {
  tc_fence_after();
  const uint32_t sbo = (uint32_t)(K / 8) * 128;
  const uint32_t idesc = idesc_bf16(128, N);
  for (int s = 0; s < K / 16; ++s)
    mma_bf16(tmem, smem_desc(a_addr + s * 256, 128, sbo), smem_desc(b_addr + s * 256, 128, sbo), idesc, s > 0 ? 1u : 0u);
  mma_commit(bar);
}

// Barrier of one group of kGroupThreads threads (named barrier id >= 1), and its AND-reduction.
__device__ __forceinline__ void group_sync(int id) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(kGroupThreads) : "memory");
}
__device__ __forceinline__ bool group_sync_and(int id, bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.and.pred q, %2, %3, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(id), "n"(kGroupThreads)
      : "memory");
  return r != 0;
}

// One member's tile: its arguments and the tile's index within the member.
struct ClosureTile {
  const MlpClosureArgs* m;
  long long lt;
};

}  // namespace

// The fused closure network over 128-face tiles.  A CTA holds four tiles in flight, one per
// group of four warps (thread = tile row = TMEM lane, 128 TMEM columns per group), so that one
// group's tensor-core layer overlaps the others' epilogues; the groups share the staged weights
// and synchronise on their own named barriers.  Plain: the tiles of one model (`a`), grid
// stride over them.  Batched: the tiles of all members of `bt` (member m owns tiles
// [start[m], start[m+1])); `a` is member 0's arguments, whose network and feature normalisation
// every member shares; each tile reads its own member's columns and writes its fluxes with its
// own output scales.
template <bool kBatch>
__device__ __forceinline__ void mlp_closure_body(const MlpClosureArgs& a, const BatchTable& bt, const uint3 bid,
                                                 const uint3 gdim) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t bar[kGroups];
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int grp = warp >> 2, quad = warp & 3;
  const int row = quad * 32 + lane;                 // this thread's tile row and TMEM lane
  auto tiles_of = [](const ColumnArgs& c) -> long long {
    return (long long)(((size_t)c.Nx * c.Ny * (c.Nz + 1) + 127) / 128);
  };
  long long ntiles;
  if constexpr (kBatch) ntiles = (long long)__ldg(bt.start + bt.n);
  else ntiles = tiles_of(a.col);
  auto tile_of = [&](long long t) -> ClosureTile {
    if constexpr (kBatch) {
      const int m = batch_member(bt, (unsigned)t);
      return {reinterpret_cast<const MlpClosureArgs*>(bt.payload + (size_t)m * bt.stride), t - (long long)__ldg(bt.start + m)};
    } else {
      return {&a, t};
    }
  };
  if (warp == 0) tmem_alloc(&tmem_base, kGroups * kCH);
  if (tid == 0) {
    for (int g = 0; g < kGroups; ++g) mbar_init(&bar[g], 1);
    fence_barrier_init();
  }
  stage_weights(smem + kSW1, static_cast<const __nv_bfloat16*>(a.W[0]), kCH, kCF);
  stage_weights(smem + kSW2, static_cast<const __nv_bfloat16*>(a.W[1]), kCH, kCH);
  stage_weights(smem + kSW3, static_cast<const __nv_bfloat16*>(a.W[2]), kCH, kCH);
  stage_weights(smem + kSW4, static_cast<const __nv_bfloat16*>(a.W[3]), kCO, kCH);
  float* sbias = reinterpret_cast<float*>(smem + kSB);
  for (int q = tid; q < 3 * kCH + kCO; q += blockDim.x) sbias[q] = a.bias[q / kCH][q % kCH];
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base + (uint32_t)(grp * kCH) + ((uint32_t)(quad * 32) << 16);   // lanes of this warp
  const uint32_t tmem_mma = tmem_base + (uint32_t)(grp * kCH);
  unsigned char* act = smem + kSA + grp * kSAB;
  const uint32_t s0 = smem_u32(smem), sact = smem_u32(act);
  const int bar_id = 1 + grp;
  uint32_t phase = 0;
  bool ok = true;
  // raw column values of this thread's face for its features: b at levels k-3..k+2 (0-5), the
  // face depth (6), the column's mixed-layer depth (7), u at faces i and i+1 (8-13, 14-19) and v
  // at faces j and j+1 (20-25, 26-31) at levels k-3..k+2; then for the faces q = k-2..k+2 the
  // inverse spacing 1/dz_f (32-36) and the reference-profile step cref[q] - cref[q-1] (37-41);
  // 0 outside the column
  float raw[42];
  auto load_raw = [&](long long tt) {
#pragma unroll
    for (int m = 0; m < 42; ++m) raw[m] = 0.0f;
    if (tt >= ntiles) return;
    const ClosureTile ct = tile_of(tt);
    const ColumnArgs& c = ct.m->col;
    const size_t plane = (size_t)c.Nx * c.Ny, nsamp = plane * (c.Nz + 1);
    const size_t sidx = (size_t)ct.lt * 128 + row;
    if (sidx >= nsamp) return;
    const uint32_t s32 = (uint32_t)sidx, p32 = (uint32_t)plane;
    const int k = (int)(s32 / p32), cc = (int)(s32 - (uint32_t)k * p32);
    const int j = cc / c.Nx, i = cc - j * c.Nx;
    const int ip = (i + 1 == c.Nx) ? 0 : i + 1, jp = (j + 1 == c.Ny) ? 0 : j + 1;
#pragma unroll
    for (int m = 0; m < 6; ++m) {
      const int lev = k - 3 + m;
      if (lev >= 0 && lev < c.Nz) {
        raw[m] = __ldg(c.b + col_id(c, i, j, lev));
        raw[8 + m] = __ldg(c.u + col_id(c, i, j, lev));
        raw[14 + m] = __ldg(c.u + col_id(c, ip, j, lev));
        raw[20 + m] = __ldg(c.v + col_id(c, i, j, lev));
        raw[26 + m] = __ldg(c.v + col_id(c, i, jp, lev));
      }
    }
    raw[6] = __ldg(c.depth + k);
    raw[7] = __ldg(c.h + (size_t)j * c.Nx + i);
#pragma unroll
    for (int m = 0; m < 5; ++m) {
      const int q = k - 2 + m;
      if (q >= 1 && q < c.Nz) {
        raw[32 + m] = __ldg(c.rdzf + q);
        if (c.cref) raw[37 + m] = __ldg(c.cref + q) - __ldg(c.cref + q - 1);
      }
    }
  };
  const long long stride = (long long)kGroups * gdim.x;
  long long t = (long long)bid.x * kGroups + grp;
  load_raw(t);
  ClosureTile cur = {&a, 0};
  for (; t < ntiles && ok; t += stride) {
    cur = tile_of(t);
    const ColumnArgs& c = cur.m->col;
    const size_t plane = (size_t)c.Nx * c.Ny;
    const size_t nsamp = plane * (c.Nz + 1), NW = nsamp;
    // ---- the 20 features of this row (db/dz, dubar/dz, dvbar/dz at faces k-2..k+2, then Jb, f,
    //      N2bg, depth, h), normalised, rounded to BF16 and stored as four 16-byte chunks
    {
      const size_t sidx = (size_t)cur.lt * 128 + row;
      const bool valid = sidx < nsamp;
      float g[20];
#pragma unroll
      for (int m = 0; m < 20; ++m) g[m] = 0.0f;
      if (valid) {
        const int k = (int)((uint32_t)sidx / (uint32_t)plane);
        // face q = k - 2 + m lies between levels q - 1 (raw index m) and q (raw index m + 1)
#pragma unroll
        for (int m = 0; m < 5; ++m) {
          const int q = k - 2 + m;
          if (q >= 1 && q < c.Nz) {
            const float rz = raw[32 + m];
            float d = raw[m + 1] - raw[m];
            if (c.cref) d += raw[37 + m];
            g[m] = d * rz;
            g[5 + m] = 0.5f * ((raw[8 + m + 1] + raw[14 + m + 1]) - (raw[8 + m] + raw[14 + m])) * rz;
            g[10 + m] = 0.5f * ((raw[20 + m + 1] + raw[26 + m + 1]) - (raw[20 + m] + raw[26 + m])) * rz;
          }
        }
        g[15] = c.Jb; g[16] = c.f; g[17] = c.N2bg; g[18] = raw[6]; g[19] = raw[7];
      }
      uint32_t pk[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int f0 = 2 * q, f1 = 2 * q + 1;
        const float x0 = (valid && f0 < 20) ? (g[f0 < 20 ? f0 : 0] - a.mu[f0]) * a.inv_sigma[f0] : 0.0f;
        const float x1 = (valid && f1 < 20) ? (g[f1 < 20 ? f1 : 0] - a.mu[f1]) * a.inv_sigma[f1] : 0.0f;
        const __nv_bfloat162 h2 = __floats2bfloat162_rn(x0, x1);
        pk[q] = *reinterpret_cast<const uint32_t*>(&h2);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
        *reinterpret_cast<uint4*>(act + cm_off(row, 8 * q, kCF)) =
            make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
    }
    // ---- prefetch the next tile's raw values: they arrive while this tile's layers run
    load_raw(t + stride);
    // ---- four layers
    for (int l = 0; l < 4 && ok; ++l) {
      fence_proxy_async();
      tc_fence_before();
      group_sync(bar_id);
      if (row == 0) {
        const int K = (l == 0) ? kCF : kCH, N = (l == 3) ? kCO : kCH;
        const uint32_t bb = s0 + (l == 0 ? kSW1 : l == 1 ? kSW2 : l == 2 ? kSW3 : kSW4);
        closure_layer_mma(tmem_mma, sact, bb, K, N, &bar[grp]);
      }
      const bool done = mbar_wait_bounded(&bar[grp], phase);
      phase ^= 1u;
      tc_fence_after();
      ok = group_sync_and(bar_id, done);
      if (!ok) break;
      if (l < 3) {
        const float* bl = sbias + l * kCH;
        // 16-column chunks, the next chunk's TMEM load in flight while this one is processed
        uint32_t ra[16], rb[16];
        tmem_ld16_async(tmem, ra);
        tmem_wait16(ra);
#pragma unroll
        for (int cb = 0; cb < kCH; cb += 16) {
          if (cb + 16 < kCH) tmem_ld16_async(tmem + (uint32_t)(cb + 16), rb);
          float bv[16];                              // 16 biases, four 16-byte shared loads
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float4 b4 = reinterpret_cast<const float4*>(bl + cb)[q];
            bv[4 * q] = b4.x; bv[4 * q + 1] = b4.y; bv[4 * q + 2] = b4.z; bv[4 * q + 3] = b4.w;
          }
          uint32_t pk[8];
#pragma unroll
          for (int q = 0; q < 8; ++q)
            pk[q] = gelu_bf16x2(__floats2bfloat162_rn(__uint_as_float(ra[2 * q]) + bv[2 * q],
                                                      __uint_as_float(ra[2 * q + 1]) + bv[2 * q + 1]));
          *reinterpret_cast<uint4*>(act + cm_off(row, cb, kCH)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
          *reinterpret_cast<uint4*>(act + cm_off(row, cb + 8, kCH)) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
          if (cb + 16 < kCH) {
            tmem_wait16(rb);
#pragma unroll
            for (int q = 0; q < 16; ++q) ra[q] = rb[q];
          }
        }
      } else {
        float v[16];
        tmem_ld16(tmem, v);
        const size_t sidx = (size_t)cur.lt * 128 + row;
        if (sidx < nsamp) {
          const int k = (int)((uint32_t)sidx / (uint32_t)plane);
          const bool wall = (k == 0 || k == c.Nz);
          const float* b4 = sbias + 3 * kCH;
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            const float y = cur.m->scale[q] * (v[q] + b4[q]);
            cur.m->F[(size_t)q * NW + sidx] = wall ? 0.0f : (cur.m->relu ? fmaxf(y, 0.0f) : y);
          }
        }
      }
    }
  }
  if (!ok) {
    if (row == 0 && cur.m->status) atomicExch(cur.m->status, 1);
    mbar_wait_bounded(&bar[grp], phase ^ 1u);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem_base, kGroups * kCH);
}

__global__ void __launch_bounds__(kClosureThreads, 1) k_mlp_closure(const MlpClosureArgs a) {
  const BatchTable none = {nullptr, nullptr, nullptr, 0, 0};
  mlp_closure_body<false>(a, none, blockIdx, gridDim);
}

__global__ void __launch_bounds__(kClosureThreads, 1) k_mlp_closure_batched(const BatchTable bt) {
  mlp_closure_body<true>(*reinterpret_cast<const MlpClosureArgs*>(bt.payload), bt, blockIdx, gridDim);
}

cudaError_t launch_mlp_closure(const MlpClosureArgs& a, cudaStream_t s) {
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) nsm = 148;
  }
  cudaError_t e = raise_smem_limit(k_mlp_closure, kClosureSmem);
  if (e != cudaSuccess) return e;
  const size_t nsamp = (size_t)a.col.Nx * a.col.Ny * (a.col.Nz + 1);
  if (nsamp + 128 >= ((size_t)1 << 31)) return cudaErrorInvalidValue;    // 32-bit face indices
  const long long ntiles = (long long)((nsamp + 127) / 128);
  const long long need = (ntiles + kGroups - 1) / kGroups;
  const int grid = (int)(need < nsm ? need : nsm);
  if (LaunchRecorder* r = active_recorder()) {
    // batched: one tile space over the members, which share the network and the normalisation
    e = raise_smem_limit(k_mlp_closure_batched, kClosureSmem);
    if (e != cudaSuccess) return e;
    LaunchRecord rec;
    rec.fn = reinterpret_cast<const void*>(&k_mlp_closure_batched);
    rec.grid = dim3((unsigned)ntiles);
    rec.block = dim3(kClosureThreads);
    rec.smem = kClosureSmem;
    rec.persistent = nsm;
    rec.per_block = kGroups;
    rec.kclass = OCN_K_COLUMN_CLOSURE;
    rec.payload.assign(batch_stride(sizeof(a)), 0);
    memcpy(rec.payload.data(), &a, sizeof(a));
    const unsigned char* w0 = reinterpret_cast<const unsigned char*>(&a.W);
    rec.shared.assign(w0, w0 + (reinterpret_cast<const unsigned char*>(&a.scale) - w0));
    r->list.push_back(std::move(rec));
    return cudaSuccess;
  }
  k_mlp_closure<<<grid, kClosureThreads, kClosureSmem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ocn

// ---------------------------------------------------------------------------------------------
// Elementwise and reduction kernels of the training step.
namespace ocn {
namespace {

// X [M][n] FP32 -> Xb [Mp][n] BF16 and (optionally) XT [n][Mp] BF16; rows >= M are zero.
__global__ void k_mlp_input(const float* __restrict__ X, int M, int Mp, int n, __nv_bfloat16* Xb,
                            __nv_bfloat16* XT) {
  const size_t total = (size_t)Mp * n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(i % Mp), c = (int)(i / Mp);      // r fastest: XT stores coalesce
    const float x = (r < M) ? X[(size_t)r * n + c] : 0.0f;
    const __nv_bfloat16 b = __float2bfloat16_rn(x);
    Xb[(size_t)r * n + c] = b;
    if (XT) XT[(size_t)c * Mp + r] = b;
  }
}

// Output error of the masked mean-square loss L = (1/2M) sum_r sum_c mask_c (y - t)^2:
// dZ = mask (y - t) / M (FP32, BF16 and BF16 transposed), rows >= M zero; loss accumulated in FP64.
__global__ void k_mlp_loss(const float* __restrict__ Y, const float* __restrict__ T, const float* __restrict__ mask,
                           int M, int Mp, int n, float* dZf, __nv_bfloat16* dZb, __nv_bfloat16* dZT, double* loss) {
  const size_t total = (size_t)Mp * n;
  double acc = 0.0;
  const float invM = 1.0f / (float)M;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(i % Mp), c = (int)(i / Mp);
    float g = 0.0f;
    if (r < M) {
      const float e = Y[(size_t)r * n + c] - T[(size_t)r * n + c];
      g = mask[c] * e * invM;
      acc += 0.5 * (double)mask[c] * (double)e * (double)e;
    }
    dZf[(size_t)r * n + c] = g;
    const __nv_bfloat16 b = __float2bfloat16_rn(g);
    dZb[(size_t)r * n + c] = b;
    dZT[(size_t)c * Mp + r] = b;
  }
  if (loss) {
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc != 0.0) atomicAdd(loss, acc / (double)M);
  }
}

// Column partial sums of dZ [Mp][n] (bias gradients): part[b][c] over the rows of block b.
__global__ void k_mlp_colsum(const float* __restrict__ dZ, int Mp, int n, float* part) {
  __shared__ float red[8][33];
  const int c = blockIdx.x * 32 + threadIdx.x;
  float acc = 0.0f;
  if (c < n)
    for (int r = blockIdx.y * 8 + threadIdx.y; r < Mp; r += gridDim.y * 8) acc += dZ[(size_t)r * n + c];
  red[threadIdx.y][threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.y == 0 && c < n) {
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += red[j][threadIdx.x];
    part[(size_t)blockIdx.y * n + c] = s;
  }
}

// out[i] = sum_s part[s*count + i]
__global__ void k_mlp_reduce(const float* __restrict__ part, int nsplit, size_t count, float* out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int k = 0; k < nsplit; ++k) s += part[(size_t)k * count + i];
    out[i] = s;
  }
}

// Adam (Kingma & Ba 2015) with bias correction: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
// p -= lr (m c1) / (sqrt(v c2) + eps), c1 = 1/(1-b1^t), c2 = 1/(1-b2^t).
__global__ void k_mlp_adam(float* p, const float* __restrict__ g, float* m, float* v, size_t n, float lr, float b1,
                           float b2, float eps, float c1, float c2) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  }
}

// BF16 copies of one layer's weights: W [no][ni] and WT [ni][no].
__global__ void k_mlp_pack(const float* __restrict__ Wf, int no, int ni, __nv_bfloat16* W, __nv_bfloat16* WT) {
  const int total = no * ni;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int o = i / ni, k = i % ni;
    const __nv_bfloat16 b = __float2bfloat16_rn(Wf[i]);
    W[i] = b;
    WT[(size_t)k * no + o] = b;
  }
}

inline int grid_for(size_t n, int threads = 256) {
  size_t b = (n + threads - 1) / threads;
  return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

}  // namespace
}  // namespace ocn

// ---------------------------------------------------------------------------------------------
// The network object.
namespace {

constexpr int kMlpMaxLayers = OCN_MLP_MAX_LAYERS;
constexpr int kColsumBlocks = 64;

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

struct ocn_mlp {
  int L = 0;
  int sizes[kMlpMaxLayers + 1] = {0};
  int max_batch = 0, Mp_max = 0, nmax = 0;
  cudaStream_t stream = nullptr;
  size_t nparams = 0;
  size_t woff[kMlpMaxLayers] = {0}, boff[kMlpMaxLayers] = {0};
  size_t arena_bytes = 0;
  bool bound = false;
  long long t_adam = 0;
  int nsplit = 1;
  size_t part_elems = 0;
  // arena offsets
  size_t o_p, o_g, o_m, o_v, o_W[kMlpMaxLayers], o_WT[kMlpMaxLayers], o_Xb, o_XT, o_Z[kMlpMaxLayers],
      o_H[kMlpMaxLayers], o_HT[kMlpMaxLayers], o_Y, o_dZf[2], o_dZb[2], o_dZT[2], o_part, o_status, o_loss;
  char* arena = nullptr;
  template <typename T> T* at(size_t off) const { return reinterpret_cast<T*>(arena + off); }
};

namespace ocn {
bool mlp_closure_layers(const ocn_mlp* n, const void** W, const float** bias) {
  static const int shape[5] = {32, 128, 128, 128, 16};
  if (!n || !n->bound || n->L != 4) return false;
  for (int l = 0; l <= 4; ++l)
    if (n->sizes[l] != shape[l]) return false;
  for (int l = 0; l < 4; ++l) {
    W[l] = n->arena + n->o_W[l];
    bias[l] = reinterpret_cast<const float*>(n->arena + n->o_p) + n->boff[l];
  }
  return true;
}
}  // namespace ocn

namespace {

ocn_status mlp_fail(ocn_status st, const char* msg) { return ocn::set_last_error(st, msg); }

ocn_status mlp_cuda(cudaError_t e, const char* where) {
  if (e == cudaSuccess) return OCN_OK;
  char buf[256];
  snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
  return ocn::set_last_error(e == cudaErrorInvalidValue ? OCN_ERR_ARG : OCN_ERR_CUDA, buf);
}

// Split-K factor for the weight gradients: about two CTAs per SM over the sample range.
int pick_nsplit(int Mp) {
  int s = 296;
  const int maxs = Mp / 64;
  if (s > maxs) s = maxs;
  return s < 1 ? 1 : s;
}

ocn_status mlp_forward_impl(ocn_mlp* n, const float* X, int M, float* Y, bool train) {
  using namespace ocn;
  cudaStream_t s = n->stream;
  const int Mp = (M + 127) / 128 * 128;
  const int n0 = n->sizes[0];
  k_mlp_input<<<grid_for((size_t)Mp * n0), 256, 0, s>>>(X, M, Mp, n0, n->at<__nv_bfloat16>(n->o_Xb),
                                                           train ? n->at<__nv_bfloat16>(n->o_XT) : nullptr);
  ocn_status st = mlp_cuda(cudaGetLastError(), "mlp input");
  if (st) return st;
  const __nv_bfloat16* hin = n->at<__nv_bfloat16>(n->o_Xb);
  for (int l = 0; l < n->L; ++l) {
    GemmArgs g;
    memset(&g, 0, sizeof(g));
    g.A = hin; g.lda = n->sizes[l];
    g.B = n->at<__nv_bfloat16>(n->o_W[l]); g.ldb = n->sizes[l];
    g.M = Mp; g.N = n->sizes[l + 1]; g.K = n->sizes[l]; g.kchunk = (g.K + 63) / 64 * 64;
    g.bias = n->at<float>(n->o_p + sizeof(float) * n->boff[l]);
    g.status = n->at<int>(n->o_status);
    if (l < n->L - 1) {
      g.mode = 1;
      g.D = train ? n->at<float>(n->o_Z[l]) : nullptr; g.ldd = g.N;
      g.H = n->at<__nv_bfloat16>(n->o_H[l]); g.ldh = g.N;
      g.HT = train ? n->at<__nv_bfloat16>(n->o_HT[l]) : nullptr; g.ldht = Mp;
      hin = n->at<__nv_bfloat16>(n->o_H[l]);
    } else {
      g.mode = 2;
      g.M = M;                     // Y holds only the M real rows
      g.D = Y; g.ldd = g.N;
    }
    st = mlp_cuda(launch_gemm_tc(g, 1, s), "mlp forward gemm");
    if (st) return st;
  }
  return OCN_OK;
}

// Gradients of the masked mean-square loss into n->g (flat, the parameter layout).
ocn_status mlp_gradients_impl(ocn_mlp* n, const float* X, const float* T, const float* mask, int M) {
  using namespace ocn;
  cudaStream_t s = n->stream;
  const int Mp = (M + 127) / 128 * 128;
  const int L = n->L;
  ocn_status st = mlp_forward_impl(n, X, M, n->at<float>(n->o_Y), true);
  if (st) return st;
  const int nL = n->sizes[L];
  int cur = 0;
  k_mlp_loss<<<grid_for((size_t)Mp * nL), 256, 0, s>>>(n->at<float>(n->o_Y), T, mask, M, Mp, nL,
                                                         n->at<float>(n->o_dZf[cur]), n->at<__nv_bfloat16>(n->o_dZb[cur]),
                                                         n->at<__nv_bfloat16>(n->o_dZT[cur]), n->at<double>(n->o_loss));
  if ((st = mlp_cuda(cudaGetLastError(), "mlp loss"))) return st;
  const int nsplit = pick_nsplit(Mp);
  const int kchunk = (Mp / nsplit + 63) / 64 * 64;
  const int nsp = (Mp + kchunk - 1) / kchunk;
  for (int l = L - 1; l >= 0; --l) {
    const int no = n->sizes[l + 1], ni = n->sizes[l];
    // dW_l = dZ_l^T H_{l-1}: rows = outputs, columns = inputs, K = samples (split)
    GemmArgs g;
    memset(&g, 0, sizeof(g));
    g.A = n->at<__nv_bfloat16>(n->o_dZT[cur]); g.lda = Mp;
    g.B = (l == 0) ? n->at<__nv_bfloat16>(n->o_XT) : n->at<__nv_bfloat16>(n->o_HT[l - 1]); g.ldb = Mp;
    g.M = no; g.N = ni; g.K = Mp; g.kchunk = kchunk;
    g.mode = 0; g.D = n->at<float>(n->o_part); g.ldd = ni;
    g.status = n->at<int>(n->o_status);
    if ((st = mlp_cuda(launch_gemm_tc(g, nsp, s), "mlp weight-gradient gemm"))) return st;
    k_mlp_reduce<<<grid_for((size_t)no * ni), 256, 0, s>>>(n->at<float>(n->o_part), nsp, (size_t)no * ni,
                                                              n->at<float>(n->o_g) + n->woff[l]);
    if ((st = mlp_cuda(cudaGetLastError(), "mlp reduce"))) return st;
    // db_l = column sums of dZ_l
    dim3 cg((no + 31) / 32, kColsumBlocks);
    k_mlp_colsum<<<cg, dim3(32, 8), 0, s>>>(n->at<float>(n->o_dZf[cur]), Mp, no, n->at<float>(n->o_part));
    k_mlp_reduce<<<grid_for(no), 256, 0, s>>>(n->at<float>(n->o_part), kColsumBlocks, (size_t)no,
                                               n->at<float>(n->o_g) + n->boff[l]);
    if ((st = mlp_cuda(cudaGetLastError(), "mlp bias gradient"))) return st;
    if (l == 0) break;
    // dZ_{l-1} = (dZ_l W_l) * gelu'(Z_{l-1})
    GemmArgs b;
    memset(&b, 0, sizeof(b));
    b.A = n->at<__nv_bfloat16>(n->o_dZb[cur]); b.lda = no;
    b.B = n->at<__nv_bfloat16>(n->o_WT[l]); b.ldb = no;
    b.M = Mp; b.N = ni; b.K = no; b.kchunk = (no + 63) / 64 * 64;
    b.mode = 3; b.Z = n->at<float>(n->o_Z[l - 1]); b.ldz = ni;
    b.D = n->at<float>(n->o_dZf[cur ^ 1]); b.ldd = ni;
    b.H = n->at<__nv_bfloat16>(n->o_dZb[cur ^ 1]); b.ldh = ni;
    b.HT = n->at<__nv_bfloat16>(n->o_dZT[cur ^ 1]); b.ldht = Mp;
    b.status = n->at<int>(n->o_status);
    if ((st = mlp_cuda(launch_gemm_tc(b, 1, s), "mlp backward gemm"))) return st;
    cur ^= 1;
  }
  return OCN_OK;
}

ocn_status mlp_pack(ocn_mlp* n) {
  using namespace ocn;
  for (int l = 0; l < n->L; ++l) {
    const int no = n->sizes[l + 1], ni = n->sizes[l];
    k_mlp_pack<<<grid_for((size_t)no * ni), 256, 0, n->stream>>>(n->at<float>(n->o_p) + n->woff[l], no, ni,
                                                                   n->at<__nv_bfloat16>(n->o_W[l]),
                                                                   n->at<__nv_bfloat16>(n->o_WT[l]));
  }
  return mlp_cuda(cudaGetLastError(), "mlp pack");
}

ocn_status mlp_check(const ocn_mlp* n, int M) {
  if (!n) return mlp_fail(OCN_ERR_ARG, "null network");
  if (!n->bound) return mlp_fail(OCN_ERR_STATE, "arena not bound");
  if (M < 1 || M > n->max_batch) return mlp_fail(OCN_ERR_ARG, "batch size out of range");
  return OCN_OK;
}

ocn_status mlp_read_status(ocn_mlp* n) {
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, n->at<int>(n->o_status), sizeof(int), cudaMemcpyDeviceToHost, n->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
  if (e != cudaSuccess) return mlp_cuda(e, "mlp status");
  if (h) return mlp_fail(OCN_ERR_TIMEOUT, "a bounded wait for the tensor cores gave up");
  return OCN_OK;
}

}  // namespace

extern "C" {

ocn_status ocn_mlp_create(int nlayers, const int* sizes, int max_batch, void* stream, ocn_mlp** out) {
  if (!out || !sizes) return mlp_fail(OCN_ERR_ARG, "null pointer");
  *out = nullptr;
  if (nlayers < 1 || nlayers > kMlpMaxLayers) return mlp_fail(OCN_ERR_ARG, "layer count out of range");
  if (max_batch < 1 || max_batch > (1 << 26)) return mlp_fail(OCN_ERR_ARG, "max_batch out of range");
  for (int l = 0; l <= nlayers; ++l)
    if (sizes[l] < 16 || sizes[l] > 256 || sizes[l] % 16) return mlp_fail(OCN_ERR_ARG, "sizes must be 16..256, multiples of 16");
  ocn_mlp* n = new (std::nothrow) ocn_mlp();
  if (!n) return mlp_fail(OCN_ERR_OOM, "host allocation");
  n->L = nlayers;
  for (int l = 0; l <= nlayers; ++l) n->sizes[l] = sizes[l];
  n->max_batch = max_batch;
  n->Mp_max = (max_batch + 127) / 128 * 128;
  n->stream = reinterpret_cast<cudaStream_t>(stream);
  size_t np = 0;
  int nmax = 0;
  for (int l = 0; l < nlayers; ++l) {
    n->woff[l] = np; np += (size_t)sizes[l + 1] * sizes[l];
    n->boff[l] = np; np += sizes[l + 1];
  }
  for (int l = 0; l <= nlayers; ++l) nmax = sizes[l] > nmax ? sizes[l] : nmax;
  n->nparams = np;
  n->nmax = nmax;
  const size_t Mp = n->Mp_max;
  const int nsp = pick_nsplit((int)Mp) + 1;
  size_t maxo = 0;
  for (int l = 0; l < nlayers; ++l) maxo = std::max(maxo, (size_t)sizes[l + 1] * sizes[l]);
  n->part_elems = std::max((size_t)nsp * maxo, (size_t)kColsumBlocks * nmax);
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
  const size_t bf = 2;
  n->o_p = take(4 * np); n->o_g = take(4 * np); n->o_m = take(4 * np); n->o_v = take(4 * np);
  for (int l = 0; l < nlayers; ++l) {
    n->o_W[l] = take(bf * sizes[l + 1] * sizes[l]);
    n->o_WT[l] = take(bf * sizes[l + 1] * sizes[l]);
  }
  n->o_Xb = take(bf * Mp * sizes[0]);
  n->o_XT = take(bf * Mp * sizes[0]);
  for (int l = 0; l < nlayers - 1; ++l) {
    n->o_Z[l] = take(4 * Mp * sizes[l + 1]);
    n->o_H[l] = take(bf * Mp * sizes[l + 1]);
    n->o_HT[l] = take(bf * Mp * sizes[l + 1]);
  }
  n->o_Y = take(4 * Mp * sizes[nlayers]);
  for (int j = 0; j < 2; ++j) {
    n->o_dZf[j] = take(4 * Mp * nmax);
    n->o_dZb[j] = take(bf * Mp * nmax);
    n->o_dZT[j] = take(bf * Mp * nmax);
  }
  n->o_part = take(4 * n->part_elems);
  n->o_status = take(sizeof(int));
  n->o_loss = take(sizeof(double));
  n->arena_bytes = off;
  *out = n;
  return OCN_OK;
}

void ocn_mlp_destroy(ocn_mlp* n) { delete n; }

ocn_status ocn_mlp_arena_bytes(const ocn_mlp* n, size_t* bytes) {
  if (!n || !bytes) return mlp_fail(OCN_ERR_ARG, "null pointer");
  *bytes = n->arena_bytes;
  return OCN_OK;
}

ocn_status ocn_mlp_bind_arena(ocn_mlp* n, void* dev, size_t bytes) {
  if (!n || !dev) return mlp_fail(OCN_ERR_ARG, "null pointer");
  if (bytes < n->arena_bytes) return mlp_fail(OCN_ERR_ARG, "arena too small");
  if (reinterpret_cast<uintptr_t>(dev) & 255) return mlp_fail(OCN_ERR_ARG, "arena not 256-byte aligned");
  n->arena = static_cast<char*>(dev);
  cudaError_t e = cudaMemsetAsync(n->arena, 0, n->arena_bytes, n->stream);
  if (e != cudaSuccess) return mlp_cuda(e, "arena clear");
  n->bound = true;
  n->t_adam = 0;
  return OCN_OK;
}

ocn_status ocn_mlp_num_params(const ocn_mlp* n, size_t* count) {
  if (!n || !count) return mlp_fail(OCN_ERR_ARG, "null pointer");
  *count = n->nparams;
  return OCN_OK;
}

ocn_status ocn_mlp_set_params(ocn_mlp* n, const float* params, size_t count, int src_is_device) {
  if (!n || !params) return mlp_fail(OCN_ERR_ARG, "null pointer");
  if (!n->bound) return mlp_fail(OCN_ERR_STATE, "arena not bound");
  if (count != n->nparams) return mlp_fail(OCN_ERR_ARG, "parameter count mismatch");
  cudaError_t e = cudaMemcpyAsync(n->at<float>(n->o_p), params, 4 * count,
                                  src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, n->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->at<float>(n->o_m), 0, 4 * count, n->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->at<float>(n->o_v), 0, 4 * count, n->stream);
  if (e != cudaSuccess) return mlp_cuda(e, "set params");
  n->t_adam = 0;
  ocn_status st = mlp_pack(n);
  if (st != OCN_OK) return st;
  // host input: return with the BF16 copies in place, so that models on other streams see them
  if (!src_is_device && (e = cudaStreamSynchronize(n->stream)) != cudaSuccess) return mlp_cuda(e, "set params");
  return OCN_OK;
}

ocn_status ocn_mlp_get_params(ocn_mlp* n, float* params, size_t count, int dst_is_device) {
  if (!n || !params) return mlp_fail(OCN_ERR_ARG, "null pointer");
  if (!n->bound) return mlp_fail(OCN_ERR_STATE, "arena not bound");
  if (count != n->nparams) return mlp_fail(OCN_ERR_ARG, "parameter count mismatch");
  cudaError_t e = cudaMemcpyAsync(params, n->at<float>(n->o_p), 4 * count,
                                  dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, n->stream);
  if (e == cudaSuccess && !dst_is_device) e = cudaStreamSynchronize(n->stream);
  return mlp_cuda(e, "get params");
}

ocn_status ocn_mlp_forward(ocn_mlp* n, const float* X, int M, float* Y) {
  ocn_status st = mlp_check(n, M);
  if (st) return st;
  if (!X || !Y) return mlp_fail(OCN_ERR_ARG, "null pointer");
  return mlp_forward_impl(n, X, M, Y, false);
}

ocn_status ocn_mlp_gradients(ocn_mlp* n, const float* X, const float* T, const float* mask, int M, float* grads,
                             double* loss) {
  ocn_status st = mlp_check(n, M);
  if (st) return st;
  if (!X || !T || !mask) return mlp_fail(OCN_ERR_ARG, "null pointer");
  cudaError_t e = cudaMemsetAsync(n->at<double>(n->o_loss), 0, sizeof(double), n->stream);
  if (e != cudaSuccess) return mlp_cuda(e, "loss clear");
  if ((st = mlp_gradients_impl(n, X, T, mask, M))) return st;
  if (grads) {
    e = cudaMemcpyAsync(grads, n->at<float>(n->o_g), 4 * n->nparams, cudaMemcpyDeviceToDevice, n->stream);
    if (e != cudaSuccess) return mlp_cuda(e, "gradient copy");
  }
  if (loss) {
    e = cudaMemcpyAsync(loss, n->at<double>(n->o_loss), sizeof(double), cudaMemcpyDeviceToHost, n->stream);
    if (e != cudaSuccess) return mlp_cuda(e, "loss copy");
  }
  return mlp_read_status(n);
}

ocn_status ocn_mlp_adam(ocn_mlp* n, const float* grads, double lr, double beta1, double beta2, double eps) {
  if (!n) return mlp_fail(OCN_ERR_ARG, "null network");
  if (!n->bound) return mlp_fail(OCN_ERR_STATE, "arena not bound");
  if (!(lr >= 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0))
    return mlp_fail(OCN_ERR_ARG, "invalid Adam hyper-parameters");
  n->t_adam += 1;
  const double c1 = 1.0 / (1.0 - pow(beta1, (double)n->t_adam));
  const double c2 = 1.0 / (1.0 - pow(beta2, (double)n->t_adam));
  ocn::k_mlp_adam<<<ocn::grid_for(n->nparams), 256, 0, n->stream>>>(
      n->at<float>(n->o_p), grads ? grads : n->at<float>(n->o_g), n->at<float>(n->o_m), n->at<float>(n->o_v),
      n->nparams, (float)lr, (float)beta1, (float)beta2, (float)eps, (float)c1, (float)c2);
  ocn_status st = mlp_cuda(cudaGetLastError(), "adam");
  if (st) return st;
  return mlp_pack(n);
}

ocn_status ocn_mlp_train_step(ocn_mlp* n, const float* X, const float* T, const float* mask, int M, double lr,
                              double* loss) {
  ocn_status st = mlp_check(n, M);
  if (st) return st;
  if (!X || !T || !mask) return mlp_fail(OCN_ERR_ARG, "null pointer");
  cudaError_t e = cudaMemsetAsync(n->at<double>(n->o_loss), 0, sizeof(double), n->stream);
  if (e != cudaSuccess) return mlp_cuda(e, "loss clear");
  if ((st = mlp_gradients_impl(n, X, T, mask, M))) return st;
  if ((st = ocn_mlp_adam(n, nullptr, lr, 0.9, 0.999, 1e-8))) return st;
  if (loss) {
    e = cudaMemcpyAsync(loss, n->at<double>(n->o_loss), sizeof(double), cudaMemcpyDeviceToHost, n->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
    if (e != cudaSuccess) return mlp_cuda(e, "loss copy");
    return mlp_read_status(n);
  }
  return OCN_OK;
}

// The timeout path of the tensor-core kernels, for failure-detection tests: the GEMM kernel runs with
// its MMA and commit left out, so its bounded mbarrier wait runs out (about 0.5 s), the kernel records
// the failure in *status, waits once more (bounded) and frees its tensor memory.
ocn_status ocn_gemm_timeout_test(int* status, void* stream) {
  if (!status) return mlp_fail(OCN_ERR_ARG, "null pointer");
  static __nv_bfloat16* zeros = nullptr;
  static float* sink = nullptr;
  if (!zeros) {
    // a 128 x 64 BF16 operand and a 128 x 16 result, allocated once for this test entry only
    cudaError_t e = cudaMalloc(&zeros, 128 * 64 * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMalloc(&sink, 128 * 16 * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(zeros, 0, 128 * 64 * sizeof(__nv_bfloat16));
    if (e != cudaSuccess) return mlp_cuda(e, "timeout test buffers");
  }
  ocn::GemmArgs g;
  memset(&g, 0, sizeof(g));
  g.A = zeros; g.lda = 64;
  g.B = zeros; g.ldb = 64;
  g.M = 128; g.N = 16; g.K = 64; g.kchunk = 64;
  g.mode = 0; g.D = sink; g.ldd = 16; g.status = status;
  g.no_issue = 1;
  return mlp_cuda(ocn::launch_gemm_tc(g, 1, reinterpret_cast<cudaStream_t>(stream)), "timeout test");
}

// C entry point for the bare GEMM (used by the tests of the tensor-core path).
ocn_status ocn_gemm_bf16(int M, int N, int K, const void* A, int lda, const void* B, int ldb, float* D, int ldd,
                         int* status, void* stream) {
  if (!A || !B || !D) return mlp_fail(OCN_ERR_ARG, "null pointer");
  ocn::GemmArgs g;
  memset(&g, 0, sizeof(g));
  g.A = A; g.lda = lda;
  g.B = B; g.ldb = ldb;
  g.M = M; g.N = N; g.K = K; g.kchunk = (K + 63) / 64 * 64;
  g.mode = 0; g.D = D; g.ldd = ldd; g.status = status;
  if (ldd < N) return mlp_fail(OCN_ERR_ARG, "ldd < N");
  return mlp_cuda(ocn::launch_gemm_tc(g, 1, reinterpret_cast<cudaStream_t>(stream)), "gemm");
}

}  // extern "C"
