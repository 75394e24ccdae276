// Batched launches for ensembles: the blocks of many members' grids in one launch.
//
// Every kernel of the time step is written as a body `K::run(args, block, grid)` that reads its
// block coordinates and grid size from arguments instead of blockIdx / gridDim.  The plain
// kernel passes its own; k_batched<K> runs a 1-D grid whose blocks are the concatenation of the
// members' grids: block b belongs to member m with start[m] <= b < start[m+1], is block
// b - start[m] of that member's grid (x fastest), and takes member m's arguments, which it first
// copies into shared memory.  One launch per kernel of the step then covers members of uneven
// sizes (a work list of (member, block) pairs), with the same arithmetic as the per-member
// launches.
//
// On the host, a thread-local recorder turns the launch functions into a record of (batched
// kernel, grid, block, shared memory, argument bytes), from which the ensemble builds the
// batched launches of its step graph.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <vector>

namespace ocn {

struct BatchTable {
  const unsigned* start;          // [n + 1] first flattened block of each member
  const uint3* dims;              // [n] member grid dimensions
  const unsigned char* payload;   // member m's arguments at payload + m * stride
  unsigned stride;                // bytes, a multiple of 16
  int n;
};

// member owning flattened block (or tile) b: the last m with start[m] <= b
__device__ __forceinline__ int batch_member(const BatchTable& t, unsigned b) {
  int lo = 0, hi = t.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(t.start + mid) <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <class K>
__global__ void __launch_bounds__(K::kThreads, K::kMinBlocks) k_batched(const BatchTable t) {
  typedef typename K::Payload P;
  constexpr int kWords = (int)((sizeof(P) + 15) / 16);
  __shared__ uint4 sp[kWords];
  const unsigned b = blockIdx.x;
  const int m = batch_member(t, b);
  const uint3 g = t.dims[m];
  const unsigned l = b - t.start[m];
  const uint3 bid = make_uint3(l % g.x, (l / g.x) % g.y, l / (g.x * g.y));
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nth = blockDim.x * blockDim.y * blockDim.z;
  const uint4* src = reinterpret_cast<const uint4*>(t.payload + (size_t)m * t.stride);
  for (int q = tid; q < kWords; q += nth) sp[q] = src[q];
  __syncthreads();
  K::run(*reinterpret_cast<const P*>(sp), bid, g);
}

// ---- host side
struct LaunchRecord {
  const void* fn = nullptr;       // the batched kernel
  dim3 grid, block;
  size_t smem = 0;
  int persistent = 0;             // > 0: grid-stride kernel over the members' blocks (tiles), launched
                                  // with min(ceil(total / per_block), persistent) blocks
  int per_block = 1;              // tiles a block of such a kernel holds at once
  int kclass = 0;
  int carveout = -1;              // >= 0: preferred shared-memory carveout (percent) of the kernel
  std::vector<unsigned char> payload;
  // arguments that must be equal across the members of one batched launch (compared bytewise)
  std::vector<unsigned char> shared;
};

struct LaunchRecorder {
  std::vector<LaunchRecord> list;
};

// The recorder active on this thread (null: launch functions launch).
LaunchRecorder*& active_recorder();

inline unsigned batch_stride(size_t bytes) { return (unsigned)((bytes + 15) / 16 * 16); }

// Record a launch of K on the active recorder; false (nothing recorded) when none is active.
template <class K>
bool record_launch(const typename K::Payload& p, dim3 grid, dim3 block, size_t smem, int kclass = 0) {
  LaunchRecorder* r = active_recorder();
  if (!r) return false;
  LaunchRecord rec;
  rec.fn = reinterpret_cast<const void*>(&k_batched<K>);
  rec.grid = grid;
  rec.block = block;
  rec.smem = smem;
  rec.kclass = kclass;
  rec.payload.assign(batch_stride(sizeof(p)), 0);
  memcpy(rec.payload.data(), &p, sizeof(p));
  r->list.push_back(std::move(rec));
  return true;
}

}  // namespace ocn
