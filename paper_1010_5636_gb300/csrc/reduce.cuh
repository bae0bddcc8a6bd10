// Deterministic FP64 global reductions fused into the epilogue of any kernel.
//
// Each thread contributes K doubles.  A block reduces them with warp shuffles (fixed tree),
// writes K partials, and the last block to finish (found with one atomic counter after a
// memory fence) sums all partials in a fixed order and writes the K results.  The order of
// every addition depends only on gridDim and blockDim, so results are bit-reproducible.
// The counter returns to zero at the end, so the same counter serves the next launch on
// the same stream.
#pragma once
#include <cuda_runtime.h>

namespace nd {

struct ReduceSlot {
  double* partials;   // >= gridDim.x * K doubles
  double* result;     // K doubles
  unsigned* counter;  // one zero-initialised counter
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  return v;
}

// Reduce v[0..K) over the block; thread 0 returns the block sums in v.  blockDim.x must be a
// multiple of 32 and at most 1024.
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K]) {
  __shared__ double sm[32][K];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = warp_sum(v[k]);
  __syncthreads();  // sm may still be in use by a previous call
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) sm[warp][k] = v[k];
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = warp_sum(lane < nw ? sm[lane][k] : 0.0);
  }
}

// Block reduction + grid-level finish.  Every thread of every block must call it.  A launch
// that runs several independent reductions passes each one's block count and this block's
// index within it (and a slot with its own partials, counter and result).
template <int K>
__device__ __forceinline__ void grid_sum(double (&v)[K], const ReduceSlot& slot, int nblocks, int bid) {
  block_sum<K>(v);
  __shared__ bool last;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) slot.partials[bid * K + k] = v[k];
    __threadfence();
    unsigned t = atomicAdd(slot.counter, 1u);
    last = (t == (unsigned)nblocks - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s[K];
#pragma unroll
  for (int k = 0; k < K; ++k) s[k] = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x)
#pragma unroll
    for (int k = 0; k < K; ++k) s[k] += __ldcg(slot.partials + i * K + k);
  block_sum<K>(s);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) slot.result[k] = s[k];
    *slot.counter = 0u;
  }
}

template <int K>
__device__ __forceinline__ void grid_sum(double (&v)[K], const ReduceSlot& slot) {
  grid_sum<K>(v, slot, (int)gridDim.x, (int)blockIdx.x);
}

}  // namespace nd
