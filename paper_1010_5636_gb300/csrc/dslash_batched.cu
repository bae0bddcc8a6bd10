// One persistent launch of Q (Sec. 2.1) over several lattices of different sizes, each with
// several right-hand sides.  The work is a list of tiles (64 output sites of one RHS of one
// lattice); tiles are ordered lattice by lattice, site block by site block, RHS fastest, so the
// blocks that read one tile of links for all RHS of a lattice run back to back and the links
// come from DRAM once.  A grid of a few blocks per SM strides through the list.
#include "dslash.cuh"
#include "kernels.h"

namespace nd {

constexpr int BT_THREADS = 64;

// Q on one site: out(x) = gamma5 ((4+m) in(x) - 1/2 hop(in)(x)).
template <int P, int R>
__device__ __forceinline__ void q_site(const Geom& g, const char* links, const void* in, void* out, double diag, int p,
                                       int h) {
  using T = typename Traits<P>::real;
  const Site s = site_of(g, p, h);
  Spinor<T> acc;
  hopping_sum<P, R>(acc, g, s, p, h, links, in);
  Spinor<T> d;
  SpinorIO<P>::load(d, in, g.Vh, p, h);
  const T dg = (T)diag;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      cx<T> v = (T)(-0.5) * acc.s[a][c] + dg * d.s[a][c];
      acc.s[a][c] = a < 2 ? v : -v;
    }
  SpinorIO<P>::store(acc, out, g.Vh, p, h);
}

// FP64 needs its registers (about 250 per thread) and is bound by the FP64 pipe: 2 blocks per SM;
// FP32 and FP16 run 8 blocks per SM (128 registers).
template <int P, int R>
__global__ void __launch_bounds__(BT_THREADS, P == P64 ? 2 : 8) q_batched_kernel(const LatticeWork* work, int nlat,
                                                                                 int total) {
  __shared__ int begin[ND_MAX_BATCH + 1];
  if (threadIdx.x <= nlat) begin[threadIdx.x] = threadIdx.x < nlat ? work[threadIdx.x].tile_begin : total;
  __syncthreads();
  for (int t = blockIdx.x; t < total; t += gridDim.x) {
    int k = 0;
    while (k + 1 < nlat && t >= begin[k + 1]) ++k;
    const LatticeWork& w = work[k];
    const int local = t - begin[k];
    const int r = local % w.nrhs, blk = local / w.nrhs;
    const int i = blk * BT_THREADS + threadIdx.x;
    int p, h;
    both_parities_site(i, &p, &h);
    if (h >= w.g.Vh) continue;
    q_site<P, R>(w.g, w.links, static_cast<const char*>(w.in) + r * w.stride, static_cast<char*>(w.out) + r * w.stride,
                 w.diag, p, h);
  }
}

template <int P>
static cudaError_t launch_b1(int recon, const LatticeWork* work, int nlat, int total, int grid, cudaStream_t st) {
  switch (recon) {
    case 18: q_batched_kernel<P, 18><<<grid, BT_THREADS, 0, st>>>(work, nlat, total); break;
    case 12: q_batched_kernel<P, 12><<<grid, BT_THREADS, 0, st>>>(work, nlat, total); break;
    case 8: q_batched_kernel<P, 8><<<grid, BT_THREADS, 0, st>>>(work, nlat, total); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

int batched_tiles(int64_t V) { return (int)((V + BT_THREADS - 1) / BT_THREADS); }

cudaError_t launch_q_batched(int prec, int recon, const LatticeWork* work_dev, int nlat, int total, int grid,
                             cudaStream_t st) {
  if (total <= 0) return cudaSuccess;
  switch (prec) {
    case P64: return launch_b1<P64>(recon, work_dev, nlat, total, grid, st);
    case P32: return launch_b1<P32>(recon, work_dev, nlat, total, grid, st);
    case P16: return launch_b1<P16>(recon, work_dev, nlat, total, grid, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace nd
